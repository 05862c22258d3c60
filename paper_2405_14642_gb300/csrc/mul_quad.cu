// Batched classical multiplication c = a * b (Section 3, Eq. (1)).
//
// Partition (Section 3.1, Fig. 3, extended to full products of unequal
// lengths).  With na >= nb (operands are swapped otherwise) the result columns
// C_k = sum_{i+j=k} A_i B_j form a trapezoid: a rising region (columns
// [0, nb), k+1 terms), a plateau (nb terms) and a falling region.  Columns are
// grouped into windows of Q consecutive columns.  A thread owns one "unit":
//   * a rising pair: window r and its mirror R-1-r of the rising region,
//   * a plateau window, or
//   * a falling pair, mirrored the same way.
// Every unit then costs the same Q*(nb + Q) word products (the paper's
// mirror pairing of C_t with C_{M-1-t}, applied to each sloped region), so
// threads finish together and no update is atomic.
//
// Window accumulation.  A thread keeps the window value
//     S = sum_{q<Q} C_{k+q} 2^{32q}
// in Q+2 registers (it stays below 2^{32(Q+2)} since nb < 2^32) and adds
// A_i * (B_{k-i}, ..., B_{k-i+Q-1}) for each i with one mad.lo carry chain
// and one mad.hi carry chain (the low chain's final carry is counted in a
// register and folded in once per window): about two multiply-adds per word
// product.  Operands are read from shared memory as 16-byte vectors, Q at a
// time; the B window slides down one word per step and is assembled from two
// consecutive Q-word chunks held in registers.  Every unit is R + 1 blocks of
// Q steps, and its windows run as one loop over them, so the lanes of a warp
// share one trip count whatever their windows (quad_device.cuh, conv_unit).
//
// Recombination (Fig. 4/5).  Each window's low Q words go to L (the result
// range [k, k+Q)), its two high words to H at k+Q and k+Q+1; windows are Q
// apart, so L and H are each written once per word.  c = L + H is then an
// ordinary addition done with the Section 2 carry scan over threads in
// memory order (2Q words per thread), and the result is copied out.
#include <utility>

#include "bn_internal.h"
#include "quad_device.cuh"

namespace bn {
namespace {

using namespace quad;

struct QuadArgs {
    const uint32_t *a, *b;  // a is the longer operand (na >= nb)
    uint32_t *c;
    uint32_t na, nb;        // true limb counts
    uint32_t nap, nbp;      // padded: nbp = roundup(nb, 2Q), nap = max(roundup(na, Q), nbp)
    uint32_t nout;          // na + nb
    uint32_t units;         // nap / Q
    uint32_t group;         // threads per instance (power of two <= 32 or multiple of 32)
    uint32_t ipb;           // instances per CTA
    uint32_t inst_words;    // shared words per instance
    uint32_t ab_words;      // A region (B region follows at ab_words)
    uint32_t l_offset;      // L words (result low words before the L + H addition)
    uint32_t hc_offset;     // H spill words (2 per window)
    uint32_t vec_a, vec_b, vec_c;  // 16-byte aligned rows
    uint64_t batch;
};

// One product a*b (instance `inst` of p's rows) by the `group` threads of one
// slot; t is this thread's index in the slot and As the slot's shared words.
// Every thread of the CTA calls this together (it contains barriers).
template <int Q, bool COLS>
__device__ __forceinline__ void quad_instance(const QuadArgs &p, uint64_t inst, bool live,
                                              uint32_t *As, uint32_t *flags, uint32_t t) {
    uint32_t *Bs = As + p.ab_words;
    uint32_t *Ls = As + p.l_offset;     // L, then the H spill words
    uint32_t *Hc = As + p.hc_offset;

    // q1: stage the operands, zero-padded (B also below 0: logical [-Q, nbp + Q)).
    stage_row(As, p.a + inst * p.na, p.na, 0, p.nap, p.vec_a, live, t, p.group);
    for (uint32_t x = t; x < Q; x += p.group) Bs[phys(x)] = 0;
    stage_row(Bs, p.b + inst * p.nb, p.nb, Q, p.nbp + Q, p.vec_b, live, t, p.group);
    __syncthreads();

    // q2/q3: the products of this thread's unit (one or two windows); each
    // window publishes its low words to L and its two spill words to H
    // (Fig. 5) as soon as it is done.  L has its own region, so no barrier
    // is needed first and nothing stays live across windows.
    const uint32_t R = p.nbp / Q;               // windows in each sloped region
    const uint32_t plateau = (p.nap - p.nbp) / Q;
    if (!COLS && t < p.units) {
        Unit u{};
        if (t < R / 2) {                        // rising pair: t+1 and R-t blocks
            u = Unit{t * Q, 0, t + 1, (R - 1 - t) * Q, 0, R - t};
        } else if (t < R / 2 + plateau) {       // plateau window: R+1 blocks
            const uint32_t k0 = p.nbp + (t - R / 2) * Q;
            u = Unit{k0, k0 - p.nbp, R + 1, 0, 0, 0};
        } else {                                // falling pair: R-r and r+1 blocks
            const uint32_t r = t - R / 2 - plateau;
            const uint32_t k0 = p.nap + r * Q, k1 = p.nap + (R - 1 - r) * Q;
            u = Unit{k0, k0 - p.nbp, R - r, k1, k1 - p.nbp, r + 1};
        }
        conv_unit<Q>(As, Bs, u, [&](uint32_t k, const uint32_t (&acc)[Q + 2]) {
            BN_DEBUG_CHECK(k + Q <= p.nap + p.nbp && p.l_offset + phys(k + Q - 1) < p.hc_offset, kDbgIndex);
            st_words<Q>(Ls, k, acc);
            *reinterpret_cast<uint2 *>(Hc + 2 * (k / Q)) = make_uint2(acc[Q], acc[Q + 1]);
        });
    } else if (t < p.units) {
        uint32_t acc[Q + 2];
        auto publish = [&](uint32_t k) {
            BN_DEBUG_CHECK(k + Q <= p.nap + p.nbp && p.l_offset + phys(k + Q - 1) < p.hc_offset, kDbgIndex);
            st_words<Q>(Ls, k, acc);
            *reinterpret_cast<uint2 *>(Hc + 2 * (k / Q)) = make_uint2(acc[Q], acc[Q + 1]);
        };
        if (t < R / 2) {                        // rising pair
            const uint32_t k0 = t * Q, k1 = (R - 1 - t) * Q;
            conv_window<Q, COLS>(As, Bs, k0, 0, k0 + Q, acc);
            publish(k0);
            conv_window<Q, COLS>(As, Bs, k1, 0, k1 + Q, acc);
            publish(k1);
        } else if (t < R / 2 + plateau) {       // plateau window
            const uint32_t k0 = p.nbp + (t - R / 2) * Q;
            conv_window<Q, COLS>(As, Bs, k0, k0 - p.nbp, p.nbp + Q, acc);
            publish(k0);
        } else {                                // falling pair
            const uint32_t r = t - R / 2 - plateau;
            const uint32_t k0 = p.nap + r * Q, k1 = p.nap + (R - 1 - r) * Q;
            conv_window<Q, COLS>(As, Bs, k0, k0 - p.nbp, p.nap - (k0 - p.nbp), acc);
            publish(k0);
            conv_window<Q, COLS>(As, Bs, k1, k1 - p.nbp, p.nap - (k1 - p.nbp), acc);
            publish(k1);
        }
    }
    __syncthreads();

    // q4: c = L + H in memory order, 2Q words (windows 2t, 2t+1) per thread.
    constexpr int W2 = 2 * Q;
    const uint32_t nw = p.nap + p.nbp;
    const uint32_t base = 2 * Q * t;
    const bool owns = base < nw;
    uint32_t s[W2];
    uint32_t g = 0, pr = 0;
    if (owns) {
        ld_words<W2>(Ls, base, s);
        uint32_t h[W2];
#pragma unroll
        for (int q = 0; q < W2; ++q) h[q] = 0;
        if (t > 0) {
            const uint2 sp = *reinterpret_cast<const uint2 *>(Hc + 2 * (2 * t - 1));
            h[0] = sp.x; h[1] = sp.y;
        }
        const uint2 sp = *reinterpret_cast<const uint2 *>(Hc + 2 * (2 * t));
        h[Q] = sp.x; h[Q + 1] = sp.y;
        uint32_t carry = 0, all = 0xffffffffu;
#pragma unroll
        for (int q = 0; q < W2; ++q) {
            const uint64_t v = (uint64_t)s[q] + h[q] + carry;
            s[q] = (uint32_t)v;
            carry = (uint32_t)(v >> 32);
            all &= s[q];
        }
        g = carry;
        pr = all == 0xffffffffu;
    }
    const uint32_t cin = group_carry_in(g, pr, p.group, flags);
    if (owns) {
        uint32_t carry = cin;
#pragma unroll
        for (int q = 0; q < W2; ++q) {
            const uint64_t v = (uint64_t)s[q] + carry;
            s[q] = (uint32_t)v;
            carry = (uint32_t)(v >> 32);
        }
        st_words<W2>(Ls, base, s);
        // The exact product has na + nb words: every word of L + H from there
        // to its end nw is zero, and no carry leaves it (Fig. 5).  (When nw
        // is an odd number of windows, the last thread's 2Q words run past nw
        // into the spent H words of its own instance: those are not product
        // words.)
#pragma unroll
        for (int q = 0; q < W2; ++q) BN_DEBUG_CHECK(base + q < p.nout || base + q >= nw || s[q] == 0, kDbgSpill);
        BN_DEBUG_CHECK(base + W2 != nw || carry == 0, kDbgSpill);
    }
    __syncthreads();
    if (!live) return;
    uint32_t *crow = p.c + inst * p.nout;
    if (p.vec_c) {
        for (uint32_t x = 4 * t; x < p.nout; x += 4 * p.group)
            st_stream_v4(crow + x, *reinterpret_cast<const uint4 *>(Ls + phys(x)));
    } else {
        for (uint32_t x = t; x < p.nout; x += p.group) st_stream(crow + x, Ls[phys(x)]);
    }
}

template <int Q, bool COLS>
__global__ void __launch_bounds__(kQuadMaxThreads) k_mul_quad(QuadArgs p) {
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t slot = threadIdx.x / p.group, t = threadIdx.x - slot * p.group;
    const uint64_t inst = (uint64_t)blockIdx.x * p.ipb + slot;
    quad_instance<Q, COLS>(p, inst, inst < p.batch, smem + slot * p.inst_words,
                           smem + p.ipb * p.inst_words, t);
}

// Mixed-size batch: each slot of `group` threads takes one item from the work
// queue (a counter the CTA's first thread advances by ipb); items are sorted
// largest first, so slots of one CTA get similar sizes and the CTA-wide
// barriers cost little.  Geometry is computed per item on the device.
template <int Q>
__global__ void __launch_bounds__(kQuadMaxThreads)
    k_mul_quad_batch(const BatchItem *items, uint32_t count, uint32_t *queue,
                     const BatchBinding *bind, uint32_t group, uint32_t ipb, uint32_t inst_words) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint32_t first;
    const uint32_t slot = threadIdx.x / group, t = threadIdx.x - slot * group;
    uint32_t *As = smem + slot * inst_words, *flags = smem + ipb * inst_words;
    const uint32_t *A0 = bind->a, *B0 = bind->b;
    uint32_t *C0 = bind->c;
    for (;;) {
        __syncthreads();  // the previous items are stored before `first` moves on
        if (threadIdx.x == 0) first = atomicAdd(queue, ipb);
        __syncthreads();
        const uint32_t base = first;
        if (base >= count) break;
        const uint32_t idx = base + slot;
        const bool live = idx < count;
        BatchItem it{0, 0, 0, 1, 1};
        if (live) it = items[idx];
        const uint32_t *a = A0 + it.off_a, *b = B0 + it.off_b;
        uint32_t na = it.na, nb = it.nb;
        if (na < nb) {
            const uint32_t *tp = a; a = b; b = tp;
            const uint32_t tn = na; na = nb; nb = tn;
        }
        const Geometry g = geometry(na, nb, Q, 0);
        QuadArgs p{};
        p.a = a; p.b = b; p.c = C0 + it.off_c;
        p.na = na; p.nb = nb; p.nap = g.nap; p.nbp = g.nbp; p.nout = na + nb;
        p.units = g.units;
        p.group = group;
        p.ipb = ipb;
        p.inst_words = inst_words;
        p.ab_words = g.ab_words;
        p.l_offset = g.l_offset;
        p.hc_offset = g.hc_offset;
        p.vec_a = (na % 4 == 0) && ((uintptr_t)a % 16 == 0);
        p.vec_b = (nb % 4 == 0) && ((uintptr_t)b % 16 == 0);
        p.vec_c = (p.nout % 4 == 0) && ((uintptr_t)p.c % 16 == 0);
        p.batch = 1;
        quad_instance<Q, false>(p, 0, live, As, flags, t);
    }
}

// ---- lane form: one product per thread ------------------------------------
//
// For operands of at most kLaneMaxLimbs words a thread computes a whole
// product.  Its windows of Q columns run in order k = 0, Q, 2Q, ...; each
// window starts from the previous one's two top words, so its low Q words are
// final when it ends and go straight to memory: no L + H pass, no carry scan
// and no barrier.  The 32 lanes of a warp take 32 consecutive instances, so
// they run the same windows and blocks without divergence, which lets the
// two triangular blocks at the ends of a window (the Q x Q corners of the
// parallelogram where the B index leaves [0, nb)) run as shortened chains
// instead of multiplying zero padding.  Block (I, J) of window K pairs A's
// word block I with B's blocks J - 1 and J, J = K - I:
//   J = nb/Q   only block J - 1 (its top words): the falling triangle,
//   1 .. nb/Q - 1   a full block,
//   J = 0      only block 0 (its low words): the rising triangle.
// Operands sit in shared memory, one row per lane at a stride of an odd
// number of 16-byte units (conflict-free vector reads), staged by the warp
// with coalesced loads.
constexpr uint32_t kLaneQ = 8;
constexpr uint32_t kLaneThreads = 128;
constexpr uint32_t kLaneMaxLimbs = 128;     // longer operand, any form request
constexpr uint32_t kLaneAutoLimbs = 96;     // default form up to this size (faster than the
                                            // thread-group form at 8-96 limbs, slower at 128)
constexpr uint64_t kLaneMinBatch = 32 * 152;

struct LaneArgs {
    const uint32_t *a, *b;  // a is the longer operand (na >= nb)
    uint32_t *c;
    uint32_t na, nb, nap, nbp, nout;  // nap, nbp: rounded up to Q
    uint32_t stride;                  // shared words per lane row
    uint32_t vec_a, vec_b, vec_c;
    uint64_t batch;
};

__host__ __device__ inline uint32_t lane_stride(uint32_t nap, uint32_t nbp) {
    uint32_t s = roundup(nap + nbp, 4);
    if ((s / 4) % 2 == 0) s += 4;
    return s;
}

// Rows 0 .. nrows-1 of `rows` (n words each, contiguous in global memory) to
// shared rows S + r * stride + off, coalesced: unit x (a 16-byte vector, or a
// word) of the block is unit o of row r, x = r d + o, and (r, o) steps with x
// by 32 = (32 / d) d + 32 % d without a division per unit.
__device__ __forceinline__ void lane_stage(uint32_t *S, uint32_t stride, uint32_t off, const uint32_t *rows,
                                           uint32_t n, uint32_t nrows, bool vec, uint32_t lane) {
    const uint32_t d = vec ? n / 4 : n, total = nrows * d;
    const uint32_t sr = 32 / d, so = 32 - sr * d;
    uint32_t r = lane / d, o = lane - r * d;
    for (uint32_t x = lane; x < total; x += 32) {
        BN_DEBUG_CHECK(r < nrows && o < d, kDbgIndex);
        if (vec)
            *reinterpret_cast<uint4 *>(S + r * stride + off + 4 * o) = ld_stream_v4(rows + 4 * (uint64_t)x);
        else
            S[r * stride + off + o] = ld_stream(rows + x);
        r += sr;
        o += so;
        if (o >= d) {
            o -= d;
            ++r;
        }
    }
}

template <int N>
__device__ __forceinline__ void ld_lane(const uint32_t *S, uint32_t (&v)[N]) {
#pragma unroll
    for (int j = 0; j < N / 4; ++j) {
        const uint4 t = *reinterpret_cast<const uint4 *>(S + 4 * j);
        v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
    }
}

// A full block: steps s = 0 .. Q-1 with A word A[s] and the B window
// (lo[s..Q), hi[0..s)) reversed into place, as window_block does.
template <int Q>
__device__ __forceinline__ void lane_block(const uint32_t *A, const uint32_t (&lo)[Q], const uint32_t (&hi)[Q],
                                           uint32_t (&acc)[Q + 2], uint32_t &cnt) {
    uint32_t av[Q];
    ld_lane<Q>(A, av);
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        uint32_t w[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int idx = Q - s + q;
            w[q] = idx < Q ? lo[idx] : hi[idx - Q];
        }
        mac<Q>(acc, cnt, av[s], w);
    }
}

// Full blocks I = i0 .. i0+n-1 of a window (B blocks J0 = K - i0 downwards).
template <int Q>
__device__ __forceinline__ void lane_full(const uint32_t *A, const uint32_t *B, uint32_t n,
                                          uint32_t (&acc)[Q + 2], uint32_t &cnt) {
    uint32_t c0[Q], c1[Q];
    ld_lane<Q>(B, c1);
    for (uint32_t m = 0; m + 1 < n; m += 2) {
        ld_lane<Q>(B - Q, c0);
        lane_block<Q>(A, c0, c1, acc, cnt);
        ld_lane<Q>(B - 2 * Q, c1);
        lane_block<Q>(A + Q, c1, c0, acc, cnt);
        A += 2 * Q;
        B -= 2 * Q;
    }
    if (n & 1) {
        ld_lane<Q>(B - Q, c0);
        lane_block<Q>(A, c0, c1, acc, cnt);
    }
}

// Rising triangle (J = 0): step s multiplies A[s] by B[0 .. Q-s) into window
// words s .. Q-1 (low halves) and s+1 .. Q (high halves).
template <int Q, int... S>
__device__ __forceinline__ void lane_rising(const uint32_t *A, const uint32_t *B, uint32_t (&acc)[Q + 2],
                                            uint32_t &cnt, std::integer_sequence<int, S...>) {
    uint32_t av[Q], b[Q];
    ld_lane<Q>(A, av);
    ld_lane<Q>(B, b);
    ((lo_chain<Q - S>(acc + S, cnt, av[S], b), hi_chain<Q - S>(acc + S + 1, acc[Q + 1], av[S], b)), ...);
}

// Falling triangle (J = nb/Q, lo = B's last block): step s >= 1 multiplies
// A[s] by lo[Q-s .. Q) into window words 0 .. s-1 (low halves) and 1 .. s
// (high halves); each chain's carry out is held for its word and all are
// added in at the end.
template <int Q, int... S>
__device__ __forceinline__ void lane_falling(const uint32_t *A, const uint32_t *Blast, uint32_t (&acc)[Q + 2],
                                             std::integer_sequence<int, S...>) {
    static_assert(Q == 8, "the pending-carry fold is written for Q = 8");
    uint32_t av[Q], lo[Q], pend[Q + 1];
    ld_lane<Q>(A, av);
    ld_lane<Q>(Blast, lo);
#pragma unroll
    for (int q = 0; q <= Q; ++q) pend[q] = 0;
    ((lo_chain<S + 1>(acc, pend[S + 1], av[S + 1], lo + Q - 1 - S),
      hi_chain<S + 1>(acc + 1, pend[S + 2], av[S + 1], lo + Q - 1 - S)), ...);
    fold_pending8(acc, pend);
}

template <int Q>
__global__ void __launch_bounds__(kLaneThreads) k_mul_quad_lane(LaneArgs p) {
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t inst0 = ((uint64_t)blockIdx.x * (kLaneThreads / 32) + warp) * 32;
    if (inst0 >= p.batch) return;  // the whole warp is past the batch (no CTA barrier follows)
    const uint32_t nrows = p.batch - inst0 < 32 ? (uint32_t)(p.batch - inst0) : 32u;
    uint32_t *S = smem + warp * 32 * p.stride;
    lane_stage(S, p.stride, 0, p.a + inst0 * p.na, p.na, nrows, p.vec_a, lane);
    lane_stage(S, p.stride, p.nap, p.b + inst0 * p.nb, p.nb, nrows, p.vec_b, lane);
    uint32_t *A = S + lane * p.stride, *B = A + p.nap;
    for (uint32_t x = p.na; x < p.nap; ++x) A[x] = 0;
    for (uint32_t x = p.nb; x < p.nbp; ++x) B[x] = 0;
    __syncwarp();

    const uint32_t NA = p.nap / Q, NB = p.nbp / Q, KW = (p.nout + Q - 1) / Q;
    const bool live = lane < nrows;
    uint32_t *crow = p.c + (inst0 + lane) * p.nout;
    uint32_t acc[Q + 2];
#pragma unroll
    for (int q = 0; q < Q + 2; ++q) acc[q] = 0;
    for (uint32_t K = 0; K < KW; ++K) {
        // Carry in the previous window's two top words.
        acc[0] = acc[Q];
        acc[1] = acc[Q + 1];
#pragma unroll
        for (int q = 2; q < Q + 2; ++q) acc[q] = 0;
        uint32_t cnt = 0;
        if (K >= NB) lane_falling<Q>(A + (K - NB) * Q, B + (NB - 1) * Q, acc, std::make_integer_sequence<int, Q - 1>{});
        const uint32_t i0 = K + 1 > NB ? K + 1 - NB : 0, i1 = K < NA ? K : NA;
        if (i1 > i0) lane_full<Q>(A + i0 * Q, B + (K - i0) * Q, i1 - i0, acc, cnt);
        if (K < NA) lane_rising<Q>(A + K * Q, B, acc, cnt, std::make_integer_sequence<int, Q>{});
        fold_count<Q>(acc, cnt);
        const uint32_t k = K * Q;
#pragma unroll
        for (int q = 0; q < Q; ++q) BN_DEBUG_CHECK(k + q < p.nout || acc[q] == 0, kDbgSpill);
        if (!live) continue;
        if (p.vec_c) {
#pragma unroll
            for (int j = 0; j < Q / 4; ++j)
                if (k + 4 * j < p.nout)
                    st_stream_v4(crow + k + 4 * j, make_uint4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]));
        } else {
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (k + q < p.nout) st_stream(crow + k + q, acc[q]);
        }
    }
    // The exact product has nout words: nothing is carried out of the last window.
    BN_DEBUG_CHECK(acc[Q] == 0 && acc[Q + 1] == 0, kDbgSpill);
}

// Window size: 8 at every size.  Timed on GB300 against 4 over the sweep
// (1K-256K bits, CTA targets 128/256/512): 8 wins by 13-22% everywhere; 4
// stays available through bn_tuning.
uint32_t default_q(uint32_t na, uint32_t nb) {
    (void)na;
    (void)nb;
    return 8;
}

}  // namespace

BN_DEBUG_ACCESSOR(debug_word_quad)

bn_status quad_configure(QuadConfig &cfg, uint32_t na, uint32_t nb, const bn_tuning *t) {
    if (na == 0 || nb == 0) return BN_EINVAL;
    if (na > BN_MUL_MAX_LIMBS || nb > BN_MUL_MAX_LIMBS) return BN_EUNSUPPORTED;
    cfg = QuadConfig{};
    cfg.na = na;
    cfg.nb = nb;
    cfg.nout = na + nb;
    const uint32_t hi = na > nb ? na : nb, lo = na > nb ? nb : na;
    cfg.q = default_q(hi, lo);
    cfg.lane_auto = hi <= kLaneAutoLimbs;
    if (t) {
        if (t->reserved || t->variant > 3) return BN_EINVAL;
        if (t->variant) {
            cfg.cols = t->variant == 2;
            cfg.lane = t->variant == 3;
            cfg.lane_auto = false;
        }
        if (cfg.lane && (hi > kLaneMaxLimbs || t->limbs_per_thread || t->cta_threads)) return BN_EUNSUPPORTED;
        if (t->limbs_per_thread) {
            if (t->limbs_per_thread != 4 && t->limbs_per_thread != 8) return BN_EINVAL;
            cfg.q = t->limbs_per_thread;
        }
        if (t->cta_threads && (t->cta_threads % 32 || t->cta_threads > 1024)) return BN_EINVAL;
        cfg.cta_threads = t->cta_threads;
    }
    if (cfg.lane) {
        cfg.threads = 1;
        return BN_OK;
    }
    const Geometry g = geometry(hi, lo, cfg.q, cfg.cta_threads ? cfg.cta_threads : 256);
    if (g.group > kQuadMaxThreads) return BN_EUNSUPPORTED;  // needs a larger window
    if (g.smem > 227u * 1024u) return BN_EUNSUPPORTED;
    cfg.threads = g.group;
    return BN_OK;
}

cudaError_t quad_launch(const QuadConfig &cfg, const uint32_t *a, const uint32_t *b, uint32_t *c,
                        uint64_t batch, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    uint32_t na = cfg.na, nb = cfg.nb;
    if (na < nb) {  // the product is symmetric; make a the longer operand
        const uint32_t *tp = a; a = b; b = tp;
        const uint32_t tn = na; na = nb; nb = tn;
    }
    if (cfg.lane || (cfg.lane_auto && batch >= kLaneMinBatch)) {
        LaneArgs la{};
        la.a = a; la.b = b; la.c = c;
        la.na = na; la.nb = nb;
        la.nap = roundup(na, kLaneQ);
        la.nbp = roundup(nb, kLaneQ);
        la.nout = na + nb;
        la.stride = lane_stride(la.nap, la.nbp);
        la.vec_a = (na % 4 == 0) && ((uintptr_t)a % 16 == 0);
        la.vec_b = (nb % 4 == 0) && ((uintptr_t)b % 16 == 0);
        la.vec_c = (la.nout % 4 == 0) && ((uintptr_t)c % 16 == 0);
        la.batch = batch;
        const uint64_t grid = (batch + kLaneThreads - 1) / kLaneThreads;
        if (grid > 0x7fffffffull) return cudaErrorInvalidConfiguration;
        const uint32_t smem = kLaneThreads * la.stride * 4;
        cudaError_t e = allow_max_smem((const void *)k_mul_quad_lane<kLaneQ>);
        if (e != cudaSuccess) return e;
        k_mul_quad_lane<kLaneQ><<<(unsigned)grid, kLaneThreads, smem, st>>>(la);
        return cudaGetLastError();
    }
    const Geometry g = geometry(na, nb, cfg.q, cfg.cta_threads ? cfg.cta_threads : 256);
    QuadArgs args{};
    args.a = a; args.b = b; args.c = c;
    args.na = na; args.nb = nb; args.nap = g.nap; args.nbp = g.nbp;
    args.nout = na + nb;
    args.units = g.units;
    args.group = g.group;
    args.ipb = g.ipb;
    args.inst_words = g.inst_words;
    args.ab_words = g.ab_words;
    args.l_offset = g.l_offset;
    args.hc_offset = g.hc_offset;
    args.vec_a = (na % 4 == 0) && ((uintptr_t)a % 16 == 0);
    args.vec_b = (nb % 4 == 0) && ((uintptr_t)b % 16 == 0);
    args.vec_c = (args.nout % 4 == 0) && ((uintptr_t)c % 16 == 0);
    args.batch = batch;
    const uint64_t grid = (batch + g.ipb - 1) / g.ipb;
    if (grid > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    const void *kern = cfg.q == 4 ? (cfg.cols ? (const void *)k_mul_quad<4, true> : (const void *)k_mul_quad<4, false>)
                                  : (cfg.cols ? (const void *)k_mul_quad<8, true> : (const void *)k_mul_quad<8, false>);
    if ((e = allow_max_smem(kern)) != cudaSuccess) return e;
    if (cfg.q == 4) {
        if (cfg.cols) k_mul_quad<4, true><<<(unsigned)grid, g.block, g.smem, st>>>(args);
        else k_mul_quad<4, false><<<(unsigned)grid, g.block, g.smem, st>>>(args);
    } else {
        if (cfg.cols) k_mul_quad<8, true><<<(unsigned)grid, g.block, g.smem, st>>>(args);
        else k_mul_quad<8, false><<<(unsigned)grid, g.block, g.smem, st>>>(args);
    }
    return cudaGetLastError();
}

bn_status quad_batch_class(QuadClass &qc, uint32_t q, uint32_t n_max, uint32_t cta_target) {
    if (n_max == 0 || n_max > BN_MUL_MAX_LIMBS || (q != 4 && q != 8)) return BN_EINVAL;
    if (cta_target == 0 || cta_target > 1024) return BN_EINVAL;
    const Geometry g = geometry(n_max, n_max, q, cta_target);
    if (g.group > kQuadMaxThreads) return BN_EUNSUPPORTED;
    qc = QuadClass{};
    qc.q = q;
    qc.n_max = n_max;
    qc.group = g.group;
    qc.ipb = g.ipb;
    qc.block = g.block;
    qc.inst_words = g.inst_words;
    qc.smem = g.smem;
    const void *kern = q == 4 ? (const void *)k_mul_quad_batch<4> : (const void *)k_mul_quad_batch<8>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = allow_max_smem(kern);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)qc.block, qc.smem);
    if (e != cudaSuccess) return BN_ECUDA;
    if (per_sm == 0) return BN_EUNSUPPORTED;
    qc.grid = (uint32_t)(sms * per_sm);
    return BN_OK;
}

cudaError_t quad_batch_launch(const QuadClass &qc, const BatchItem *items, uint32_t count,
                              uint32_t *queue, const BatchBinding *bind, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const uint32_t need = (count + qc.ipb - 1) / qc.ipb;
    const uint32_t grid = need < qc.grid ? need : qc.grid;
    if (qc.q == 4)
        k_mul_quad_batch<4><<<grid, qc.block, qc.smem, st>>>(items, count, queue, bind, qc.group,
                                                             qc.ipb, qc.inst_words);
    else
        k_mul_quad_batch<8><<<grid, qc.block, qc.smem, st>>>(items, count, queue, bind, qc.group,
                                                             qc.ipb, qc.inst_words);
    return cudaGetLastError();
}

}  // namespace bn
