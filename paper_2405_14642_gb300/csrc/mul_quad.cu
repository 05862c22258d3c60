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
    if (t) {
        if (t->reserved || t->variant > 2) return BN_EINVAL;
        if (t->variant) cfg.cols = t->variant == 2;
        if (t->limbs_per_thread) {
            if (t->limbs_per_thread != 4 && t->limbs_per_thread != 8) return BN_EINVAL;
            cfg.q = t->limbs_per_thread;
        }
        if (t->cta_threads && (t->cta_threads % 32 || t->cta_threads > 1024)) return BN_EINVAL;
        cfg.cta_threads = t->cta_threads;
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
