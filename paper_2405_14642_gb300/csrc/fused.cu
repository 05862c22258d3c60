// Section 6's fused programs and the paper's same-length product, all with
// results modulo 2^(32 n) for n-limb operands (the paper keeps results the
// input length, Section 2):
//   * bn_mul_low: c = a*b mod 2^(32n).  Only the columns 0..n-1 are needed,
//     the rising triangle of Fig. 3, and its mirror pairing (thread t owns
//     windows t and R-1-t) balances it exactly: half the work of a full
//     product.  The window spills that land at or above column n are dropped.
//   * bn_poly: c = (a*a + b)*(b*b + b) + a*b mod 2^(32n), one kernel; the
//     four low products and three additions of an instance run in one slot of
//     threads with every intermediate in shared memory (block-level fusion).
//   * bn_add6: six dependent additions x_{k+1} = x_k + x_{k-1} from x_0 = a,
//     x_1 = b (so c = x_7 = 8a + 13b mod 2^(32n)), intermediates in registers.
#include "bn_internal.h"
#include "quad_device.cuh"

namespace bn {
namespace {

using namespace quad;

// Low np words of A*B.  A is staged at phys(x), B at phys(x + Q) with zeros in
// [-Q, 0); np is a multiple of 2Q.  Threads t < np/(2Q) of the slot own one
// mirrored pair of windows each; the sum L + H (carry out of the top dropped)
// goes to `out` (padded layout).  Ends with a barrier.
template <int Q>
__device__ void low_product(const uint32_t *As, const uint32_t *Bs, uint32_t np, uint32_t *Ls,
                            uint32_t *Hc, uint32_t *out, uint32_t *flags, uint32_t t, uint32_t group) {
    const uint32_t R = np / Q;
    if (t < R / 2) {
        uint32_t acc[Q + 2];
        const uint32_t k0 = t * Q, k1 = (R - 1 - t) * Q;
        conv_window<Q, false>(As, Bs, k0, 0, k0 + Q, acc);
        st_words<Q>(Ls, k0, acc);
        *reinterpret_cast<uint2 *>(Hc + 2 * (k0 / Q)) = make_uint2(acc[Q], acc[Q + 1]);
        conv_window<Q, false>(As, Bs, k1, 0, k1 + Q, acc);
        st_words<Q>(Ls, k1, acc);
        *reinterpret_cast<uint2 *>(Hc + 2 * (k1 / Q)) = make_uint2(acc[Q], acc[Q + 1]);
    }
    __syncthreads();
    constexpr int W2 = 2 * Q;
    const uint32_t base = 2 * Q * t;
    const bool owns = base < np;
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
    const uint32_t cin = group_carry_in(g, pr, group, flags);
    if (owns) {
        uint32_t carry = cin;
#pragma unroll
        for (int q = 0; q < W2; ++q) {
            const uint64_t v = (uint64_t)s[q] + carry;
            s[q] = (uint32_t)v;
            carry = (uint32_t)(v >> 32);
        }
        st_words<W2>(out, base, s);
    }
    __syncthreads();
}

// out = (X + Y) mod 2^(32 np), X in shared memory (padded), Y in shared memory
// (padded) or a global row of n words (zero-extended); 2Q words per thread.
// `out` may be X.  Ends with a barrier.
template <int Q>
__device__ void add_words(const uint32_t *X, const uint32_t *Ys, const uint32_t *Yg, uint32_t n,
                          uint32_t np, uint32_t *out, uint32_t *flags, uint32_t t, uint32_t group) {
    constexpr int W2 = 2 * Q;
    const uint32_t base = 2 * Q * t;
    const bool owns = base < np;
    uint32_t s[W2];
    uint32_t g = 0, pr = 0;
    if (owns) {
        uint32_t y[W2];
        ld_words<W2>(X, base, s);
        if (Ys) {
            ld_words<W2>(Ys, base, y);
        } else {
#pragma unroll
            for (int q = 0; q < W2; ++q) y[q] = base + q < n ? Yg[base + q] : 0u;
        }
        uint32_t carry = 0, all = 0xffffffffu;
#pragma unroll
        for (int q = 0; q < W2; ++q) {
            const uint64_t v = (uint64_t)s[q] + y[q] + carry;
            s[q] = (uint32_t)v;
            carry = (uint32_t)(v >> 32);
            all &= s[q];
        }
        g = carry;
        pr = all == 0xffffffffu;
    }
    const uint32_t cin = group_carry_in(g, pr, group, flags);
    if (owns) {
        uint32_t carry = cin;
#pragma unroll
        for (int q = 0; q < W2; ++q) {
            const uint64_t v = (uint64_t)s[q] + carry;
            s[q] = (uint32_t)v;
            carry = (uint32_t)(v >> 32);
        }
        st_words<W2>(out, base, s);
    }
    __syncthreads();
}

// Copies np words between padded shared regions (B's offset Q is applied by
// the caller through `off`).
__device__ __forceinline__ void copy_words(const uint32_t *src, uint32_t *dst, uint32_t off,
                                           uint32_t np, uint32_t t, uint32_t group) {
    for (uint32_t x = t; x < np; x += group) dst[phys(x + off)] = src[phys(x)];
}

struct LowArgs {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t n, np, group, ipb, slot_words, vec_a, vec_b;
    uint32_t a_words, b_words, l_words;  // region sizes in words
    uint64_t batch;
};

template <int Q>
__device__ __forceinline__ void stage_pair(uint32_t *As, uint32_t *Bs, const uint32_t *ra, const uint32_t *rb,
                                           const LowArgs &p, bool live, uint32_t t) {
    stage_row(As, ra, p.n, 0, p.np, p.vec_a, live, t, p.group);
    for (uint32_t x = t; x < Q; x += p.group) Bs[phys(x)] = 0;
    stage_row(Bs, rb, p.n, Q, p.np + Q, p.vec_b, live, t, p.group);
    __syncthreads();
}

__device__ __forceinline__ void store_out(const uint32_t *S, uint32_t *crow, uint32_t n, bool live,
                                          uint32_t t, uint32_t group) {
    if (!live) return;
    for (uint32_t x = t; x < n; x += group) st_stream(crow + x, S[phys(x)]);
}

// c = a*b mod 2^(32n).
template <int Q>
__global__ void __launch_bounds__(1024) k_mul_low(LowArgs p) {
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t slot = threadIdx.x / p.group, t = threadIdx.x - slot * p.group;
    const uint64_t inst = (uint64_t)blockIdx.x * p.ipb + slot;
    const bool live = inst < p.batch;
    uint32_t *As = smem + slot * p.slot_words, *Bs = As + p.a_words, *Ls = Bs + p.b_words;
    uint32_t *Hc = Ls + p.l_words, *flags = smem + p.ipb * p.slot_words;
    stage_pair<Q>(As, Bs, p.a + inst * p.n, p.b + inst * p.n, p, live, t);
    low_product<Q>(As, Bs, p.np, Ls, Hc, Ls, flags, t, p.group);
    store_out(Ls, p.c + inst * p.n, p.n, live, t, p.group);
}

// c = (a*a + b)*(b*b + b) + a*b mod 2^(32n), all in one slot.
template <int Q>
__global__ void __launch_bounds__(1024) k_poly(LowArgs p) {
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t slot = threadIdx.x / p.group, t = threadIdx.x - slot * p.group;
    const uint64_t inst = (uint64_t)blockIdx.x * p.ipb + slot;
    const bool live = inst < p.batch;
    uint32_t *As = smem + slot * p.slot_words, *Bs = As + p.a_words, *Ls = Bs + p.b_words;
    uint32_t *T1 = Ls + p.l_words, *T2 = T1 + p.l_words, *Hc = T2 + p.l_words;
    uint32_t *flags = smem + p.ipb * p.slot_words;
    const uint32_t *ra = p.a + inst * p.n, *rb = p.b + inst * p.n;
    // T1 = a*a + b
    stage_pair<Q>(As, Bs, ra, ra, p, live, t);
    low_product<Q>(As, Bs, p.np, Ls, Hc, T1, flags, t, p.group);
    add_words<Q>(T1, nullptr, live ? rb : ra, live ? p.n : 0, p.np, T1, flags, t, p.group);
    // T2 = b*b + b
    stage_pair<Q>(As, Bs, rb, rb, p, live, t);
    low_product<Q>(As, Bs, p.np, Ls, Hc, T2, flags, t, p.group);
    add_words<Q>(T2, nullptr, live ? rb : ra, live ? p.n : 0, p.np, T2, flags, t, p.group);
    // T1 = T1 * T2
    copy_words(T1, As, 0, p.np, t, p.group);
    copy_words(T2, Bs, Q, p.np, t, p.group);
    __syncthreads();
    low_product<Q>(As, Bs, p.np, Ls, Hc, T1, flags, t, p.group);
    // T2 = a*b, then c = T1 + T2
    stage_pair<Q>(As, Bs, ra, rb, p, live, t);
    low_product<Q>(As, Bs, p.np, Ls, Hc, T2, flags, t, p.group);
    add_words<Q>(T1, T2, nullptr, p.n, p.np, T1, flags, t, p.group);
    store_out(T1, p.c + inst * p.n, p.n, live, t, p.group);
}

// ---- 6-Add ------------------------------------------------------------------

template <int VEC>
__device__ __forceinline__ void load_chunk(const uint32_t *row, uint32_t j, bool in, uint32_t (&v)[VEC]) {
    if constexpr (VEC == 4) {
        const uint4 t = in ? ld_stream_v4(row + 4 * j) : make_uint4(0, 0, 0, 0);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        v[0] = in ? ld_stream(row + j) : 0u;
    }
}

template <int VEC>
__device__ __forceinline__ void store_chunk(uint32_t *row, uint32_t j, const uint32_t (&v)[VEC]) {
    if constexpr (VEC == 4) st_stream_v4(row + 4 * j, make_uint4(v[0], v[1], v[2], v[3]));
    else st_stream(row + j, v[0]);
}

struct Add6Args {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t n, chunks, group, log2_group, warps_per_team, teams_per_cta;
    uint64_t batch;
};

// Instances of at most 32 chunks: `group` lanes (a power of two) per instance,
// one chunk per lane, each addition one segmented warp scan.
template <int VEC>
__global__ void __launch_bounds__(256) k_add6_sub(Add6Args p) {
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t inst = gt >> p.log2_group;
    const uint32_t j = (uint32_t)gt & (p.group - 1);
    const bool live = inst < p.batch && j < p.chunks;
    uint32_t x[2][VEC];
    load_chunk<VEC>(p.a + inst * p.n, j, live, x[0]);
    load_chunk<VEC>(p.b + inst * p.n, j, live, x[1]);
    // Step k overwrites x_{k-1} (set k % 2) with x_{k+1} = x_k + x_{k-1}.
#pragma unroll
    for (int step = 0; step < 6; ++step) {
        uint32_t(&z)[VEC] = x[step % 2];
        const uint32_t g = chunk_add<VEC>(z, x[(step + 1) % 2], z);
        const uint32_t cin = group_carry_in(g, chunk_all_ones<VEC>(z), p.group, nullptr);
        chunk_inc<VEC>(z, cin);
    }
    if (live) store_chunk<VEC>(p.c + inst * p.n, j, x[1]);
}

// z = z + y over the team's chunks (R rows of 32 chunks of VEC limbs per
// warp), carries resolved across the team as in k_add_team; no carry out.
// The warp summaries alternate between two buffers, so one barrier per
// addition suffices: a warp writes buffer k % 2 only after passing addition
// k-1's barrier, which every reader of addition k-2 reached after its read.
template <int VEC, int R>
__device__ __forceinline__ void team_add(uint32_t (&z)[R][VEC], const uint32_t (&y)[R][VEC],
                                         uint32_t w, uint32_t team_in_cta, uint32_t warps_per_team,
                                         uint32_t *warp_flags) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t gbits = 0, pbits = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        gbits |= chunk_add<VEC>(z[r], y[r], z[r]) << r;
        pbits |= chunk_all_ones<VEC>(z[r]) << r;
    }
    uint32_t wg = 0, wp = 1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const RowFlags f{__ballot_sync(FULL_MASK, (gbits >> r) & 1u), __ballot_sync(FULL_MASK, (pbits >> r) & 1u)};
        uint32_t rg;
        row_carries(f, 0, rg);
        carry_compose(wg, wp, rg, f.P == FULL_MASK);
    }
    if (lane == 0) warp_flags[warp] = wg | (wp << 1);
    __syncthreads();
    const uint32_t sw = lane < warps_per_team ? warp_flags[team_in_cta * warps_per_team + lane] : 0u;
    const RowFlags fw{__ballot_sync(FULL_MASK, sw & 1u), __ballot_sync(FULL_MASK, (sw >> 1) & 1u)};
    uint32_t unused;
    uint32_t cin = (row_carries(fw, 0, unused) >> w) & 1u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const RowFlags f{__ballot_sync(FULL_MASK, (gbits >> r) & 1u), __ballot_sync(FULL_MASK, (pbits >> r) & 1u)};
        uint32_t cout;
        const uint32_t ci = (row_carries(f, cin, cout) >> lane) & 1u;
        cin = cout;
        chunk_inc<VEC>(z[r], ci);
    }
}

// Instances of more than 32 chunks: a team of whole warps per instance.
template <int VEC, int R>
__global__ void __launch_bounds__(512) k_add6_team(Add6Args p) {
    __shared__ uint32_t warp_flags[2][16];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t team_in_cta = warp / p.warps_per_team, w = warp - team_in_cta * p.warps_per_team;
    const uint64_t inst = (uint64_t)blockIdx.x * p.teams_per_cta + team_in_cta;
    const bool live = inst < p.batch;
    const uint32_t j0 = w * R * 32 + lane;
    uint32_t x[2][R][VEC];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t j = j0 + r * 32;
        const bool in = live && j < p.chunks;
        load_chunk<VEC>(p.a + inst * p.n, j, in, x[0][r]);
        load_chunk<VEC>(p.b + inst * p.n, j, in, x[1][r]);
    }
#pragma unroll
    for (int step = 0; step < 6; ++step)
        team_add<VEC, R>(x[step % 2], x[(step + 1) % 2], w, team_in_cta, p.warps_per_team,
                         warp_flags[step % 2]);
    if (!live) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t j = j0 + r * 32;
        if (j < p.chunks) store_chunk<VEC>(p.c + inst * p.n, j, x[1][r]);
    }
}

// ---- host side ---------------------------------------------------------------

struct LowGeometry {
    uint32_t q, np, group, ipb, block, slot_words, a_words, b_words, l_words, smem;
};

LowGeometry low_geometry(uint32_t n, bool poly) {
    LowGeometry g{};
    // Window size from GB300 timings over the 1K..256K-bit sweep: Q = 4 puts
    // twice the threads on an instance for the same shared memory, which wins
    // where shared memory bounds the resident CTAs (small instances packed
    // many to a CTA, and Poly's six buffers); Q = 8 halves the shared-memory
    // loads per word product, which wins elsewhere.
    const bool q4 = poly ? (n <= 192 || (n > 384 && n <= 1536)) : (n <= 48 || (n > 384 && n <= 768));
    g.q = q4 ? 4 : 8;
    g.np = roundup(n, 2 * g.q);
    const uint32_t units = g.np / (2 * g.q);
    if (units <= 32) {
        g.group = 1;
        while (g.group < units) g.group <<= 1;
    } else {
        g.group = roundup(units, 32);
    }
    g.ipb = g.group < 256 ? 256 / g.group : 1;
    g.block = g.group * g.ipb;
    g.a_words = roundup(phys_size(g.np), 4);
    g.b_words = roundup(phys_size(g.np + 2 * g.q), 4);
    g.l_words = roundup(phys_size(g.np), 4);
    const uint32_t hc_words = 2 * (g.np / g.q);
    g.slot_words = roundup(g.a_words + g.b_words + (poly ? 3 : 1) * g.l_words + hc_words, 4);
    g.smem = 4 * (g.slot_words * g.ipb + 32);
    return g;
}

bn_status launch_low(bool poly, const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t n,
                     uint64_t batch, cudaStream_t st) {
    const LowGeometry g = low_geometry(n, poly);
    if (g.group > 1024 || g.smem > 227u * 1024u) return BN_EUNSUPPORTED;
    LowArgs p{};
    p.a = a; p.b = b; p.c = c;
    p.n = n; p.np = g.np; p.group = g.group; p.ipb = g.ipb; p.slot_words = g.slot_words;
    p.a_words = g.a_words; p.b_words = g.b_words; p.l_words = g.l_words;
    // Poly stages a into the B region too, so both rows take the same path.
    p.vec_a = p.vec_b = (n % 4 == 0) && ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0);
    p.batch = batch;
    const uint64_t grid = (batch + g.ipb - 1) / g.ipb;
    if (grid > 0x7fffffffull) return BN_EUNSUPPORTED;
    const void *kern = poly ? (g.q == 4 ? (const void *)k_poly<4> : (const void *)k_poly<8>)
                            : (g.q == 4 ? (const void *)k_mul_low<4> : (const void *)k_mul_low<8>);
    if (allow_max_smem(kern) != cudaSuccess) return BN_ECUDA;
    if (poly) {
        if (g.q == 4) k_poly<4><<<(unsigned)grid, g.block, g.smem, st>>>(p);
        else k_poly<8><<<(unsigned)grid, g.block, g.smem, st>>>(p);
    } else {
        if (g.q == 4) k_mul_low<4><<<(unsigned)grid, g.block, g.smem, st>>>(p);
        else k_mul_low<8><<<(unsigned)grid, g.block, g.smem, st>>>(p);
    }
    if (cudaError_t e = cudaGetLastError()) {
        record_error(cudaGetErrorString(e));
        return BN_ECUDA;
    }
    return BN_OK;
}

template <int VEC, int R>
void launch_add6_t(const Add6Args &p, uint32_t block, uint64_t grid, cudaStream_t st) {
    k_add6_team<VEC, R><<<(unsigned)grid, block, 0, st>>>(p);
}

bn_status launch_add6(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t n, uint64_t batch,
                      cudaStream_t st) {
    const bool vec = (n % 4 == 0) && ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0);
    Add6Args p{};
    p.a = a; p.b = b; p.c = c; p.n = n; p.batch = batch;
    const uint32_t V = vec ? 4 : 1;
    p.chunks = (n + V - 1) / V;
    if (p.chunks <= 32) {
        p.group = 1;
        p.log2_group = 0;
        while (p.group < p.chunks) {
            p.group <<= 1;
            ++p.log2_group;
        }
        const uint32_t block = 256;
        const uint64_t grid = ((batch << p.log2_group) + block - 1) / block;
        if (grid > 0x7fffffffull) return BN_EUNSUPPORTED;
        if (vec) k_add6_sub<4><<<(unsigned)grid, block, 0, st>>>(p);
        else k_add6_sub<1><<<(unsigned)grid, block, 0, st>>>(p);
    } else {
        // Up to 16 limbs a thread in each of the two register sets.
        const uint32_t r_max = vec ? 4 : 16;
        uint32_t R = 1, W = (p.chunks + 31) / 32;
        while (W > 8 && R < r_max) {
            R *= 2;
            W = (p.chunks + 32 * R - 1) / (32 * R);
        }
        if (W > 16) return BN_EUNSUPPORTED;
        p.warps_per_team = W;
        p.teams_per_cta = 256 > 32 * W ? 256 / (32 * W) : 1;
        const uint32_t block = 32 * W * p.teams_per_cta;
        const uint64_t grid = (batch + p.teams_per_cta - 1) / p.teams_per_cta;
        if (grid > 0x7fffffffull) return BN_EUNSUPPORTED;
        if (vec) {
            if (R == 1) launch_add6_t<4, 1>(p, block, grid, st);
            else if (R == 2) launch_add6_t<4, 2>(p, block, grid, st);
            else launch_add6_t<4, 4>(p, block, grid, st);
        } else {
            if (R == 1) launch_add6_t<1, 1>(p, block, grid, st);
            else if (R == 2) launch_add6_t<1, 2>(p, block, grid, st);
            else if (R == 4) launch_add6_t<1, 4>(p, block, grid, st);
            else if (R == 8) launch_add6_t<1, 8>(p, block, grid, st);
            else launch_add6_t<1, 16>(p, block, grid, st);
        }
    }
    if (cudaError_t e = cudaGetLastError()) {
        record_error(cudaGetErrorString(e));
        return BN_ECUDA;
    }
    return BN_OK;
}

bn_status check_same_length(const uint32_t *a, const uint32_t *b, const uint32_t *c, uint32_t n,
                            uint64_t batch, uint32_t max_n) {
    if (n == 0) {
        record_error("zero limb count");
        return BN_EINVAL;
    }
    if (n > max_n) {
        record_error("size not supported by this program");
        return BN_EUNSUPPORTED;
    }
    if (batch && (!a || !b || !c)) {
        record_error("null operand or result pointer");
        return BN_EINVAL;
    }
    const uintptr_t bytes = batch * n * 4ull, pc = (uintptr_t)c, pa = (uintptr_t)a, pb = (uintptr_t)b;
    if (batch && ((pc < pa + bytes && pa < pc + bytes) || (pc < pb + bytes && pb < pc + bytes))) {
        record_error("result overlaps an operand");
        return BN_EINVAL;
    }
    return BN_OK;
}

}  // namespace
}  // namespace bn

extern "C" {

bn_status bn_mul_low(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t n, uint64_t batch,
                     void *stream) {
    bn_status s = bn::check_same_length(a, b, c, n, batch, BN_MUL_MAX_LIMBS);
    if (s != BN_OK || batch == 0) return s;
    return bn::launch_low(false, a, b, c, n, batch, (cudaStream_t)stream);
}

bn_status bn_poly(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t n, uint64_t batch,
                  void *stream) {
    bn_status s = bn::check_same_length(a, b, c, n, batch, BN_MUL_MAX_LIMBS);
    if (s != BN_OK || batch == 0) return s;
    return bn::launch_low(true, a, b, c, n, batch, (cudaStream_t)stream);
}

bn_status bn_add6(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t n, uint64_t batch,
                  void *stream) {
    bn_status s = bn::check_same_length(a, b, c, n, batch, BN_MUL_MAX_LIMBS);
    if (s != BN_OK || batch == 0) return s;
    return bn::launch_add6(a, b, c, n, batch, (cudaStream_t)stream);
}

}  // extern "C"
