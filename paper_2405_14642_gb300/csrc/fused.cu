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
        const Unit u{t * Q, 0, t + 1, (R - 1 - t) * Q, 0, R - t};
        conv_unit<Q>(As, Bs, u, [&](uint32_t k, const uint32_t (&acc)[Q + 2]) {
            st_words<Q>(Ls, k, acc);
            *reinterpret_cast<uint2 *>(Hc + 2 * (k / Q)) = make_uint2(acc[Q], acc[Q + 1]);
        });
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
//
// Each thread owns one contiguous run of L = 16 limbs of an instance, so an
// addition costs L add-with-carry steps, an all-ones test and ONE carry scan
// per thread (the scan, not the limb arithmetic, dominated with 4-limb chunks).

// s = a + b over 8 limbs, returns the carry out; s may alias a.
__device__ __forceinline__ uint32_t add8(const uint32_t *a, const uint32_t *b, uint32_t *s, uint32_t cin) {
    uint32_t c = cin;
    asm("add.cc.u32 %8, %8, 0xffffffff;\n\t"   // CF = (cin != 0)
        "addc.cc.u32 %0, %9, %17;\n\t"
        "addc.cc.u32 %1, %10, %18;\n\t"
        "addc.cc.u32 %2, %11, %19;\n\t"
        "addc.cc.u32 %3, %12, %20;\n\t"
        "addc.cc.u32 %4, %13, %21;\n\t"
        "addc.cc.u32 %5, %14, %22;\n\t"
        "addc.cc.u32 %6, %15, %23;\n\t"
        "addc.cc.u32 %7, %16, %24;\n\t"
        "addc.u32 %8, 0, 0;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]),
          "=r"(s[7]), "+r"(c)
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
          "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
    return c;
}

// s += cin (cin in {0, 1}) over 8 limbs, returns the carry out.
__device__ __forceinline__ uint32_t inc8(uint32_t *s, uint32_t cin) {
    uint32_t c;
    asm("add.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.cc.u32 %4, %4, 0;\n\t"
        "addc.cc.u32 %5, %5, 0;\n\t"
        "addc.cc.u32 %6, %6, 0;\n\t"
        "addc.cc.u32 %7, %7, 0;\n\t"
        "addc.u32 %8, 0, 0;"
        : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4]), "+r"(s[5]), "+r"(s[6]),
          "+r"(s[7]), "=r"(c)
        : "r"(cin));
    return c;
}

template <int L>
__device__ __forceinline__ uint32_t add_run(const uint32_t (&a)[L], const uint32_t (&b)[L], uint32_t (&s)[L]) {
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < L; k += 8) c = add8(a + k, b + k, s + k, c);
    return c;
}

template <int L>
__device__ __forceinline__ void inc_run(uint32_t (&s)[L], uint32_t cin) {
#pragma unroll
    for (int k = 0; k < L; k += 8) cin = inc8(s + k, cin);
}

template <int L>
__device__ __forceinline__ uint32_t all_ones_run(const uint32_t (&s)[L]) {
    uint32_t x = s[0];
#pragma unroll
    for (int k = 1; k < L; ++k) x &= s[k];
    return x == 0xffffffffu;
}

// Run j (limbs L*j .. L*j+L-1) of a row of n limbs, zero beyond n.  With VEC
// the row start is 16-byte aligned and n a multiple of 4, so each group of 4
// limbs is wholly inside or outside the row.
template <int L, bool VEC>
__device__ __forceinline__ void load_run(const uint32_t *row, uint32_t j, uint32_t n, bool live,
                                         uint32_t (&v)[L]) {
    const uint32_t x0 = L * j;
    if constexpr (VEC) {
#pragma unroll
        for (int k = 0; k < L; k += 4) {
            const bool in = live && x0 + k < n;
            const uint4 t = in ? ld_stream_v4(row + x0 + k) : make_uint4(0, 0, 0, 0);
            v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < L; ++k) v[k] = (live && x0 + k < n) ? ld_stream(row + x0 + k) : 0u;
    }
}

template <int L, bool VEC>
__device__ __forceinline__ void store_run(uint32_t *row, uint32_t j, uint32_t n, const uint32_t (&v)[L]) {
    const uint32_t x0 = L * j;
    if constexpr (VEC) {
#pragma unroll
        for (int k = 0; k < L; k += 4)
            if (x0 + k < n) st_stream_v4(row + x0 + k, make_uint4(v[k], v[k + 1], v[k + 2], v[k + 3]));
    } else {
#pragma unroll
        for (int k = 0; k < L; ++k)
            if (x0 + k < n) st_stream(row + x0 + k, v[k]);
    }
}

struct Add6Args {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t n, group, ipb;
    uint64_t batch;
};

// `group` threads per instance (a power of two <= 32, or whole warps), `ipb`
// instances per CTA.  Step k overwrites x_{k-1} (register set k % 2) with
// x_{k+1} = x_k + x_{k-1}; after six steps set 1 holds x_7.  For whole-warp
// groups the warp summaries alternate between two buffers, so one barrier
// per addition suffices: a warp writes buffer k % 2 only after passing
// addition k-1's barrier, which every reader of addition k-2 reached after
// its read.
template <int L, bool VEC>
__global__ void __launch_bounds__(512) k_add6(Add6Args p) {
    __shared__ uint32_t flags[2][16];
    const uint32_t slot = threadIdx.x / p.group, t = threadIdx.x - slot * p.group;
    const uint64_t inst = (uint64_t)blockIdx.x * p.ipb + slot;
    const bool live = inst < p.batch;
    uint32_t x[2][L];
    load_run<L, VEC>(p.a + inst * p.n, t, p.n, live, x[0]);
    load_run<L, VEC>(p.b + inst * p.n, t, p.n, live, x[1]);
#pragma unroll
    for (int step = 0; step < 6; ++step) {
        uint32_t(&z)[L] = x[step % 2];
        const uint32_t g = add_run<L>(z, x[(step + 1) % 2], z);
        const uint32_t cin = group_carry_in(g, all_ones_run<L>(z), p.group, flags[step % 2]);
        inc_run<L>(z, cin);
    }
    if (live) store_run<L, VEC>(p.c + inst * p.n, t, p.n, x[1]);
}

// ---- host side ---------------------------------------------------------------

struct LowGeometry {
    uint32_t q, np, group, ipb, block, slot_words, a_words, b_words, l_words, smem;
};

LowGeometry low_geometry(uint32_t n, bool poly) {
    LowGeometry g{};
    // Window size from GB300 timings over the 1K..256K-bit sweep: Q = 4 puts
    // twice the threads on an instance for the same shared memory, which wins
    // only for the smallest instances (packed many to a CTA, where shared
    // memory bounds the resident CTAs); Q = 8 halves the shared-memory loads
    // per word product and wins from 2K bits (1-Mul) or 4K bits (Poly) up.
    const bool q4 = poly ? n <= 96 : n <= 48;
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

template <int L, bool VEC>
void launch_add6_t(const Add6Args &p, uint32_t block, uint64_t grid, cudaStream_t st) {
    k_add6<L, VEC><<<(unsigned)grid, block, 0, st>>>(p);
}

bn_status launch_add6(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t n, uint64_t batch,
                      cudaStream_t st) {
    const bool vec = (n % 4 == 0) && ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0);
    Add6Args p{};
    p.a = a; p.b = b; p.c = c; p.n = n; p.batch = batch;
    // 16 limbs a thread: timed against 8 (the scan's cost is per thread, so
    // 16 wins up to 16K bits and ties above) and 32 (register-bound, slower
    // from 32K bits on).
    constexpr uint32_t L = 16;
    const uint32_t runs = (n + L - 1) / L;
    if (runs <= 32) {
        p.group = 1;
        while (p.group < runs) p.group <<= 1;
    } else {
        p.group = roundup(runs, 32);
    }
    if (p.group > 512) return BN_EUNSUPPORTED;
    p.ipb = p.group < 256 ? 256 / p.group : 1;
    const uint32_t block = p.group * p.ipb;
    const uint64_t grid = (batch + p.ipb - 1) / p.ipb;
    if (grid > 0x7fffffffull) return BN_EUNSUPPORTED;
    if (vec) launch_add6_t<L, true>(p, block, grid, st);
    else launch_add6_t<L, false>(p, block, grid, st);
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
