// Device code of the three-prime transform product (BN_OP_MUL_NTT3; see
// mul_ntt32.cu for the method): the 32-bit fields, the per-prime product, the
// Garner recombination and the kernels, templated on log2 of the transform
// length so that the passes run with compile-time strides (ntt_device.cuh).
// Included by the translation units that instantiate the kernels.
#pragma once
#include "bn_internal.h"
#include "ntt_device.cuh"

namespace bn {
namespace ntt3 {

using namespace ntt;

constexpr uint32_t kMaxLength3 = 16384;  // both u32 spectra in shared memory

// Z_P for a prime P < 2^30 in Montgomery form with R = 2^32; NINV = -P^-1
// mod 2^32.  Elements are kept lazily in [0, 2P); canon() maps to [0, P).
//   mul(a, b): t = a b < 4P^2 (a, b < 2P); the quotient
//   m = t_lo NINV makes t + m P divisible by 2^32, and (t + m P) / 2^32 =
//   t_hi + hi(m P) + (t_lo != 0) < 4P^2 / 2^32 + P < 2P.
template <uint32_t P, uint32_t NINV>
struct MontField32 {
    using Elem = uint32_t;
    static constexpr uint32_t P_VALUE = P;
    static constexpr uint32_t TWO_P = 2 * P;
    static constexpr uint32_t RECIP = (uint32_t)((1ull << 32) / P);  // floor(2^32 / P)
    static_assert(P < (1u << 30), "4P < 2^32");
    static_assert((uint32_t)(P * NINV) == 0xffffffffu, "NINV = -P^-1 mod 2^32");
    // Reductions as unsigned minima: for r < 4P, r - 2P wraps above r exactly
    // when r < 2P, so min(r, r - 2P) is r mod-reduced into [0, 2P) (one
    // min and one subtract instead of a compare, a select and a subtract).
    __device__ static __forceinline__ uint32_t add(uint32_t a, uint32_t b) {
        const uint32_t r = a + b;
        return min(r, r - TWO_P);
    }
    __device__ static __forceinline__ uint32_t sub(uint32_t a, uint32_t b) {
        const uint32_t r = a + TWO_P - b;
        return min(r, r - TWO_P);
    }
    __device__ static __forceinline__ uint32_t canon(uint32_t a) { return min(a, a - P); }
    __device__ static __forceinline__ uint32_t mul(uint32_t a, uint32_t b) {
        const uint32_t lo = a * b, hi = __umulhi(a, b);
        const uint32_t m = lo * NINV;
        return hi + __umulhi(m, P) + (lo != 0u);
    }
    // Any 32-bit digit d into [0, 2P): Shoup's product with the pair (1, RECIP),
    // d - hi(d RECIP) P (two multiplies).
    __device__ static __forceinline__ uint32_t from_digit(uint32_t d) { return d - __umulhi(d, RECIP) * P; }
    // Twiddles by Shoup's method: an entry is (w, w' = floor(w 2^32 / P)) with
    // w < P, and for any a < 2^32, q = hi(a w') gives a w - q P in [0, 2P),
    // exact in 32-bit arithmetic.  One high and two low multiplies, against
    // Montgomery's two high, two low and a correction.
    using Tw = uint2;
    __device__ static __forceinline__ uint32_t twiddle(uint32_t a, uint2 w) {
        const uint32_t q = __umulhi(a, w.y);
        return a * w.x - q * P;
    }
    __device__ static __forceinline__ uint32_t twiddle_lazy(uint32_t a, uint2 w) { return twiddle(a, w); }
    // Butterflies on [0, 2P): the difference u - v + 2P (< 4P) goes to the
    // twiddle product unreduced.
    __device__ static __forceinline__ void dif(uint32_t &u, uint32_t &v, uint2 w) {
        const uint32_t x = u, y = v;
        u = add(x, y);
        v = twiddle(x + TWO_P - y, w);
    }
    __device__ static __forceinline__ void dif1(uint32_t &u, uint32_t &v) {
        const uint32_t x = u, y = v;
        u = add(x, y);
        v = sub(x, y);
    }
    __device__ static __forceinline__ void dit(uint32_t &u, uint32_t &v, uint2 w) {
        const uint32_t x = u, t = twiddle_lazy(v, w);
        u = add(x, t);
        v = sub(x, t);
    }
    __device__ static __forceinline__ void dit1(uint32_t &u, uint32_t &v) { dif1(u, v); }
};

using F0 = MontField32<469762049u, 0x1bffffffu>;  // 7 * 2^26 + 1
using F1 = MontField32<754974721u, 0x2cffffffu>;  // 45 * 2^24 + 1
using F2 = MontField32<998244353u, 0x3b7fffffu>;  // 119 * 2^23 + 1
static_assert(F0::P_VALUE < F1::P_VALUE && F1::P_VALUE < F2::P_VALUE, "Garner order");

struct Tab3 {
    const uint2 *twf;     // [N]: twf[h + j] = Shoup pair of w_{2h}^j
    const uint2 *twi;     // [N]: Shoup pair of w_{2h}^-j
    uint2 scale;          // Shoup pair of N^-1 R mod p: also undoes the 1/R of the pointwise product
};

struct Ntt3Args {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t na, nb, nout, N, logN;
    uint64_t batch;
    uint32_t *scratch;        // per CTA: residues mod p0 [N], mod p1 [N]
    uint64_t scratch_stride;  // u32 words per CTA
    Tab3 t[3];
    uint32_t g01, g02, g12;   // form(p0^-1 mod p1), form(p0^-1 mod p2), form(p1^-1 mod p2)
};

// Threads per CTA for a transform of 2^LOGN points: one per radix-8 group,
// between one warp and 1024.
template <uint32_t LOGN>
__host__ __device__ constexpr uint32_t threads_for() {
    return (1u << LOGN) / 8 < 32 ? 32u : ((1u << LOGN) / 8 > 1024 ? 1024u : (1u << LOGN) / 8);
}

// Coefficients 0 .. nout-1 of a*b mod F's prime (canonical) to dest, or, with
// dest == nullptr, to B (padded layout).  Ends with a barrier.
template <class F, uint32_t LOGN>
__device__ void prime_product3(const Ntt3Args &p, const Tab3 &tb, const uint32_t *arow,
                               const uint32_t *brow, uint32_t *A, uint32_t *B, uint32_t *dest) {
    constexpr uint32_t N = 1u << LOGN, NT = threads_for<LOGN>();
    for (uint32_t j = threadIdx.x; j < N; j += NT) {                  // n1: digits
        A[phys4(j)] = j < p.na ? F::from_digit(__ldg(arow + j)) : 0u;
        B[phys4(j)] = j < p.nb ? F::from_digit(__ldg(brow + j)) : 0u;
    }
    __syncthreads();
    forward2_c<F, LOGN, NT>(tb.twf, A, B);                              // n2: forward transforms
    for (uint32_t j = threadIdx.x; j < N; j += NT)                    // n3: pointwise
        B[phys4(j)] = F::mul(A[phys4(j)], B[phys4(j)]);
    __syncthreads();
    inverse_c<F, LOGN, NT>(tb.twi, B);                                  // n4: inverse (unscaled)
    for (uint32_t j = threadIdx.x; j < p.nout; j += NT) {
        const uint32_t v = F::canon(F::twiddle(B[phys4(j)], tb.scale));
        if (dest) dest[j] = v;
        else B[phys4(j)] = v;
    }
    __syncthreads();
}

// n5: the coefficient with residues r0, r1, r2 (canonical): c = v0 + v1 p0 +
// v2 p0 p1 with v0 = r0, v1 = (r1 - v0) / p0 mod p1, v2 = ((r2 - v0) / p0 -
// v1) / p1 mod p2 (Garner), exact since c < p0 p1 p2.
__device__ __forceinline__ u128 garner3(const Ntt3Args &p, uint32_t r0, uint32_t r1, uint32_t r2) {
    uint32_t d = r1 >= r0 ? r1 - r0 : r1 + F1::P_VALUE - r0;  // r0 < p0 < p1
    const uint32_t v1 = F1::canon(F1::mul(d, p.g01));
    d = r2 >= r0 ? r2 - r0 : r2 + F2::P_VALUE - r0;            // r0 < p0 < p2
    uint32_t e = F2::canon(F2::mul(d, p.g02));
    e = e >= v1 ? e - v1 : e + F2::P_VALUE - v1;                // v1 < p1 < p2
    const uint32_t v2 = F2::canon(F2::mul(e, p.g12));
    constexpr uint64_t P01 = (uint64_t)F0::P_VALUE * F1::P_VALUE;
    return (u128)((uint64_t)r0 + (uint64_t)v1 * F0::P_VALUE) + (u128)v2 * P01;
}

// Shared-memory layout of a CTA: both spectra, then the normalisation's spill
// words and warp flags.
struct Smem3 {
    uint32_t *A, *B;
    uint64_t *spill;
    uint32_t *flags;
};

template <uint32_t LOGN>
__device__ __forceinline__ Smem3 smem3(uint32_t *sm32) {
    constexpr uint32_t Np = (phys4_words(1u << LOGN) + 3) & ~3u;  // B stays 16-byte aligned
    Smem3 s;
    s.A = sm32;
    s.B = sm32 + Np;
    s.spill = reinterpret_cast<uint64_t *>(s.B + Np);
    s.flags = reinterpret_cast<uint32_t *>(s.spill + threads_for<LOGN>());
    return s;
}

// One pair: the three primes, then n6, recombination and carrying into limbs
// (A's words serve as the staging row).
template <uint32_t LOGN>
__device__ __forceinline__ void pair_product3(const Ntt3Args &p, const uint32_t *arow, const uint32_t *brow,
                                              uint32_t *crow, const Smem3 &s, uint32_t *R0, uint32_t *R1) {
    prime_product3<F0, LOGN>(p, p.t[0], arow, brow, s.A, s.B, R0);
    prime_product3<F1, LOGN>(p, p.t[1], arow, brow, s.A, s.B, R1);
    prime_product3<F2, LOGN>(p, p.t[2], arow, brow, s.A, s.B, nullptr);
    const uint32_t *B = s.B;
    normalize_limbs(p.nout, crow, s.A, s.spill, s.flags,
                    [&](uint32_t k) { return garner3(p, R0[k], R1[k], B[phys4(k)]); });
}

// Plain batch: CTA i walks pairs i, i + gridDim.x, ... (persistent grid).
template <uint32_t LOGN>
__global__ void __launch_bounds__(1024) k_mul_ntt3(Ntt3Args p) {
    extern __shared__ __align__(16) uint32_t sm32[];
    const Smem3 s = smem3<LOGN>(sm32);
    uint32_t *R0 = p.scratch + blockIdx.x * p.scratch_stride;
    uint32_t *R1 = R0 + p.N;
    for (uint64_t inst = blockIdx.x; inst < p.batch; inst += gridDim.x)
        pair_product3<LOGN>(p, p.a + inst * p.na, p.b + inst * p.nb, p.c + inst * p.nout, s, R0, R1);
}

// Mixed-size batch of products sharing the transform length: the CTA takes
// the next item from the work queue (largest first) and uses its sizes and rows.
template <uint32_t LOGN>
__global__ void __launch_bounds__(1024)
    k_mul_ntt3_batch(Ntt3Args p, const BatchItem *items, uint32_t count, uint32_t *queue,
                     const BatchBinding *bind) {
    extern __shared__ __align__(16) uint32_t sm32[];
    __shared__ uint32_t next;
    const Smem3 s = smem3<LOGN>(sm32);
    uint32_t *R0 = p.scratch + blockIdx.x * p.scratch_stride;
    uint32_t *R1 = R0 + p.N;
    for (;;) {
        __syncthreads();  // the previous item is stored before `next` moves on
        if (threadIdx.x == 0) next = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t i = next;
        if (i >= count) break;
        const BatchItem it = items[i];
        p.na = it.na;
        p.nb = it.nb;
        p.nout = it.na + it.nb;
        pair_product3<LOGN>(p, bind->a + it.off_a, bind->b + it.off_b, bind->c + it.off_c, s, R0, R1);
    }
}

// The kernels of one length, for the host code: (plain, batch).
struct Kernels3 {
    const void *plain, *batch;
};

template <uint32_t LOGN>
Kernels3 kernels3() {
    return {(const void *)k_mul_ntt3<LOGN>, (const void *)k_mul_ntt3_batch<LOGN>};
}

}  // namespace ntt3

// Kernel table of the three-prime transform, split over translation units so
// that the instantiations compile in parallel (mul_ntt32_k*.cu): the kernels
// for log2 N in [lo, hi] of each unit, or {nullptr, nullptr} outside it.
ntt3::Kernels3 ntt3_kernels_small(uint32_t log_n);   // log2 N = 1 .. 10
ntt3::Kernels3 ntt3_kernels_mid(uint32_t log_n);     // 11 .. 12
ntt3::Kernels3 ntt3_kernels_large(uint32_t log_n);   // 13 .. 14

}  // namespace bn
