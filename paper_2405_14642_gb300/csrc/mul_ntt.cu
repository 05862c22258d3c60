// Batched multiplication through a number-theoretic transform (Section 4).
//
// Fields (Section 4.1, with the digit sizes read so that every convolution
// coefficient stays below the modulus):
//   * BN_OP_MUL_NTT64: PrimeField64, p1 = 29*2^57 + 1 with root g = 21 of
//     order 2^57, 16-bit digits (coefficients < 2^46 at 256K bits);
//   * BN_OP_MUL_NTT_CRT: 32-bit digits over p1 and p2 = 27*2^56 + 1 (root
//     5^27 of order 2^56), recombined by Garner's form of the CRT
//     (coefficients < 2^77 < p1 p2).
// Transform length N = next power of two >= digits(a) + digits(b), so the
// cyclic convolution does not wrap (inputs are zero-padded).
//
// Arithmetic.  Section 4.1's field multiplies with a full-width modulo; here
// the butterflies multiply by twiddles with Shoup's method (each table entry
// is a pair (w, floor(w 2^64 / p)), so a product costs one high and two low
// 64-bit multiplies and no division) and keep Harvey's lazy ranges: the
// forward (decimation-in-frequency) passes hold values in [0, 2p), the
// inverse (decimation-in-time) passes in [0, 4p), one conditional
// subtraction per butterfly (both primes are below 2^62, so 4p < 2^64).
// The pointwise product of two spectra is a Montgomery product (R = 2^64),
// cheap because each prime's low 32-bit word is 1; the final scale by 1/N
// also cancels its 1/R.
//
// Work mapping.  A transform of up to 8192 points is one CTA's: both spectra
// in shared memory, forward transforms natural order in / bit-reversed out,
// the inverse bit-reversed in / natural out (no permutation pass; Section
// 4.2's fft reorders first), stages grouped into radix-8 passes (a thread
// loads 8 elements, runs 3 stages in registers, stores them back: one
// barrier per 3 stages).  A persistent grid walks the batch.
//
// Longer transforms (N = S*L, S in {2, 4}, L = 8192) are split into S
// sub-problems and run on a cluster of two CTAs that share their shared
// memory; each CTA owns S/2 sub-problems.  For sub-problem s the first
// radix-S decimation-in-frequency stage is folded into the digit load (y_s[j]
// = w_N^{js} sum_r x[j + rL] w_S^{rs}, from the operand rows in global
// memory), then its forward transforms, pointwise product and inverse run as
// above, and the last radix-S inverse stage's factor N^-1 w_N^{-js} is
// applied to its result z_s.  A CTA with two sub-problems keeps the first
// one's result in a third shared buffer.  The remaining radix-S butterfly,
// sum over s of w_S^{-qs} z_s[j] for output quarter q, is evaluated by the
// CTA that owns position j (half of the positions each), reading z_s[j] from
// both CTAs.  Nothing goes through global scratch.  The two-prime form keeps
// the first prime's coefficients in the third buffer while the second prime
// runs (in global scratch, L2-resident, only for short one-CTA transforms,
// where a third buffer would cost occupancy).
//
// Normalisation (Section 4.2's splitFftReg/baddRegMul2Fft, here with whole
// 16/32-bit digits).  Each thread folds the coefficients of its window of
// limbs into limbs plus a carried spill, the spill is added into the next
// window (across CTAs of a cluster through shared memory), and the
// remaining one-bit carries are resolved with the Section 2 carry scan
// across threads and then across the cluster's CTAs.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "bn_internal.h"
#include "ntt_device.cuh"

namespace bn {

namespace {

using namespace ntt;

constexpr uint32_t kMaxSubLength = 8192;  // both spectra in shared memory
constexpr uint32_t kMaxSplit = 4;         // N <= 32768

// CTAs per product: a split transform runs on a cluster of two.
__host__ __device__ constexpr uint32_t cluster_of(uint32_t S) { return S > 1 ? 2u : 1u; }

// ---- clusters ---------------------------------------------------------------

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster; orders shared-memory writes
// before the barrier before reads after it, across the cluster.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of `p` (this CTA's shared memory) in the shared memory of the
// cluster's CTA `rank`, for ld.shared::cluster.
__device__ __forceinline__ uint32_t dsmem_addr(const void *p, uint32_t rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ uint64_t ld_dsmem_u64(uint32_t addr) {
    uint64_t v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_dsmem_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// ---- device fields ---------------------------------------------------------

// Shoup pair of a constant w < P: (w, floor(w 2^64 / P)).
typedef ulonglong2 Tw64;

// Z_P for a prime P = k 2^m + 1 with m >= 32 (so P's low 32-bit word is 1)
// and P < 2^62 (so 4P + 2^48 < 2^64).
//   * shoup(x, (w, w')): for any 64-bit x, q = hi64(x w') and x w - q P lies
//     in [0, 2P) and is x w mod P up to one P (Shoup; exact in 64-bit
//     arithmetic since the result is below 2^64).
//   * mont(a, b) for a, b < 2^63: a b / 2^64 mod P in [0, 2P).  The 128-bit
//     product comes from four 32x32->64 multiply-adds with no carry handling
//     (a, b < 2^63 keep the cross sum below 2^64).  Reduction: -P^-1 = P - 2
//     (mod 2^64), so the quotient m = t_lo (P - 2) has words (-x0, x0*P_hi -
//     x1 - borrow); m*P needs two more multiply-adds since P's low word is 1;
//     the result is < 2P because 4P < 2^64.
//   * Forward (decimation-in-frequency) butterflies keep Harvey's range
//     [0, 2P): dif gives u + v reduced into [0, 2P) and (u - v + 2P) w by
//     Shoup (< 2P).  The constant added before a subtraction must be a
//     multiple of P that is at least the value subtracted, and only 4.4 P
//     fit in 64 bits for p1: so these values are reduced exactly.
//   * Inverse (decimation-in-time) butterflies: dit takes t = v w by Shoup
//     (< 2P, exact range) and x = red(u), and gives x + t and x - t + 2P.
//     red(r) subtracts 2P when the high word of r exceeds the high word H of
//     2P (then r >= (H + 1) 2^32 > 2P, no wrap), else leaves r (< (H + 1)
//     2^32 <= 2P + 2^32): one compare of one word.  From the pointwise
//     products (< 2P) the inverse values stay below 4P + 2^32.  The twiddle-1
//     butterfly reduces the value standing in for the product exactly
//     (red2, into [0, 2P)).
template <uint64_t P>
struct Field64 {
    using Elem = uint64_t;
    using Tw = Tw64;
    static constexpr uint64_t P_VALUE = P;
    static constexpr uint32_t PH = (uint32_t)(P >> 32);
    static constexpr uint64_t TWO_P = 2 * P;
    static constexpr uint32_t H = (uint32_t)(TWO_P >> 32);
    static_assert((P & 0xffffffffull) == 1 && P < (1ull << 62), "P = k 2^m + 1, m >= 32, P < 2^62");
    static_assert(((uint64_t)(H + 1) << 32) >= TWO_P, "red never wraps");
    static_assert(P < (~0ull - (1ull << 33)) / 4, "4P + 2^33 fits in 64 bits");
    // r < 4P into [0, 2P): r - 2P wraps above r exactly when r < 2P.
    __device__ static __forceinline__ uint64_t rexact(uint64_t r) {
        const uint64_t t = r - TWO_P;
        return t < r ? t : r;
    }
    __device__ static __forceinline__ uint64_t red(uint64_t r) {
        return (uint32_t)(r >> 32) > H ? r - TWO_P : r;
    }
    // r < 4P + 2^33 into [0, 2P).
    __device__ static __forceinline__ uint64_t red2(uint64_t r) { return rexact(red(r)); }
    // a, b < 2P.
    __device__ static __forceinline__ uint64_t add(uint64_t a, uint64_t b) { return rexact(a + b); }
    __device__ static __forceinline__ uint64_t sub(uint64_t a, uint64_t b) { return rexact(a + TWO_P - b); }
    // a mod P for a < 2P, and for a < 4P.
    __device__ static __forceinline__ uint64_t canon(uint64_t a) { return a >= P ? a - P : a; }
    __device__ static __forceinline__ uint64_t exact(uint64_t a) { return canon(rexact(a)); }
    __device__ static __forceinline__ uint64_t shoup(uint64_t x, Tw64 w) {
        const uint64_t q = __umul64hi(x, w.y);
        const uint64_t qp = q + ((uint64_t)((uint32_t)q * PH) << 32);  // q * P mod 2^64
        return x * w.x - qp;
    }
    __device__ static __forceinline__ uint64_t mont(uint64_t a, uint64_t b) {
        const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
        const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
        const uint64_t p00 = (uint64_t)a0 * b0;
        uint64_t t = (uint64_t)a0 * b1 + (p00 >> 32);
        t += (uint64_t)a1 * b0;
        const uint64_t hi = (uint64_t)a1 * b1 + (t >> 32);
        const uint32_t x0 = (uint32_t)p00, x1 = (uint32_t)t;
        const uint32_t m0 = 0u - x0;
        const uint32_t m1 = x0 * PH - x1 - (x0 != 0u);
        const uint64_t sm = (uint64_t)m0 * PH + m1;
        const uint64_t h = (uint64_t)m1 * PH + (sm >> 32);
        return hi + h + ((x0 | x1) != 0u);
    }
    __device__ static __forceinline__ void dif(uint64_t &u, uint64_t &v, Tw64 w) {
        const uint64_t x = u, y = v;
        u = add(x, y);
        v = shoup(x + TWO_P - y, w);
    }
    __device__ static __forceinline__ void dif1(uint64_t &u, uint64_t &v) {
        const uint64_t x = u, y = v;
        u = add(x, y);
        v = sub(x, y);
    }
    __device__ static __forceinline__ void dit(uint64_t &u, uint64_t &v, Tw64 w) {
        const uint64_t x = red(u), t = shoup(v, w);
        u = x + t;
        v = x + TWO_P - t;
    }
    __device__ static __forceinline__ void dit1(uint64_t &u, uint64_t &v) {
        const uint64_t x = red(u), t = red2(v);
        u = x + t;
        v = x + TWO_P - t;
    }
};

using FieldP1 = Field64<4179340454199820289ull>;  // 29 * 2^57 + 1 (PrimeField64)
using FieldP2 = Field64<1945555039024054273ull>;  // 27 * 2^56 + 1

struct PrimeTab {
    const Tw64 *twf;    // [L]: twf[h + j] = w_{2h}^j (h = 1 .. L/2, j < h)
    const Tw64 *twi;    // [L]: w_{2h}^-j
    const Tw64 *ffold;  // [S*L]: w_N^{js}                 (S > 1)
    const Tw64 *ifold;  // [S*L]: N^-1 R w_N^{-js}          (S > 1)
    Tw64 w4, iw4;       // w_4 and w_4^-1                   (S = 4)
    Tw64 scale;         // N^-1 R                           (S = 1)
};

struct NttArgs {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t na, nb, nout;
    uint32_t N, L, logL, S, digit_bits;
    uint32_t z_smem;          // a third shared buffer: the first prime's coefficients (two
                              // primes) or the first sub-problem's result (S = 4)
    uint64_t batch;
    uint64_t *scratch;        // two primes, z_smem == 0: one slot per CTA
    uint64_t scratch_stride;  // u64 words per CTA
    Tw64 garner;              // p1^-1 mod p2
    PrimeTab t1, t2;
};

__host__ __device__ constexpr uint32_t buf_words(uint32_t L) { return (phys_words(L) + 1) & ~1u; }

// Dynamic shared memory of one CTA: `bufs` padded length-L buffers, one
// spill word per thread, the warp flags, the cluster carry words (2 per
// segment of the CTA) and the batch queue slot.
__host__ __device__ constexpr uint32_t smem_bytes(uint32_t L, uint32_t bufs, uint32_t threads) {
    return 8u * (bufs * buf_words(L) + threads) + 4u * (32u + 2u * kMaxSplit + 2u);
}

struct Smem64 {
    uint64_t *A, *B, *Z;  // Z: the third buffer (z_smem)
    uint64_t *spill;
    uint32_t *flags, *xflag, *next;
};

__device__ __forceinline__ Smem64 smem64(const NttArgs &p, uint64_t *sm) {
    const uint32_t W = buf_words(p.L);
    Smem64 s;
    s.A = sm;
    s.B = sm + W;
    s.Z = p.z_smem ? sm + 2 * W : nullptr;
    s.spill = sm + (p.z_smem ? 3 : 2) * W;
    s.flags = reinterpret_cast<uint32_t *>(s.spill + blockDim.x);
    s.xflag = s.flags + 32;
    s.next = s.xflag + 2 * kMaxSplit;
    return s;
}

// The radix-S fold of sub-problem s (S = 1, 2, 4) over digits x[r] =
// x_{j + rL}: sum_r x_r w_S^{rs}, for which w_2 = w_4^2 = -1, so only w_4
// (times x1 - x3) takes a product.  Values in [0, 2P).
template <class F, uint32_t S>
__device__ __forceinline__ uint64_t fold(const uint64_t (&x)[S], uint32_t s, Tw64 w4) {
    if constexpr (S == 1) return x[0];
    else if constexpr (S == 2) return s == 0 ? F::add(x[0], x[1]) : F::sub(x[0], x[1]);
    else {
    if (s == 0) return F::add(F::add(x[0], x[2]), F::add(x[1], x[3]));
    if (s == 2) return F::sub(F::add(x[0], x[2]), F::add(x[1], x[3]));
    const uint64_t o = F::sub(x[0], x[2]), q = F::shoup(F::sub(x[1], x[3]), w4);
    return s == 1 ? F::add(o, q) : F::sub(o, q);
    }
}

// n1 for sub-problem s of both operands: y_s[j] = w_N^{js} sum_r x[j + rL]
// w_S^{rs} into A (from arow) and B (from brow), values in [0, 2P).  Each
// thread takes positions j, j + 1 (j even): with 16-bit digits one 32-bit
// word of each row quarter holds both.  All global loads of U iterations
// are issued before any is used.
template <class F, uint32_t S, bool D16>
__device__ void load_fold(const NttArgs &p, const PrimeTab &tb, const uint32_t *arow, const uint32_t *brow,
                          uint32_t s, uint64_t *A, uint64_t *B) {
    constexpr bool d16 = D16;
    const uint32_t wa = p.na, wb = p.nb;  // 32-bit words per row
    const uint32_t half = p.L / 2;
    // word index of digit position m; 16-bit digits: position pairs share one word
    auto word = [&](const uint32_t *row, uint32_t nw, uint32_t m) -> uint32_t {
        const uint32_t w = d16 ? m >> 1 : m;
        return w < nw ? __ldg(row + w) : 0u;
    };
    constexpr int U = D16 || S == 1 ? 2 : 1;
    for (uint32_t q0 = threadIdx.x; q0 < half; q0 += U * blockDim.x) {
        uint32_t ra[U][S][2], rb[U][S][2];
        Tw64 f[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t j = 2 * (q0 + u * blockDim.x);
#pragma unroll
            for (uint32_t r = 0; r < S; ++r) {
                const bool live = j < p.L;
                const uint32_t m = j + r * p.L;
                ra[u][r][0] = live ? word(arow, wa, m) : 0u;
                rb[u][r][0] = live ? word(brow, wb, m) : 0u;
                ra[u][r][1] = live && !d16 ? word(arow, wa, m + 1) : 0u;
                rb[u][r][1] = live && !d16 ? word(brow, wb, m + 1) : 0u;
            }
            const bool tw = S > 1 && j < p.L && s != 0;
            f[u][0] = tw ? __ldg(tb.ffold + s * p.L + j) : make_ulonglong2(0, 0);
            f[u][1] = tw ? __ldg(tb.ffold + s * p.L + j + 1) : make_ulonglong2(0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t j = 2 * (q0 + u * blockDim.x);
            if (j >= p.L) break;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                uint64_t xa[S], xb[S];
#pragma unroll
                for (uint32_t r = 0; r < S; ++r) {
                    xa[r] = d16 ? (ra[u][r][0] >> (16 * e)) & 0xFFFFu : ra[u][r][e];
                    xb[r] = d16 ? (rb[u][r][0] >> (16 * e)) & 0xFFFFu : rb[u][r][e];
                }
                uint64_t ya = fold<F, S>(xa, s, tb.w4), yb = fold<F, S>(xb, s, tb.w4);
                if (S > 1 && s != 0) {
                    ya = F::shoup(ya, f[u][e]);
                    yb = F::shoup(yb, f[u][e]);
                }
                A[phys(j + e)] = ya;
                B[phys(j + e)] = yb;
            }
        }
    }
}

// Forward transforms of a sub-problem: the compile-time passes for
// the lengths the 16K..256K-bit range uses most (L = 4096 and 8192 with their
// default thread counts; 7-8% faster), the runtime passes otherwise.
template <class F>
__device__ __forceinline__ void forward_sub(const NttArgs &p, const Tw64 *tw, uint64_t *A, uint64_t *B) {
    if (p.logL == 13 && blockDim.x == 1024) forward2_c<F, 13, 1024>(tw, A, B);
    else if (p.logL == 12 && blockDim.x == 512) forward2_c<F, 12, 512>(tw, A, B);
    else forward2<F>(p.L, p.logL, tw, A, B);
}


// Drops a per-CTA scratch region from L2 after its last read: its lines are
// dead, and writing them back to memory when they are evicted would only add
// DRAM traffic.  Whole CTA, after a barrier that follows the last read; a
// region that is not whole 128-byte lines is left alone.
__device__ __forceinline__ void discard_scratch(const uint64_t *ptr, uint32_t words) {
    const size_t g = __cvta_generic_to_global(ptr), bytes = 8ull * words;
    if ((g | bytes) & 127u) return;
    for (size_t off = 128ull * threadIdx.x; off < bytes; off += 128ull * blockDim.x)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(g + off) : "memory");
}

// The last inverse pass's epilogue: x -> x f (canonical), f the factor of
// position j (TABLE: a per-position table; else one factor), also stored to
// dest (padded layout) when dest is not null.
template <class F, bool TABLE>
struct ScaleEpi {
    const Tw64 *fold;
    Tw64 scale;
    uint64_t *dest;
    __device__ __forceinline__ uint64_t operator()(uint32_t j, uint64_t x) const {
        const uint64_t v = F::canon(F::shoup(x, TABLE ? __ldg(fold + j) : scale));
        if (dest) dest[phys(j)] = v;
        return v;
    }
};

// Sub-problem s of a*b mod the field's prime (n1..n4): z_s scaled by the last
// inverse stage's factor (N^-1 R w_N^{-js}; N^-1 R when S = 1), canonical, to
// dest (padded layout; dest may be B).  The compile-time inverse folds the
// scaling into its last pass.  Ends with a barrier.
template <class F, uint32_t S, bool D16>
__device__ void sub_product(const NttArgs &p, const PrimeTab &tb, const uint32_t *arow,
                            const uint32_t *brow, uint32_t s, uint64_t *A, uint64_t *B, uint64_t *dest) {
    load_fold<F, S, D16>(p, tb, arow, brow, s, A, B);  // n1: digits (and the folded first stage)
    __syncthreads();
    forward_sub<F>(p, tb.twf, A, B);              // n2: forward transforms
    for (uint32_t j = threadIdx.x; j < p.L; j += blockDim.x)   // n3: pointwise
        B[phys(j)] = F::mont(A[phys(j)], B[phys(j)]);
    __syncthreads();
    // n4: inverse transform and its scale
    const ScaleEpi<F, (S > 1)> epi{S > 1 ? tb.ifold + s * p.L : nullptr, tb.scale, dest == B ? nullptr : dest};
    if (p.logL == 13 && blockDim.x == 1024) {
        inverse_c<F, 13, 1024>(tb.twi, B, epi);
    } else if (p.logL == 12 && blockDim.x == 512) {
        inverse_c<F, 12, 512>(tb.twi, B, epi);
    } else {
        inverse<F>(p.L, p.logL, tb.twi, B);
#pragma unroll 4
        for (uint32_t j = threadIdx.x; j < p.L; j += blockDim.x) {
            const uint64_t v = epi(j, B[phys(j)]);
            if (dest == B) B[phys(j)] = v;
        }
        __syncthreads();
    }
}

// Addresses of a buffer in the shared memory of each CTA of the cluster.
struct Remote {
    uint32_t base[kMaxSplit];
};

__device__ __forceinline__ Remote remote(const uint64_t *buf, uint32_t S) {
    Remote v;
    for (uint32_t s = 0; s < kMaxSplit; ++s) v.base[s] = s < S ? dsmem_addr(buf, s) : 0u;
    return v;
}

// The last radix-S inverse stage at position j, from the sub-problems'
// scaled results of the cluster's CTAs: c[q] = sum_s w_S^{-qs} z_s[j] for
// every q (canonical).  One read of each z_s[j].
template <class F, uint32_t S>
__device__ __forceinline__ void combine(const PrimeTab &tb, const Remote &zv, uint32_t j, uint64_t (&c)[S]) {
    const uint32_t off = 8u * phys(j);
    uint64_t z[S];
#pragma unroll
    for (uint32_t s = 0; s < S; ++s) z[s] = ld_dsmem_u64(zv.base[s] + off);
    if constexpr (S == 2) {
        c[0] = F::exact(F::add(z[0], z[1]));
        c[1] = F::exact(F::sub(z[0], z[1]));
    } else {
        const uint64_t e0 = F::add(z[0], z[2]), e1 = F::add(z[1], z[3]);
        const uint64_t o0 = F::sub(z[0], z[2]), o1 = F::shoup(F::sub(z[1], z[3]), tb.iw4);
        c[0] = F::exact(F::add(e0, e1));
        c[2] = F::exact(F::sub(e0, e1));
        c[1] = F::exact(F::add(o0, o1));
        c[3] = F::exact(F::sub(o0, o1));
    }
}

// Garner's step: v = (r2 - r1) p1^-1 mod p2 for r1 < p1, r2 < p2 canonical;
// the coefficient is r1 + v p1 (exact, since it is below p1 p2).
__device__ __forceinline__ uint64_t garner_v(const NttArgs &p, uint64_t r1, uint64_t r2) {
    uint64_t r1m = r1;  // r1 mod p2 (p1 < 3 p2)
    if (r1m >= FieldP2::P_VALUE) r1m -= FieldP2::P_VALUE;
    if (r1m >= FieldP2::P_VALUE) r1m -= FieldP2::P_VALUE;
    const uint64_t d = r2 >= r1m ? r2 - r1m : r2 + FieldP2::P_VALUE - r1m;
    return FieldP2::canon(FieldP2::shoup(d, p.garner));
}

// n6 for a product split over a cluster of NC CTAs.  Its limbs fall into
// NQ*NC segments of `seg` limbs, in limb order sigma = q NC + r; CTA r holds
// segments q = 0 .. NQ-1 (its positions of every output quarter q), and
// thread group q (T/NQ threads) of the CTA normalises segment q: limb(q, k)
// gives the part of the product that starts in limb k.  Each thread folds
// the limbs of its window, carrying inside the window; the window's carry
// spills into the next window (the first window of a segment takes the last
// spill of segment sigma - 1, from another CTA); the one-bit carries left are
// resolved by the Section 2 carry scan over the group's threads, then over
// the segments in limb order (one warp scans all segments' (g, p) pairs,
// read from every CTA).  Each segment is staged in out_s (segment q at
// q (seg + seg/16 + 1), limb i at i + i/16) and copied to crow.  Every
// thread of the cluster.
template <uint32_t NC, uint32_t NQ, class LimbFn>
__device__ void normalize_segments(uint32_t nout, uint32_t seg, uint32_t rank, uint32_t *crow, uint32_t *out_s,
                                   uint64_t *spill, uint32_t *flags, uint32_t *xflag, LimbFn &&limb) {
    static_assert(NC * NQ <= 32 && NQ <= kMaxSplit, "one warp scans the segments");
    const uint32_t T = blockDim.x, t = threadIdx.x, G = T / NQ;
    const uint32_t q = t / G, i = t - q * G;  // group (segment) and thread within it
    const uint32_t lane = t & 31, warp = t >> 5, wpg = G >> 5, wig = warp - q * wpg;
    const uint32_t s_lo = (q * NC + rank) * seg;
    const uint32_t k_lo = s_lo < nout ? s_lo : nout;
    const uint32_t k_hi = s_lo + seg < nout ? s_lo + seg : nout;
    uint32_t *stage = out_s + q * (seg + seg / 16 + 1);
    uint32_t QN = (seg + G - 1) / G;
    if (QN < 2) QN = 2;  // a window must absorb a two-word spill
    const uint32_t k0 = k_lo + i * QN < k_hi ? k_lo + i * QN : k_hi;
    const uint32_t k1 = k0 + QN < k_hi ? k0 + QN : k_hi;
    u128 carry = 0;
    for (uint32_t k = k0; k < k1; ++k) {
        const u128 v = limb(q, k) + carry;
        stage[stage_index(k - k_lo)] = (uint32_t)v;
        carry = v >> 32;
    }
    spill[t] = (uint64_t)carry;  // < 2^64: the coefficients are below 2^96
    cluster_sync();
    uint64_t c = 0;
    if (i > 0) c = spill[t - 1];
    else if (rank > 0) c = ld_dsmem_u64(dsmem_addr(spill + q * G + G - 1, rank - 1));
    else if (q > 0) c = ld_dsmem_u64(dsmem_addr(spill + (q - 1) * G + G - 1, NC - 1));
    uint32_t all = 0xffffffffu;
    for (uint32_t k = k0; k < k1; ++k) {
        const uint64_t v = (uint64_t)stage[stage_index(k - k_lo)] + (c & 0xffffffffu);
        stage[stage_index(k - k_lo)] = (uint32_t)v;
        c = (c >> 32) + (v >> 32);
        all &= (uint32_t)v;
    }
    const bool owns = k0 < k1;
    BN_DEBUG_CHECK(!(owns && k1 == nout) || c == 0, kDbgSpill);  // nothing leaves the product
    BN_DEBUG_CHECK(owns || c == 0, kDbgSpill);
    // Carry scan: warps, then the group's warps, then the segments.
    const RowFlags f{__ballot_sync(FULL_MASK, owns && c != 0), __ballot_sync(FULL_MASK, owns && all == 0xffffffffu)};
    uint32_t wc, unused;
    row_carries(f, 0, wc);
    if (lane == 0) flags[warp] = wc | ((f.P == FULL_MASK) << 1);
    __syncthreads();
    const uint32_t sw = lane < wpg ? flags[q * wpg + lane] : 2u;  // lanes past the group pass a carry through
    const RowFlags fw{__ballot_sync(FULL_MASK, sw & 1u), __ballot_sync(FULL_MASK, (sw >> 1) & 1u)};
    if (wig == 0 && lane == 0) {
        uint32_t gg;
        row_carries(fw, 0, gg);
        xflag[q] = gg | ((fw.P == FULL_MASK) << 1);
    }
    cluster_sync();
    if (warp == 0) {  // lane sigma: segment sigma's pair, from CTA sigma mod NC
        const uint32_t x = lane < NC * NQ ? ld_dsmem_u32(dsmem_addr(xflag + lane / NC, lane % NC)) : 2u;
        const RowFlags fs{__ballot_sync(FULL_MASK, x & 1u), __ballot_sync(FULL_MASK, (x >> 1) & 1u)};
        const uint32_t into = row_carries(fs, 0, unused);  // bit sigma: the carry into segment sigma
        if (lane < NQ) xflag[NQ + lane] = (into >> (lane * NC + rank)) & 1u;
    }
    __syncthreads();
    const uint32_t wcin = (row_carries(fw, xflag[NQ + q], unused) >> wig) & 1u;
    const uint32_t cin = (row_carries(f, wcin, unused) >> lane) & 1u;
    BN_DEBUG_CHECK(!(owns && k1 == nout && cin && all == 0xffffffffu), kDbgSpill);
    if (cin)
        for (uint32_t k = k0; k < k1; ++k)
            if (++stage[stage_index(k - k_lo)] != 0) break;
    __syncthreads();
    for (uint32_t x = k_lo + i; x < k_hi; x += G) st_stream(crow + x, stage[stage_index(x - k_lo)]);
}

// One product by a CTA (S = 1) or a cluster of two CTAs (this one of rank
// `rank`).  zk: where the first prime's coefficients go (two primes).
//
// In a cluster, CTA r owns the positions j in [rL/2, (r+1)L/2) of every
// output quarter: it reads z_s[j] of all S sub-problems once (thread-
// consecutive j, so each warp reads whole runs of both CTAs' buffers),
// evaluates the last radix-S stage for all quarters into its own A; 16-bit
// digits: as limb values c[j] + c[j+1] 2^16 (quarter q at q L/4); two primes:
// the first prime's coefficients (quarter q at q L/2), then Garner's v into
// its Z.  Only then is it normalised, from local memory, with B (no longer
// read by the other CTA) as the staging row.
template <bool CRT, uint32_t S>
__device__ void pair_product(const NttArgs &p, const uint32_t *arow, const uint32_t *brow, uint32_t *crow,
                             const Smem64 &s, uint64_t *zk, uint32_t rank) {
    constexpr uint32_t C = cluster_of(S), SP = S / C;  // CTAs, sub-problems per CTA
    if constexpr (CRT) {
        static_assert(SP == 1, "two primes split at most in two");
        sub_product<FieldP1, S, false>(p, p.t1, arow, brow, rank, s.A, s.B, zk);
        sub_product<FieldP2, S, false>(p, p.t2, arow, brow, rank, s.A, s.B, s.B);
    } else if constexpr (SP == 2) {
        sub_product<FieldP1, S, true>(p, p.t1, arow, brow, 2 * rank, s.A, s.B, s.Z);
        sub_product<FieldP1, S, true>(p, p.t1, arow, brow, 2 * rank + 1, s.A, s.B, s.B);
    } else {
        sub_product<FieldP1, S, true>(p, p.t1, arow, brow, rank, s.A, s.B, s.B);
    }
    if constexpr (S == 1) {
        uint32_t *out_s = reinterpret_cast<uint32_t *>(s.A);
        if constexpr (!CRT) {
            // 16-bit digits: limb k holds coefficients 2k and 2k + 1 (< 2^46 + 2^62).
            normalize_limbs(p.nout, crow, out_s, s.spill, s.flags, [&](uint32_t k) {
                return (u128)(s.B[phys(2 * k)] + (s.B[phys(2 * k + 1)] << 16));
            });
        } else {
            normalize_limbs(p.nout, crow, out_s, s.spill, s.flags, [&](uint32_t k) {
                const uint64_t r1 = zk[phys(k)];
                return (u128)r1 + (u128)garner_v(p, r1, s.B[phys(k)]) * FieldP1::P_VALUE;
            });
            if (!p.z_smem) discard_scratch(zk, buf_words(p.L));  // consumed
        }
        return;
    } else {
        const uint32_t Q = p.L / C, j0 = rank * Q;  // this CTA's positions
        cluster_sync();  // every sub-problem's result is in place
        if constexpr (!CRT) {
            // sub-problem s: in CTA s / SP, in Z for the first of two, else in B
            Remote zb;
#pragma unroll
            for (uint32_t t = 0; t < S; ++t)
                zb.base[t] = dsmem_addr(SP == 2 && t % 2 == 0 ? s.Z : s.B, t / SP);
#pragma unroll 2
            for (uint32_t h = threadIdx.x; h < Q / 2; h += blockDim.x) {
                uint64_t c0[S], c1[S];
                combine<FieldP1, S>(p.t1, zb, j0 + 2 * h, c0);
                combine<FieldP1, S>(p.t1, zb, j0 + 2 * h + 1, c1);
#pragma unroll
                for (uint32_t q = 0; q < S; ++q) {
                    BN_DEBUG_CHECK(phys(q * (Q / 2) + h) < buf_words(p.L), kDbgIndex);
                    s.A[phys(q * (Q / 2) + h)] = c0[q] + (c1[q] << 16);
                }
            }
        } else {
            const Remote z1 = remote(zk, S), z2 = remote(s.B, S);
            for (uint32_t j = threadIdx.x; j < Q; j += blockDim.x) {
                uint64_t c[S];
                combine<FieldP1, S>(p.t1, z1, j0 + j, c);
#pragma unroll
                for (uint32_t q = 0; q < S; ++q) s.A[phys(q * Q + j)] = c[q];
            }
            cluster_sync();  // the other CTA reads Z no more: it takes Garner's v
            for (uint32_t j = threadIdx.x; j < Q; j += blockDim.x) {
                uint64_t c[S];
                combine<FieldP2, S>(p.t2, z2, j0 + j, c);
#pragma unroll
                for (uint32_t q = 0; q < S; ++q) zk[phys(q * Q + j)] = garner_v(p, s.A[phys(q * Q + j)], c[q]);
            }
        }
        cluster_sync();  // the other CTA reads B no more: it becomes the staging row
        uint32_t *out_s = reinterpret_cast<uint32_t *>(s.B);
        const uint64_t *c1 = s.A, *gv = zk;
        if constexpr (!CRT) {
            // limb k of segment (q, rank) starts at A[q Q/2 + k - its first limb]
            normalize_segments<C, S>(p.nout, Q / 2, rank, crow, out_s, s.spill, s.flags, s.xflag,
                                     [&](uint32_t q, uint32_t k) {
                                         return (u128)c1[phys(q * (Q / 2) + k - (q * C + rank) * (Q / 2))];
                                     });
        } else {
            normalize_segments<C, S>(p.nout, Q, rank, crow, out_s, s.spill, s.flags, s.xflag,
                                     [&](uint32_t q, uint32_t k) {
                                         const uint32_t x = q * Q + k - (q * C + rank) * Q;
                                         return (u128)c1[phys(x)] + (u128)gv[phys(x)] * FieldP1::P_VALUE;
                                     });
        }
        // No barrier here: the other CTA reads this one's B and Z only before
        // the barrier above, and its spill and carry words only before it
        // reaches the next product's first barrier, which this CTA must reach
        // too before it writes them again.  The kernels hold a last barrier
        // before exit.
    }
}

template <bool CRT>
__device__ __forceinline__ uint64_t *zk_slot(const NttArgs &p, const Smem64 &s) {
    if constexpr (!CRT) return nullptr;
    return p.z_smem ? s.Z : p.scratch + blockIdx.x * p.scratch_stride;
}

template <bool CRT, uint32_t S>
__global__ void __launch_bounds__(1024) k_mul_ntt(NttArgs p) {
    extern __shared__ __align__(16) uint64_t sm64[];
    const Smem64 s = smem64(p, sm64);
    uint64_t *zk = zk_slot<CRT>(p, s);
    constexpr bool cl = S > 1;  // a cluster of cluster_of(S) CTAs per product
    const uint32_t rank = cl ? cluster_rank() : 0u;
    const uint64_t first = cl ? cluster_index() : blockIdx.x, stride = cl ? cluster_count() : gridDim.x;
    for (uint64_t inst = first; inst < p.batch; inst += stride)
        pair_product<CRT, S>(p, p.a + inst * p.na, p.b + inst * p.nb, p.c + inst * p.nout, s, zk, rank);
    if constexpr (cl) cluster_sync();  // no CTA exits while the other may read its shared memory
}

// Mixed-size batch of products that share the transform length N (and so
// the tables and geometry in p): the CTA (or the cluster, through its rank 0)
// takes the next item from the work queue, largest items first, and uses
// that item's sizes and rows.
template <bool CRT, uint32_t S>
__global__ void __launch_bounds__(1024)
    k_mul_ntt_batch(NttArgs p, const BatchItem *items, uint32_t count, uint32_t *queue,
                    const BatchBinding *bind) {
    extern __shared__ __align__(16) uint64_t sm64[];
    const Smem64 s = smem64(p, sm64);
    uint64_t *zk = zk_slot<CRT>(p, s);
    constexpr bool cl = S > 1;
    const uint32_t rank = cl ? cluster_rank() : 0u;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) *s.next = atomicAdd(queue, 1u);
        if (cl) cluster_sync();
        else __syncthreads();
        const uint32_t i = rank == 0 ? *s.next : ld_dsmem_u32(dsmem_addr(s.next, 0));
        if (cl) cluster_sync();  // rank 0 neither moves on nor exits before every rank has read
        else __syncthreads();
        if (i >= count) break;
        const BatchItem it = items[i];
        NttArgs q = p;
        q.na = it.na;
        q.nb = it.nb;
        q.nout = it.na + it.nb;
        q.batch = 1;
        pair_product<CRT, S>(q, bind->a + it.off_a, bind->b + it.off_b, bind->c + it.off_c, s, zk, rank);
    }
    if constexpr (cl) cluster_sync();  // no CTA exits while the other may read its shared memory
}

// ---- host side: fields, tables, plan ----------------------------------------

struct HostField {
    uint64_t p, g;  // g has order exactly 2^n
    uint32_t n;
};

uint64_t hmul(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }

uint64_t hpow(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = hmul(r, a, p);
        a = hmul(a, a, p);
        e >>= 1;
    }
    return r;
}

uint64_t hinv(uint64_t a, uint64_t p) { return hpow(a, p - 2, p); }

HostField field_p1() { return {FieldP1::P_VALUE, 21, 57}; }  // Section 4.1

HostField field_p2() {
    const uint64_t p = FieldP2::P_VALUE;  // 27 * 2^56 + 1; 5^27 has order 2^56
    return {p, hpow(5, 27, p), 56};
}

Tw64 shoup_pair(uint64_t w, uint64_t p) {
    w %= p;
    return make_ulonglong2(w, (uint64_t)(((u128)w << 64) / p));
}

// Montgomery form x R mod p (R = 2^64): the device's table generator works in it.
uint64_t mont_form(uint64_t x, uint64_t p) { return (uint64_t)((((u128)(x % p)) << 64) % p); }

uint64_t root_of_unity(const HostField &f, uint64_t m) { return hpow(f.g, (1ull << f.n) / m, f.p); }

// N^-1 R mod p: the final scale, which also cancels the 1/R of the
// Montgomery pointwise product.
uint64_t final_scale(const HostField &f, uint32_t N) {
    const uint64_t R = (uint64_t)(((u128)1 << 64) % f.p);
    return hmul(hinv(N % f.p, f.p), R, f.p);
}

// Host copy of one prime's tables.
struct HostTables {
    std::vector<Tw64> twf, twi, ffold, ifold;
    Tw64 w4{0, 0}, iw4{0, 0}, scale{0, 0};
};

HostTables make_tables(const HostField &f, uint32_t N, uint32_t S) {
    const uint32_t L = N / S;
    HostTables t;
    const uint64_t wN = root_of_unity(f, N), wL = hpow(wN, S, f.p);
    const uint64_t wLi = hinv(wL, f.p), wNi = hinv(wN, f.p);
    t.twf.assign(L, make_ulonglong2(0, 0));
    t.twi.assign(L, make_ulonglong2(0, 0));
    for (uint32_t h = 1; h < L; h <<= 1) {
        const uint64_t w = hpow(wL, L / (2 * h), f.p), wi = hpow(wLi, L / (2 * h), f.p);
        uint64_t x = 1, xi = 1;
        for (uint32_t j = 0; j < h; ++j) {
            t.twf[h + j] = shoup_pair(x, f.p);
            t.twi[h + j] = shoup_pair(xi, f.p);
            x = hmul(x, w, f.p);
            xi = hmul(xi, wi, f.p);
        }
    }
    const uint64_t scale = final_scale(f, N);
    t.scale = shoup_pair(scale, f.p);
    if (S > 1) {
        t.ffold.assign((size_t)S * L, make_ulonglong2(0, 0));
        t.ifold.assign((size_t)S * L, make_ulonglong2(0, 0));
        for (uint32_t s = 0; s < S; ++s) {
            const uint64_t ws = hpow(wN, s, f.p), wsi = hpow(wNi, s, f.p);
            uint64_t x = 1, xi = scale;
            for (uint32_t j = 0; j < L; ++j) {
                t.ffold[(size_t)s * L + j] = shoup_pair(x, f.p);
                t.ifold[(size_t)s * L + j] = shoup_pair(xi, f.p);
                x = hmul(x, ws, f.p);
                xi = hmul(xi, wsi, f.p);
            }
        }
        const uint64_t w4 = hpow(wN, N / 4, f.p);  // used when S = 4
        t.w4 = shoup_pair(w4, f.p);
        t.iw4 = shoup_pair(hinv(w4, f.p), f.p);
    }
    return t;
}

uint32_t next_pow2(uint32_t x) {
    uint32_t t = 1;
    while (t < x) t <<= 1;
    return t;
}

// Geometry of a transform product of na x nb limbs.
struct Geometry {
    uint32_t N, S, L, logL, T;
};

Geometry geometry(bool crt, uint32_t na, uint32_t nb, uint32_t cta) {
    Geometry g{};
    const uint32_t digits = crt ? na + nb : 2 * (na + nb);
    g.N = next_pow2(digits < 2 ? 2 : digits);
    g.S = g.N > kMaxSubLength ? g.N / kMaxSubLength : 1;
    g.L = g.N / g.S;
    while ((1u << g.logL) < g.L) ++g.logL;
    uint32_t T = g.L / 8;
    if (T < 32) T = 32;
    if (T > 1024) T = 1024;
    g.T = cta ? cta : T;
    return g;
}

using PlainKernel = void (*)(NttArgs);
using BatchKernel = void (*)(NttArgs, const BatchItem *, uint32_t, uint32_t *, const BatchBinding *);

// The kernels of a form and split: two primes never split more than in two
// (32-bit digits, N <= 16384).
PlainKernel plain_kernel(bool crt, uint32_t S) {
    if (crt) return S == 1 ? k_mul_ntt<true, 1> : k_mul_ntt<true, 2>;
    return S == 1 ? k_mul_ntt<false, 1> : (S == 2 ? k_mul_ntt<false, 2> : k_mul_ntt<false, 4>);
}
BatchKernel batch_kernel(bool crt, uint32_t S) {
    if (crt) return S == 1 ? k_mul_ntt_batch<true, 1> : k_mul_ntt_batch<true, 2>;
    return S == 1 ? k_mul_ntt_batch<false, 1> : (S == 2 ? k_mul_ntt_batch<false, 2> : k_mul_ntt_batch<false, 4>);
}

// Largest co-resident grid of the plain kernel for the geometry (whole
// clusters); 0 if it does not fit.
cudaError_t max_grid_of(const void *kern, const Geometry &g, uint32_t smem, int sms, uint32_t *grid) {
    *grid = 0;
    if (g.S == 1) {
        int per_sm = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)g.T, smem);
        if (e == cudaSuccess) *grid = (uint32_t)(sms * per_sm);
        return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    const uint32_t C = cluster_of(g.S);
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C * (uint32_t)sms, 1, 1);
    cfg.blockDim = dim3(g.T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e == cudaSuccess) *grid = (uint32_t)clusters * C;
    return e;
}

// Launch with clusters of cluster_of(S) CTAs when S > 1.
template <class... Args>
cudaError_t launch(void (*kern)(Args...), uint32_t grid, uint32_t threads, uint32_t smem, uint32_t S,
                   cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    if (S > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster_of(S);
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace

BN_DEBUG_ACCESSOR(debug_word_ntt)

struct NttPlan {
    bool crt = false;
    uint32_t na = 0, nb = 0, nout = 0, N = 0, L = 0, logL = 0, S = 1, threads = 0;
    uint32_t smem = 0, max_grid = 0, z_smem = 0;
    uint64_t scratch_stride = 0;
    size_t scratch_bytes = 0;
    void *dev = nullptr;          // tables followed by scratch
    uint64_t *scratch = nullptr;  // max_grid slots of scratch_stride words
    PrimeTab t1{}, t2{};
    Tw64 garner{0, 0};
};

bn_status ntt_create(NttPlan **out, bool crt, uint32_t na, uint32_t nb, const bn_tuning *tun) {
    *out = nullptr;
    if (na == 0 || nb == 0) return BN_EINVAL;
    if (na > BN_MUL_MAX_LIMBS || nb > BN_MUL_MAX_LIMBS) return BN_EUNSUPPORTED;
    uint32_t cta = 0;
    if (tun) {
        if (tun->reserved || tun->variant || tun->limbs_per_thread) return BN_EINVAL;
        if (tun->cta_threads && (tun->cta_threads % 32 || tun->cta_threads > 1024)) return BN_EINVAL;
        cta = tun->cta_threads;
    }
    const Geometry g = geometry(crt, na, nb, cta);
    NttPlan *p = new (std::nothrow) NttPlan();
    if (!p) return BN_ENOMEM;
    p->crt = crt;
    p->na = na;
    p->nb = nb;
    p->nout = na + nb;
    p->N = g.N;
    p->S = g.S;
    p->L = g.L;
    p->logL = g.logL;
    p->threads = g.T;

    cudaError_t e;
    const void *kern = (const void *)plain_kernel(crt, g.S);
    e = allow_max_smem(kern);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // A third shared buffer: for S = 4 (two sub-problems per CTA); for two
    // primes in a cluster, and for one-CTA two-prime products when it costs
    // no occupancy (else the first prime's coefficients go to scratch).
    uint32_t grid2 = 0, grid3 = 0;
    if (e == cudaSuccess) e = max_grid_of(kern, g, smem_bytes(g.L, 2, g.T), sms, &grid2);
    if (e == cudaSuccess) e = max_grid_of(kern, g, smem_bytes(g.L, 3, g.T), sms, &grid3);
    if (e != cudaSuccess) {
        delete p;
        return BN_ECUDA;
    }
    p->z_smem = (g.S == 4 || (crt && (g.S > 1 || grid3 >= grid2))) ? 1u : 0u;
    p->smem = smem_bytes(g.L, p->z_smem ? 3 : 2, g.T);
    p->max_grid = p->z_smem ? grid3 : grid2;
    if (p->max_grid == 0) {
        delete p;
        return BN_EUNSUPPORTED;
    }
    p->scratch_stride = crt && !p->z_smem ? buf_words(g.L) : 0;

    // Tables for each prime, then scratch, in one allocation.
    std::vector<HostTables> tabs;
    tabs.push_back(make_tables(field_p1(), p->N, p->S));
    if (crt) tabs.push_back(make_tables(field_p2(), p->N, p->S));
    size_t entries = 0;
    for (auto &t : tabs) entries += t.twf.size() + t.twi.size() + t.ffold.size() + t.ifold.size();
    const size_t table_bytes = (entries * sizeof(Tw64) + 255) & ~size_t(255);
    p->scratch_bytes = (size_t)p->max_grid * p->scratch_stride * 8u;
    e = cudaMalloc(&p->dev, table_bytes + p->scratch_bytes);
    if (e != cudaSuccess) {
        delete p;
        return e == cudaErrorMemoryAllocation ? BN_ENOMEM : BN_ECUDA;
    }
    std::vector<Tw64> host(table_bytes / sizeof(Tw64), make_ulonglong2(0, 0));
    size_t off = 0;
    Tw64 *dtab = static_cast<Tw64 *>(p->dev);
    for (size_t i = 0; i < tabs.size(); ++i) {
        HostTables &t = tabs[i];
        PrimeTab &pt = i == 0 ? p->t1 : p->t2;
        auto put = [&](const std::vector<Tw64> &v) -> const Tw64 * {
            if (v.empty()) return nullptr;
            std::memcpy(host.data() + off, v.data(), v.size() * sizeof(Tw64));
            const Tw64 *d = dtab + off;
            off += v.size();
            return d;
        };
        pt.twf = put(t.twf);
        pt.twi = put(t.twi);
        pt.ffold = put(t.ffold);
        pt.ifold = put(t.ifold);
        pt.w4 = t.w4;
        pt.iw4 = t.iw4;
        pt.scale = t.scale;
    }
    e = cudaMemcpy(p->dev, host.data(), table_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->dev);
        delete p;
        return BN_ECUDA;
    }
    p->scratch = reinterpret_cast<uint64_t *>(static_cast<char *>(p->dev) + table_bytes);
    const HostField f1 = field_p1(), f2 = field_p2();
    p->garner = shoup_pair(hinv(f1.p % f2.p, f2.p), f2.p);
    *out = p;
    return BN_OK;
}

void ntt_destroy(NttPlan *p) {
    if (!p) return;
    cudaFree(p->dev);
    delete p;
}

size_t ntt_scratch_bytes(const NttPlan *p) { return p ? p->scratch_bytes : 0; }

uint32_t ntt_length(const NttPlan *p) { return p ? p->N : 0; }

namespace {

NttArgs plan_args(const NttPlan *p) {
    NttArgs args{};
    args.na = p->na;
    args.nb = p->nb;
    args.nout = p->nout;
    args.N = p->N;
    args.L = p->L;
    args.logL = p->logL;
    args.S = p->S;
    args.digit_bits = p->crt ? 32 : 16;
    args.z_smem = p->z_smem;
    args.scratch = p->scratch;
    args.scratch_stride = p->scratch_stride;
    args.garner = p->garner;
    args.t1 = p->t1;
    args.t2 = p->t2;
    return args;
}

// Grid for `units` products: persistent, at most max_grid CTAs, whole clusters.
uint32_t grid_for(const NttPlan *p, uint64_t units) {
    const uint64_t ctas = units * cluster_of(p->S);
    return (uint32_t)(ctas < p->max_grid ? ctas : p->max_grid);
}

}  // namespace

cudaError_t ntt_launch(NttPlan *p, const uint32_t *a, const uint32_t *b, uint32_t *c,
                       uint64_t batch, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    NttArgs args = plan_args(p);
    args.a = a;
    args.b = b;
    args.c = c;
    args.batch = batch;
    const uint32_t grid = grid_for(p, batch);
    return launch(plain_kernel(p->crt, p->S), grid, p->threads, p->smem, p->S, st, args);
}

cudaError_t ntt_launch_sized(NttPlan *p, uint32_t na, uint32_t nb, const uint32_t *a,
                             const uint32_t *b, uint32_t *c, cudaStream_t st) {
    NttArgs args = plan_args(p);
    args.a = a;
    args.b = b;
    args.c = c;
    args.na = na;
    args.nb = nb;
    args.nout = na + nb;
    args.batch = 1;
    return launch(plain_kernel(p->crt, p->S), cluster_of(p->S), p->threads, p->smem, p->S, st, args);
}

bn_status ntt_batch_plan(NttPlan **out, bool crt, uint32_t N) {
    // A plan whose transform length is exactly N: digits(a) + digits(b) = N.
    if (N < 4 || (N & (N - 1))) return BN_EINVAL;
    const uint32_t per_side = crt ? N / 2 : N / 4;
    if (per_side > BN_MUL_MAX_LIMBS) return BN_EUNSUPPORTED;
    const bn_status st = ntt_create(out, crt, per_side, per_side, nullptr);
    if (st != BN_OK) return st;
    if (allow_max_smem((const void *)batch_kernel(crt, (*out)->S)) != cudaSuccess) {
        ntt_destroy(*out);
        *out = nullptr;
        return BN_ECUDA;
    }
    return BN_OK;
}

cudaError_t ntt_batch_launch(NttPlan *p, const BatchItem *items, uint32_t count, uint32_t *queue,
                             const BatchBinding *bind, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const NttArgs args = plan_args(p);
    const uint32_t grid = grid_for(p, count);
    const BatchKernel kern = batch_kernel(p->crt, p->S);
    if (cudaError_t e = allow_max_smem((const void *)kern)) return e;
    return launch(kern, grid, p->threads, p->smem, p->S, st, args, items, count, queue, bind);
}

// ---- transform multiplication without allocation ------------------------
//
// bn_mul_ntt_noalloc (include/bn.h) runs the same kernel as the plans above,
// but its scratch and twiddle tables live in two file-scope device arrays
// instead of plan-owned memory, for callers that cannot call cudaMalloc.  The
// tables are generated by a small kernel on the caller's stream, so neither
// host nor device memory is allocated on any call.

namespace {

constexpr size_t kNoAllocScratchWords = BN_NOALLOC_SCRATCH_BYTES / 8;
// Largest table set: two primes at N = 16384 split into two 8192-point
// halves, each prime holding twf + twi (2 L) and both folds (2 N) entries.
constexpr size_t kNoAllocTableEntries = 2 * (2 * 8192 + 2 * 16384);
static_assert(kNoAllocTableEntries >= 2 * 8192 + 2 * 32768, "one prime at N = 32768 fits");

static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocScratchWords];
static __device__ __align__(256) Tw64 g_noalloc_tables[kNoAllocTableEntries];

constexpr int kNoAllocMaxDevices = 64;
struct NoAllocDevice {
    bool ready = false;
    uint64_t *scratch = nullptr;  // device addresses of the arrays
    Tw64 *tables = nullptr;
    int sms = 0;
    bool have_tables = false;  // the table array holds (crt, N)
    bool crt = false;
    uint32_t N = 0;
    // Set once a call has been captured into a graph: a replay of that graph
    // rewrites the table array at a time the host cannot see, so from then
    // on every call regenerates its tables.
    bool captured = false;
};
NoAllocDevice g_noalloc_devices[kNoAllocMaxDevices];
std::mutex g_noalloc_mutex;

// x^e in Montgomery form (x and one in Montgomery form).
template <class F>
__device__ uint64_t form_pow(uint64_t base, uint64_t e, uint64_t one) {
    uint64_t r = one;
    while (e) {
        if (e & 1) r = F::mont(r, base);
        base = F::mont(base, base);
        e >>= 1;
    }
    return r;
}

// Shoup pair of the Montgomery-form value xf: w = xf / R canonical (a
// Montgomery product by 1), and floor(w 2^64 / P) by binary long division
// (w < P < 2^62, so the running remainder doubled stays below 2^63).
template <class F>
__device__ Tw64 shoup_of_form(uint64_t xf) {
    const uint64_t w = F::canon(F::mont(xf, 1));
    uint64_t r = w, q = 0;
    for (int i = 0; i < 64; ++i) {
        r <<= 1;
        q <<= 1;
        if (r >= F::P_VALUE) {
            r -= F::P_VALUE;
            q |= 1;
        }
    }
    return make_ulonglong2(w, q);
}

// One prime's tables (layout twf[L] | twi[L] | ffold[S L] | ifold[S L]), the
// same values the plans build on the host; inputs in Montgomery form.
template <class F>
__global__ void k_noalloc_tables(Tw64 *tab, uint32_t L, uint32_t S, uint64_t one, uint64_t wL,
                                 uint64_t wLi, uint64_t wN, uint64_t wNi, uint64_t scale) {
    const uint32_t total = 2 * L + (S > 1 ? 2 * S * L : 0);
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += gridDim.x * blockDim.x) {
        uint64_t v;
        if (idx < 2 * L) {
            const uint32_t inv = idx >= L, i = idx - inv * L;
            v = 0;
            if (i > 0) {
                const uint32_t h = 1u << (31 - __clz(i)), j = i - h;
                v = form_pow<F>(form_pow<F>(inv ? wLi : wL, L / (2 * h), one), j, one);
            }
        } else {
            const uint32_t k = idx - 2 * L, inv = k >= S * L, r = k - inv * S * L;
            const uint32_t sidx = r / L, j = r - sidx * L;
            const uint64_t w = form_pow<F>(inv ? wNi : wN, (uint64_t)j * sidx, one);
            v = inv ? F::mont(scale, w) : w;
        }
        tab[idx] = shoup_of_form<F>(v);
    }
}

// Host constants of one prime for (N, S); no allocation.
struct NoAllocPrime {
    uint64_t one, wL, wLi, wN, wNi, scale;  // Montgomery form, for the generator
    PrimeTab tab;
};

NoAllocPrime noalloc_prime(const HostField &f, uint32_t N, uint32_t S, Tw64 *dtab) {
    NoAllocPrime c{};
    const uint32_t L = N / S;
    const uint64_t wN = root_of_unity(f, N), wL = hpow(wN, S, f.p);
    const uint64_t scale = final_scale(f, N);
    c.one = mont_form(1, f.p);
    c.wL = mont_form(wL, f.p);
    c.wLi = mont_form(hinv(wL, f.p), f.p);
    c.wN = mont_form(wN, f.p);
    c.wNi = mont_form(hinv(wN, f.p), f.p);
    c.scale = mont_form(scale, f.p);
    c.tab.twf = dtab;
    c.tab.twi = dtab + L;
    c.tab.ffold = S > 1 ? dtab + 2 * L : nullptr;
    c.tab.ifold = S > 1 ? dtab + 2 * L + (size_t)S * L : nullptr;
    c.tab.scale = shoup_pair(scale, f.p);
    if (S > 1) {
        const uint64_t w4 = hpow(wN, N / 4, f.p);
        c.tab.w4 = shoup_pair(w4, f.p);
        c.tab.iw4 = shoup_pair(hinv(w4, f.p), f.p);
    }
    return c;
}

size_t noalloc_prime_entries(uint32_t N, uint32_t S) {
    return 2 * (N / S) + (S > 1 ? 2 * (size_t)N : 0);
}

}  // namespace

}  // namespace bn

extern "C" bn_status bn_mul_ntt_noalloc(const uint32_t *a, const uint32_t *b, uint32_t *c,
                                        uint32_t na, uint32_t nb, uint64_t batch, int crt_flag,
                                        void *stream) {
    using namespace bn;
    if (na == 0 || nb == 0) {
        record_error("zero limb count");
        return BN_EINVAL;
    }
    if (na > BN_NOALLOC_MAX_LIMBS || nb > BN_NOALLOC_MAX_LIMBS) {
        record_error("operand above BN_NOALLOC_MAX_LIMBS (8192 limbs) for bn_mul_ntt_noalloc");
        return BN_EUNSUPPORTED;
    }
    if (batch == 0) return BN_OK;
    if (!a || !b || !c) {
        record_error("null operand or result pointer");
        return BN_EINVAL;
    }
    const uint32_t nout = na + nb;
    {
        const uintptr_t ca = (uintptr_t)c, ce = ca + batch * nout * 4ull;
        const uintptr_t aa = (uintptr_t)a, ae = aa + batch * na * 4ull;
        const uintptr_t ba = (uintptr_t)b, be = ba + batch * nb * 4ull;
        if ((ca < ae && aa < ce) || (ca < be && ba < ce)) {
            record_error("result overlaps an operand");
            return BN_EINVAL;
        }
    }
    const bool crt = crt_flag != 0;
    cudaStream_t st = (cudaStream_t)stream;
    // Geometry, as for a plan; the first prime's coefficients of a two-prime
    // product go to the scratch array unless the transform is split.
    const Geometry g = geometry(crt, na, nb, 0);
    const PlainKernel kern = plain_kernel(crt, g.S);
    const uint32_t z_smem = g.S == 4 || (crt && g.S > 1) ? 1u : 0u;
    const uint32_t smem = smem_bytes(g.L, z_smem ? 3 : 2, g.T);
    const uint64_t stride = crt && !z_smem ? buf_words(g.L) : 0;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        record_error("no usable current device for bn_mul_ntt_noalloc");
        return BN_ECUDA;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) {
        record_error("bn_mul_ntt_noalloc: cudaStreamIsCapturing failed on the stream");
        return BN_ECUDA;
    }
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocDevice &d = g_noalloc_devices[dev];
    if (!d.ready && capturing) {
        record_error("bn_mul_ntt_noalloc: the first call on a device must come before stream capture");
        return BN_EINVAL;
    }
    if (!d.ready) {  // once per device, with that device current
        void *ps = nullptr, *pt = nullptr;
        int optin = 0;
        e = cudaGetSymbolAddress(&ps, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&pt, g_noalloc_tables);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const PlainKernel all[] = {plain_kernel(false, 1), plain_kernel(false, 2), plain_kernel(false, 4),
                                   plain_kernel(true, 1), plain_kernel(true, 2)};
        for (PlainKernel k : all)
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) {
            record_error("bn_mul_ntt_noalloc device set-up failed");
            return BN_ECUDA;
        }
        d.scratch = static_cast<uint64_t *>(ps);
        d.tables = static_cast<Tw64 *>(pt);
        d.ready = true;
    }
    uint32_t max_grid = 0;
    e = max_grid_of((const void *)kern, g, smem, d.sms, &max_grid);
    if (e != cudaSuccess || max_grid == 0) {
        record_error("bn_mul_ntt_noalloc: kernel does not fit on this device");
        return BN_ECUDA;
    }
    if (stride > 0 && kNoAllocScratchWords / stride < max_grid) max_grid = (uint32_t)(kNoAllocScratchWords / stride);

    const NoAllocPrime c1 = noalloc_prime(field_p1(), g.N, g.S, d.tables);
    const NoAllocPrime c2 = noalloc_prime(field_p2(), g.N, g.S, d.tables + noalloc_prime_entries(g.N, g.S));
    // A captured call records its own table kernel (replays regenerate the
    // tables they read) and leaves the host's record of the table contents
    // unusable for every later call.
    if (capturing) d.captured = true;
    if (capturing || d.captured || !d.have_tables || d.crt != crt || d.N != g.N) {
        const uint32_t entries = (uint32_t)noalloc_prime_entries(g.N, g.S);
        const unsigned blocks = (entries + 255) / 256 < 1024 ? (entries + 255) / 256 : 1024;
        k_noalloc_tables<FieldP1><<<blocks, 256, 0, st>>>(d.tables, g.L, g.S, c1.one, c1.wL, c1.wLi,
                                                           c1.wN, c1.wNi, c1.scale);
        if (crt)
            k_noalloc_tables<FieldP2><<<blocks, 256, 0, st>>>(d.tables + entries, g.L, g.S, c2.one, c2.wL,
                                                               c2.wLi, c2.wN, c2.wNi, c2.scale);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            d.have_tables = false;
            record_error("bn_mul_ntt_noalloc table kernel launch failed");
            return BN_ECUDA;
        }
        d.have_tables = !d.captured;
        d.crt = crt;
        d.N = g.N;
    }

    NttArgs args{};
    args.a = a;
    args.b = b;
    args.c = c;
    args.na = na;
    args.nb = nb;
    args.nout = nout;
    args.N = g.N;
    args.L = g.L;
    args.logL = g.logL;
    args.S = g.S;
    args.digit_bits = crt ? 32 : 16;
    args.z_smem = z_smem;
    args.batch = batch;
    args.scratch = d.scratch;
    args.scratch_stride = stride;
    args.garner = shoup_pair(hinv(field_p1().p % field_p2().p, field_p2().p), field_p2().p);
    args.t1 = c1.tab;
    args.t2 = c2.tab;
    const uint64_t ctas = batch * cluster_of(g.S);
    const uint32_t grid = (uint32_t)(ctas < max_grid ? ctas : max_grid);
    e = launch(kern, grid, g.T, smem, g.S, st, args);
    if (e != cudaSuccess) {
        record_error("bn_mul_ntt_noalloc kernel launch failed");
        return BN_ECUDA;
    }
    return BN_OK;
}
