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
// both primes use a lazy Montgomery multiplication (R = 2^64, values kept in
// [0, 2p)) that is cheap because each prime's low 32-bit word is 1 (see
// MontField).  Twiddles are stored in Montgomery form so that
// mul(x, form(w)) = x*w; the pointwise product and the final 1/N scale absorb
// Montgomery's extra 1/R.
//
// Work mapping.  One CTA transforms one integer pair at a time in shared
// memory (a persistent grid walks the batch).  Forward transforms are
// decimation-in-frequency (natural order in, bit-reversed out), the inverse
// is decimation-in-time (bit-reversed in, natural out), so no permutation
// pass is needed (Section 4.2's fft reorders first).  Stages are grouped into
// radix-8 passes: a thread loads 8 elements, runs 3 butterfly stages in
// registers and stores them back, one barrier per pass instead of one per
// stage.
//
// Sizes beyond shared memory.  Both spectra of a sub-transform of length L
// must fit (L <= 8192 u64 each).  A longer transform, N = S*L with S in
// {2, 4}, is split into S independent length-L problems: the first radix-S
// decimation-in-frequency stage is folded into the digit load (sub-problem s
// transforms y_s[j] = w_N^{js} sum_r x[j + rL] w_S^{rs}), each sub-problem is
// multiplied pointwise and inverted on its own, and the last radix-S inverse
// stage is folded into the final combine, reading the S partial results back
// from a per-CTA scratch slot (L2-resident, since the grid is persistent).
//
// Normalisation (Section 4.2's splitFftReg/baddRegMul2Fft, here with whole
// 16/32-bit digits).  Each thread folds the coefficients of its window of
// limbs into limbs plus a carried spill, the spill is added into the next
// window, and the remaining one-bit carries are resolved with the Section 2
// carry scan across threads.
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

// ---- device fields ---------------------------------------------------------

// Z_P for a prime P = k 2^m + 1 with m >= 32 (so P's low 32-bit word is 1)
// and P < 2^62, in Montgomery form with R = 2^64.  Elements are kept lazily
// in [0, 2P); canon() maps to [0, P).
//   * mul: for a, b < 2P the 128-bit product comes from four 32x32->64
//     multiply-adds with no carry handling (a, b < 2^63 keep the cross sum
//     below 2^64).  Reduction: -P^-1 = P - 2 (mod 2^64), so the quotient
//     m = t_lo (P - 2) has words (-x0, x0*P_hi - x1 - borrow); m*P needs two
//     more multiply-adds since P's low word is 1; the result is < 2P because
//     4P < 2^64.
template <uint64_t P>
struct MontField {
    using Elem = uint64_t;
    using Tw = uint64_t;  // twiddles in Montgomery form
    static constexpr uint64_t P_VALUE = P;
    static constexpr uint32_t PH = (uint32_t)(P >> 32);
    static constexpr uint64_t TWO_P = 2 * P;
    static_assert((P & 0xffffffffull) == 1 && P < (1ull << 62), "P = k 2^m + 1, m >= 32, P < 2^62");
    __device__ static __forceinline__ uint64_t add(uint64_t a, uint64_t b) {
        const uint64_t r = a + b;
        return r >= TWO_P ? r - TWO_P : r;
    }
    __device__ static __forceinline__ uint64_t sub(uint64_t a, uint64_t b) {
        const uint64_t r = a + TWO_P - b;
        return r >= TWO_P ? r - TWO_P : r;
    }
    __device__ static __forceinline__ uint64_t canon(uint64_t a) { return a >= P ? a - P : a; }
    // a * b / 2^64 mod P, inputs and output in [0, 2P).
    __device__ static __forceinline__ uint64_t mul(uint64_t a, uint64_t b) {
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
    // a * b / 2^64 mod P for any 64-bit a and a canonical b < P (a twiddle):
    // a*b < P 2^64 keeps the result in [0, 2P); the cross sum takes one more
    // add because a's high word may use all 32 bits.
    __device__ static __forceinline__ uint64_t mulw(uint64_t a, uint64_t b) {
        const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
        const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
        const uint64_t p00 = (uint64_t)a0 * b0;
        const uint64_t t1 = (uint64_t)a1 * b0 + (p00 >> 32);
        const uint64_t t2 = (uint64_t)a0 * b1 + (uint32_t)t1;
        const uint64_t hi = (uint64_t)a1 * b1 + (t1 >> 32) + (t2 >> 32);
        const uint32_t x0 = (uint32_t)p00, x1 = (uint32_t)t2;
        const uint32_t m0 = 0u - x0;
        const uint32_t m1 = x0 * PH - x1 - (x0 != 0u);
        const uint64_t sm = (uint64_t)m0 * PH + m1;
        const uint64_t h = (uint64_t)m1 * PH + (sm >> 32);
        return hi + h + ((x0 | x1) != 0u);
    }
    __device__ static __forceinline__ uint64_t twiddle(uint64_t a, uint64_t w) { return mulw(a, w); }
    __device__ static __forceinline__ uint64_t twiddle_lazy(uint64_t a, uint64_t w) { return mul(a, w); }
};

using FieldP1 = MontField<4179340454199820289ull>;  // 29 * 2^57 + 1 (PrimeField64)
using FieldP2 = MontField<1945555039024054273ull>;  // 27 * 2^56 + 1

struct PrimeTab {
    const uint64_t *twf;    // [L]: twf[h + j] = w_{2h}^j (h = 1 .. L/2, j < h)
    const uint64_t *twi;    // [L]: w_{2h}^-j
    const uint64_t *ffold;  // [S*L]: w_N^{js}            (S > 1)
    const uint64_t *ifold;  // [S*L]: scale * w_N^{-js}   (S > 1)
    uint64_t ws[4], iws[4]; // w_S^k, w_S^-k
    uint64_t scale;         // N^-1 (times R for p1), S == 1
};

struct NttArgs {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t na, nb, nout;
    uint32_t N, L, logL, S, digit_bits;
    uint64_t batch;
    uint64_t *scratch;
    uint64_t scratch_stride;  // u64 words per CTA
    uint64_t garner_inv;      // p1^-1 mod p2
    PrimeTab t1, t2;
};

__device__ __forceinline__ uint64_t digit(const uint32_t *row, uint32_t ndig, uint32_t m,
                                          uint32_t bits) {
    if (m >= ndig) return 0;
    return bits == 16 ? (row[m >> 1] >> ((m & 1u) << 4)) & 0xFFFFu : row[m];
}

// Sub-problem s of the forward transform: y_s[j] = w_N^{js} sum_r x[j + rL] w_S^{rs}.
// For S = 2 and 4 the inner sum is a radix-S butterfly: w_2 = w_4^2 = -1, so
// only w_4 (times x1 - x3) takes a product, and w_N^0 = 1 takes none.
template <class F>
__device__ void load_fold(const NttArgs &p, const PrimeTab &tb, const uint32_t *row, uint32_t n,
                          uint32_t s, uint64_t *buf) {
    const uint32_t ndig = p.digit_bits == 16 ? 2 * n : n;
    if (p.S == 2 || p.S == 4) {
        for (uint32_t j = threadIdx.x; j < p.L; j += blockDim.x) {
            const uint64_t x0 = digit(row, ndig, j, p.digit_bits), x1 = digit(row, ndig, j + p.L, p.digit_bits);
            uint64_t acc;
            if (p.S == 2) {
                acc = s == 0 ? F::add(x0, x1) : F::sub(x0, x1);
            } else {
                const uint64_t x2 = digit(row, ndig, j + 2 * p.L, p.digit_bits);
                const uint64_t x3 = digit(row, ndig, j + 3 * p.L, p.digit_bits);
                if (s == 0) acc = F::add(F::add(x0, x2), F::add(x1, x3));
                else if (s == 2) acc = F::sub(F::add(x0, x2), F::add(x1, x3));
                else {
                    const uint64_t o = F::sub(x0, x2), q = F::mul(F::sub(x1, x3), tb.ws[1]);
                    acc = s == 1 ? F::add(o, q) : F::sub(o, q);
                }
            }
            if (s != 0) acc = F::mul(acc, tb.ffold[s * p.L + j]);
            buf[phys(j)] = acc;
        }
        return;
    }
    for (uint32_t j = threadIdx.x; j < p.L; j += blockDim.x) {
        uint64_t acc = digit(row, ndig, j, p.digit_bits);
        if (p.S > 1) {
            for (uint32_t r = 1; r < p.S; ++r) {
                const uint32_t m = j + r * p.L;
                if (m >= ndig) break;
                const uint64_t d = digit(row, ndig, m, p.digit_bits);
                const uint32_t k = (r * s) & (p.S - 1);
                acc = F::add(acc, k == 0 ? d : F::mul(d, tb.ws[k]));
            }
            acc = F::mul(acc, tb.ffold[s * p.L + j]);
        }
        buf[phys(j)] = acc;
    }
}

// Forward / inverse transforms of a sub-problem: the compile-time passes for
// the lengths the 16K..256K-bit range uses most (L = 4096 and 8192 with their
// default thread counts; 7-8% faster), the runtime passes otherwise.
template <class F>
__device__ __forceinline__ void forward_sub(const NttArgs &p, const uint64_t *tw, uint64_t *A, uint64_t *B) {
    if (p.logL == 13 && blockDim.x == 1024) forward2_c<F, 13, 1024>(tw, A, B);
    else if (p.logL == 12 && blockDim.x == 512) forward2_c<F, 12, 512>(tw, A, B);
    else forward2<F>(p.L, p.logL, tw, A, B);
}

template <class F>
__device__ __forceinline__ void inverse_sub(const NttArgs &p, const uint64_t *tw, uint64_t *B) {
    if (p.logL == 13 && blockDim.x == 1024) inverse_c<F, 13, 1024>(tw, B);
    else if (p.logL == 12 && blockDim.x == 512) inverse_c<F, 12, 512>(tw, B);
    else inverse<F>(p.L, p.logL, tw, B);
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

// Coefficients of a*b mod the field's prime, scaled by 1/N.  With keep and
// S == 1 they stay in B (padded layout); otherwise they go to dest[0 .. N).
template <class F>
__device__ void prime_product(const NttArgs &p, const PrimeTab &tb, const uint32_t *arow,
                              const uint32_t *brow, uint64_t *A, uint64_t *B, uint64_t *Z,
                              uint64_t *dest, bool keep) {
    for (uint32_t s = 0; s < p.S; ++s) {
        load_fold<F>(p, tb, arow, p.na, s, A);   // n1: digits (and the folded first stage)
        load_fold<F>(p, tb, brow, p.nb, s, B);
        __syncthreads();
        forward_sub<F>(p, tb.twf, A, B);          // n2: forward transforms
        for (uint32_t j = threadIdx.x; j < p.L; j += blockDim.x)   // n3: pointwise
            B[phys(j)] = F::mul(A[phys(j)], B[phys(j)]);
        __syncthreads();
        inverse_sub<F>(p, tb.twi, B);             // n4: inverse transform (unscaled)
        if (p.S > 1) {
            for (uint32_t j = threadIdx.x; j < p.L; j += blockDim.x) Z[s * p.L + j] = B[phys(j)];
            __syncthreads();
        }
    }
    if (p.S == 1) {
        for (uint32_t j = threadIdx.x; j < p.L; j += blockDim.x) {
            const uint64_t v = F::canon(F::mul(B[phys(j)], tb.scale));
            if (keep) B[phys(j)] = v;
            else dest[j] = v;
        }
    } else {
        // Last radix-S inverse stage: c[j + rL] = sum_s w_S^{-rs} (scale w_N^{-js} z_s[j]);
        // for S = 2 and 4 a radix-S butterfly with one product, by w_4^-1.
        for (uint32_t j = threadIdx.x; j < p.L; j += blockDim.x) {
            uint64_t u[4];
            for (uint32_t s = 0; s < p.S; ++s) u[s] = F::mul(Z[s * p.L + j], tb.ifold[s * p.L + j]);
            if (p.S == 2) {
                dest[j] = F::canon(F::add(u[0], u[1]));
                dest[j + p.L] = F::canon(F::sub(u[0], u[1]));
                continue;
            }
            if (p.S == 4) {
                const uint64_t e0 = F::add(u[0], u[2]), e1 = F::add(u[1], u[3]);
                const uint64_t o0 = F::sub(u[0], u[2]), o1 = F::mul(F::sub(u[1], u[3]), tb.iws[1]);
                dest[j] = F::canon(F::add(e0, e1));
                dest[j + p.L] = F::canon(F::add(o0, o1));
                dest[j + 2 * p.L] = F::canon(F::sub(e0, e1));
                dest[j + 3 * p.L] = F::canon(F::sub(o0, o1));
                continue;
            }
            for (uint32_t r = 0; r < p.S; ++r) {
                uint64_t acc = u[0];
                for (uint32_t s = 1; s < p.S; ++s) {
                    const uint32_t k = (r * s) & (p.S - 1);
                    acc = F::add(acc, k == 0 ? u[s] : F::mul(u[s], tb.iws[k]));
                }
                dest[j + r * p.L] = F::canon(acc);
            }
        }
        __syncthreads();
        discard_scratch(Z, p.N);  // the partial results are consumed
    }
    __syncthreads();
}

// Limb k's share of the product: the digit coefficients that start in limb k.
template <bool CRT>
__device__ __forceinline__ u128 limb_value(const NttArgs &p, uint32_t k, const uint64_t *B,
                                           bool in_smem, const uint64_t *C1, const uint64_t *Cs) {
    if constexpr (!CRT) {
        const uint64_t c0 = in_smem ? B[phys(2 * k)] : Cs[2 * k];
        const uint64_t c1 = in_smem ? B[phys(2 * k + 1)] : Cs[2 * k + 1];
        return (u128)(c0 + (c1 << 16));  // < 2^46 + 2^62
    } else {
        const uint64_t r1 = C1[k];                     // canonical mod p1
        const uint64_t r2 = in_smem ? B[phys(k)] : Cs[k];  // canonical mod p2
        // Garner: c = r1 + p1 * ((r2 - r1) p1^-1 mod p2), exact since c < p1 p2.
        uint64_t r1m = r1;                             // r1 mod p2 (p1 < 3 p2)
        if (r1m >= FieldP2::P_VALUE) r1m -= FieldP2::P_VALUE;
        if (r1m >= FieldP2::P_VALUE) r1m -= FieldP2::P_VALUE;
        const uint64_t d = r2 >= r1m ? r2 - r1m : r2 + FieldP2::P_VALUE - r1m;
        const uint64_t v = FieldP2::canon(FieldP2::mul(d, p.garner_inv));
        return (u128)r1 + (u128)v * FieldP1::P_VALUE;
    }
}

template <bool CRT>
__device__ void normalize(const NttArgs &p, uint64_t inst, uint32_t *out_s, const uint64_t *B,
                          bool in_smem, const uint64_t *C1, const uint64_t *Cs, uint64_t *spill,
                          uint32_t *flags) {
    normalize_limbs(p.nout, p.c + inst * p.nout, out_s, spill, flags,
                    [&](uint32_t k) { return limb_value<CRT>(p, k, B, in_smem, C1, Cs); });
}

template <bool CRT>
__global__ void __launch_bounds__(1024) k_mul_ntt(NttArgs p) {
    extern __shared__ __align__(16) uint64_t sm64[];
    const uint32_t Lp = phys_words(p.L);
    uint64_t *A = sm64;
    uint64_t *B = sm64 + ((Lp + 1) & ~1u);
    uint64_t *spill = B + ((Lp + 1) & ~1u);
    uint32_t *flags = reinterpret_cast<uint32_t *>(spill + blockDim.x);
    uint64_t *scr = p.scratch + blockIdx.x * p.scratch_stride;
    uint64_t *Z = scr;                                  // [N] partial results (S > 1)
    uint64_t *C1 = scr + (p.S > 1 ? p.N : 0);           // [N] p1 coefficients (CRT)
    uint64_t *Cs = C1 + (CRT ? p.N : 0);                // [N] final-prime coefficients (S > 1)
    for (uint64_t inst = blockIdx.x; inst < p.batch; inst += gridDim.x) {
        const uint32_t *arow = p.a + inst * p.na, *brow = p.b + inst * p.nb;
        const bool keep = p.S == 1;
        if constexpr (CRT) {
            prime_product<FieldP1>(p, p.t1, arow, brow, A, B, Z, C1, false);
            prime_product<FieldP2>(p, p.t2, arow, brow, A, B, Z, Cs, keep);
        } else {
            prime_product<FieldP1>(p, p.t1, arow, brow, A, B, Z, Cs, keep);
        }
        normalize<CRT>(p, inst, reinterpret_cast<uint32_t *>(A), B, keep, C1, Cs, spill, flags);
        if (CRT) discard_scratch(C1, p.N);  // the coefficients are consumed
        if (!keep) discard_scratch(Cs, p.N);
    }
}

// Mixed-size batch of products that share the transform length N (and so
// the tables and geometry in p): the CTA takes the next item from the work
// queue, largest items first, and uses that item's sizes and rows.
template <bool CRT>
__global__ void __launch_bounds__(1024)
    k_mul_ntt_batch(NttArgs p, const BatchItem *items, uint32_t count, uint32_t *queue,
                    const BatchBinding *bind) {
    extern __shared__ __align__(16) uint64_t sm64[];
    __shared__ uint32_t next;
    const uint32_t Lp = phys_words(p.L);
    uint64_t *A = sm64;
    uint64_t *B = sm64 + ((Lp + 1) & ~1u);
    uint64_t *spill = B + ((Lp + 1) & ~1u);
    uint32_t *flags = reinterpret_cast<uint32_t *>(spill + blockDim.x);
    uint64_t *scr = p.scratch + blockIdx.x * p.scratch_stride;
    uint64_t *Z = scr;
    uint64_t *C1 = scr + (p.S > 1 ? p.N : 0);
    uint64_t *Cs = C1 + (CRT ? p.N : 0);
    for (;;) {
        __syncthreads();  // the previous item is stored before `next` moves on
        if (threadIdx.x == 0) next = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t i = next;
        if (i >= count) break;
        const BatchItem it = items[i];
        NttArgs q = p;
        q.a = bind->a + it.off_a;
        q.b = bind->b + it.off_b;
        q.c = bind->c + it.off_c;
        q.na = it.na;
        q.nb = it.nb;
        q.nout = it.na + it.nb;
        q.batch = 1;
        const bool keep = q.S == 1;
        if constexpr (CRT) {
            prime_product<FieldP1>(q, q.t1, q.a, q.b, A, B, Z, C1, false);
            prime_product<FieldP2>(q, q.t2, q.a, q.b, A, B, Z, Cs, keep);
        } else {
            prime_product<FieldP1>(q, q.t1, q.a, q.b, A, B, Z, Cs, keep);
        }
        normalize<CRT>(q, 0, reinterpret_cast<uint32_t *>(A), B, keep, C1, Cs, spill, flags);
        if (CRT) discard_scratch(C1, q.N);  // the coefficients are consumed
        if (!keep) discard_scratch(Cs, q.N);
    }
}

// ---- host side: fields, tables, plan ----------------------------------------

struct HostField {
    uint64_t p, g;  // g has order exactly 2^n
    uint32_t n;
    bool montgomery;
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

HostField field_p1() { return {FieldP1::P_VALUE, 21, 57, true}; }  // Section 4.1

HostField field_p2() {
    const uint64_t p = FieldP2::P_VALUE;  // 27 * 2^56 + 1; 5^27 has order 2^56
    return {p, hpow(5, 27, p), 56, true};
}

// The form in which the device keeps constants: mul(x, form(w)) = x*w.
uint64_t to_form(const HostField &f, uint64_t x) {
    return f.montgomery ? (uint64_t)((((u128)x) << 64) % f.p) : x;
}

uint64_t root_of_unity(const HostField &f, uint64_t m) { return hpow(f.g, (1ull << f.n) / m, f.p); }

// Host copy of one prime's tables; offsets are in u64 words.
struct HostTables {
    std::vector<uint64_t> twf, twi, ffold, ifold;
    uint64_t ws[4] = {0, 0, 0, 0}, iws[4] = {0, 0, 0, 0}, scale = 0;
};

HostTables make_tables(const HostField &f, uint32_t N, uint32_t S) {
    const uint32_t L = N / S;
    HostTables t;
    const uint64_t wN = root_of_unity(f, N), wL = hpow(wN, S, f.p);
    const uint64_t wLi = hinv(wL, f.p), wNi = hinv(wN, f.p);
    t.twf.assign(L, 0);
    t.twi.assign(L, 0);
    for (uint32_t h = 1; h < L; h <<= 1) {
        const uint64_t w = hpow(wL, L / (2 * h), f.p), wi = hpow(wLi, L / (2 * h), f.p);
        uint64_t x = 1, xi = 1;
        for (uint32_t j = 0; j < h; ++j) {
            t.twf[h + j] = to_form(f, x);
            t.twi[h + j] = to_form(f, xi);
            x = hmul(x, w, f.p);
            xi = hmul(xi, wi, f.p);
        }
    }
    // 1/N, times R for Montgomery fields (the pointwise product divided by R).
    const uint64_t R = f.montgomery ? (uint64_t)(((u128)1 << 64) % f.p) : 1;
    const uint64_t scale = hmul(hinv(N % f.p, f.p), R, f.p);
    t.scale = to_form(f, scale);
    if (S > 1) {
        t.ffold.assign((size_t)S * L, 0);
        t.ifold.assign((size_t)S * L, 0);
        for (uint32_t s = 0; s < S; ++s) {
            const uint64_t ws = hpow(wN, s, f.p), wsi = hpow(wNi, s, f.p);
            uint64_t x = 1, xi = scale;
            for (uint32_t j = 0; j < L; ++j) {
                t.ffold[(size_t)s * L + j] = to_form(f, x);
                t.ifold[(size_t)s * L + j] = to_form(f, xi);
                x = hmul(x, ws, f.p);
                xi = hmul(xi, wsi, f.p);
            }
        }
        const uint64_t wS = hpow(wN, N / S, f.p), wSi = hinv(wS, f.p);
        for (uint32_t k = 0; k < S; ++k) {
            t.ws[k] = to_form(f, hpow(wS, k, f.p));
            t.iws[k] = to_form(f, hpow(wSi, k, f.p));
        }
    }
    return t;
}

uint32_t next_pow2(uint32_t x) {
    uint32_t t = 1;
    while (t < x) t <<= 1;
    return t;
}

}  // namespace

struct NttPlan {
    bool crt = false;
    uint32_t na = 0, nb = 0, nout = 0, N = 0, L = 0, logL = 0, S = 1, threads = 0;
    uint32_t smem = 0, max_grid = 0;
    uint64_t scratch_stride = 0;
    size_t scratch_bytes = 0;
    uint64_t *dev = nullptr;      // tables followed by scratch
    uint64_t *scratch = nullptr;  // max_grid slots of scratch_stride words
    PrimeTab t1{}, t2{};
    uint64_t garner_inv = 0;
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
    NttPlan *p = new (std::nothrow) NttPlan();
    if (!p) return BN_ENOMEM;
    p->crt = crt;
    p->na = na;
    p->nb = nb;
    p->nout = na + nb;
    const uint32_t digits = crt ? na + nb : 2 * (na + nb);
    p->N = next_pow2(digits < 2 ? 2 : digits);
    p->S = p->N > kMaxSubLength ? p->N / kMaxSubLength : 1;
    p->L = p->N / p->S;
    while ((1u << p->logL) < p->L) ++p->logL;
    uint32_t T = p->L / 8;
    if (T < 32) T = 32;
    if (T > 1024) T = 1024;
    if (cta) T = cta;
    p->threads = T;
    const uint32_t Lp2 = (phys_words(p->L) + 1) & ~1u;
    p->smem = 8u * (2u * Lp2 + T) + 4u * 32u;

    cudaError_t e;
    auto *kern = crt ? k_mul_ntt<true> : k_mul_ntt<false>;
    e = allow_max_smem((const void *)kern);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)T, p->smem);
    if (e != cudaSuccess || per_sm == 0) {
        delete p;
        return e == cudaSuccess ? BN_EUNSUPPORTED : BN_ECUDA;
    }
    p->max_grid = (uint32_t)(sms * per_sm);
    p->scratch_stride = (p->S > 1 ? 2ull * p->N : 0ull) + (crt ? (uint64_t)p->N : 0ull);

    // Tables for each prime, then scratch, in one allocation.
    std::vector<HostTables> tabs;
    tabs.push_back(make_tables(field_p1(), p->N, p->S));
    if (crt) tabs.push_back(make_tables(field_p2(), p->N, p->S));
    size_t words = 0;
    for (auto &t : tabs) words += t.twf.size() + t.twi.size() + t.ffold.size() + t.ifold.size();
    const size_t table_words = (words + 31) & ~size_t(31);
    p->scratch_bytes = (size_t)p->max_grid * p->scratch_stride * 8u;
    e = cudaMalloc(&p->dev, table_words * 8u + p->scratch_bytes);
    if (e != cudaSuccess) {
        delete p;
        return e == cudaErrorMemoryAllocation ? BN_ENOMEM : BN_ECUDA;
    }
    std::vector<uint64_t> host(table_words, 0);
    size_t off = 0;
    for (size_t i = 0; i < tabs.size(); ++i) {
        HostTables &t = tabs[i];
        PrimeTab &pt = i == 0 ? p->t1 : p->t2;
        auto put = [&](const std::vector<uint64_t> &v) -> const uint64_t * {
            if (v.empty()) return nullptr;
            std::memcpy(host.data() + off, v.data(), v.size() * 8u);
            const uint64_t *d = p->dev + off;
            off += v.size();
            return d;
        };
        pt.twf = put(t.twf);
        pt.twi = put(t.twi);
        pt.ffold = put(t.ffold);
        pt.ifold = put(t.ifold);
        std::memcpy(pt.ws, t.ws, sizeof pt.ws);
        std::memcpy(pt.iws, t.iws, sizeof pt.iws);
        pt.scale = t.scale;
    }
    e = cudaMemcpy(p->dev, host.data(), table_words * 8u, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->dev);
        delete p;
        return BN_ECUDA;
    }
    p->scratch = p->dev + table_words;
    const HostField f1 = field_p1(), f2 = field_p2();
    p->garner_inv = to_form(f2, hinv(f1.p % f2.p, f2.p));
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
    args.scratch = p->scratch;
    args.scratch_stride = p->scratch_stride;
    args.garner_inv = p->garner_inv;
    args.t1 = p->t1;
    args.t2 = p->t2;
    return args;
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
    const uint64_t grid = batch < p->max_grid ? batch : p->max_grid;
    if (p->crt) k_mul_ntt<true><<<(unsigned)grid, p->threads, p->smem, st>>>(args);
    else k_mul_ntt<false><<<(unsigned)grid, p->threads, p->smem, st>>>(args);
    return cudaGetLastError();
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
    if (p->crt) k_mul_ntt<true><<<1, p->threads, p->smem, st>>>(args);
    else k_mul_ntt<false><<<1, p->threads, p->smem, st>>>(args);
    return cudaGetLastError();
}

bn_status ntt_batch_plan(NttPlan **out, bool crt, uint32_t N) {
    // A plan whose transform length is exactly N: digits(a) + digits(b) = N.
    if (N < 4 || (N & (N - 1))) return BN_EINVAL;
    const uint32_t per_side = crt ? N / 2 : N / 4;
    if (per_side > BN_MUL_MAX_LIMBS) return BN_EUNSUPPORTED;
    cudaError_t e = allow_max_smem((const void *)k_mul_ntt_batch<true>);
    if (e == cudaSuccess) e = allow_max_smem((const void *)k_mul_ntt_batch<false>);
    if (e != cudaSuccess) return BN_ECUDA;
    return ntt_create(out, crt, per_side, per_side, nullptr);
}

cudaError_t ntt_batch_launch(NttPlan *p, const BatchItem *items, uint32_t count, uint32_t *queue,
                             const BatchBinding *bind, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const NttArgs args = plan_args(p);
    const uint32_t grid = count < p->max_grid ? count : p->max_grid;
    if (p->crt) {
        if (cudaError_t e = allow_max_smem((const void *)k_mul_ntt_batch<true>)) return e;
        k_mul_ntt_batch<true><<<grid, p->threads, p->smem, st>>>(args, items, count, queue, bind);
    } else {
        if (cudaError_t e = allow_max_smem((const void *)k_mul_ntt_batch<false>)) return e;
        k_mul_ntt_batch<false><<<grid, p->threads, p->smem, st>>>(args, items, count, queue, bind);
    }
    return cudaGetLastError();
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
// halves, each prime holding twf + twi (2 L) and both folds (2 N) words.
constexpr size_t kNoAllocTableWords = 2 * (2 * 8192 + 2 * 16384);
static_assert(kNoAllocTableWords >= 2 * 8192 + 2 * 32768, "one prime at N = 32768 fits");

static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocScratchWords];
static __device__ __align__(256) uint64_t g_noalloc_tables[kNoAllocTableWords];

constexpr int kNoAllocMaxDevices = 64;
struct NoAllocDevice {
    bool ready = false;
    uint64_t *scratch = nullptr, *tables = nullptr;  // device addresses of the arrays
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

template <class F>
__device__ uint64_t form_pow(uint64_t base, uint64_t e, uint64_t one) {
    uint64_t r = one;
    while (e) {
        if (e & 1) r = F::mul(r, base);
        base = F::mul(base, base);
        e >>= 1;
    }
    return r;
}

// One prime's tables (layout twf[L] | twi[L] | ffold[S L] | ifold[S L]), the
// same values the plans build on the host; all inputs are in twiddle form.
template <class F>
__global__ void k_noalloc_tables(uint64_t *tab, uint32_t L, uint32_t S, uint64_t one, uint64_t wL,
                                 uint64_t wLi, uint64_t wN, uint64_t wNi, uint64_t scale) {
    const uint32_t total = 2 * L + (S > 1 ? 2 * S * L : 0);
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += gridDim.x * blockDim.x) {
        if (idx < 2 * L) {
            const uint32_t inv = idx >= L, i = idx - inv * L;
            uint64_t v = 0;
            if (i > 0) {
                const uint32_t h = 1u << (31 - __clz(i)), j = i - h;
                v = form_pow<F>(form_pow<F>(inv ? wLi : wL, L / (2 * h), one), j, one);
            }
            tab[idx] = F::canon(v);
        } else {
            const uint32_t k = idx - 2 * L, inv = k >= S * L, r = k - inv * S * L;
            const uint32_t sidx = r / L, j = r - sidx * L;
            const uint64_t w = form_pow<F>(inv ? wNi : wN, (uint64_t)j * sidx, one);
            tab[idx] = F::canon(inv ? F::mul(scale, w) : w);
        }
    }
}

// Host constants of one prime for (N, S), in twiddle form; no allocation.
struct NoAllocPrime {
    uint64_t one, wL, wLi, wN, wNi, scale;
    PrimeTab tab;
};

NoAllocPrime noalloc_prime(const HostField &f, uint32_t N, uint32_t S, uint64_t *dtab) {
    NoAllocPrime c{};
    const uint32_t L = N / S;
    const uint64_t wN = root_of_unity(f, N), wL = hpow(wN, S, f.p);
    const uint64_t R = f.montgomery ? (uint64_t)(((u128)1 << 64) % f.p) : 1;
    const uint64_t scale = hmul(hinv(N % f.p, f.p), R, f.p);
    c.one = to_form(f, 1);
    c.wL = to_form(f, wL);
    c.wLi = to_form(f, hinv(wL, f.p));
    c.wN = to_form(f, wN);
    c.wNi = to_form(f, hinv(wN, f.p));
    c.scale = to_form(f, scale);
    c.tab.twf = dtab;
    c.tab.twi = dtab + L;
    c.tab.ffold = S > 1 ? dtab + 2 * L : nullptr;
    c.tab.ifold = S > 1 ? dtab + 2 * L + (size_t)S * L : nullptr;
    c.tab.scale = c.scale;
    if (S > 1) {
        const uint64_t wS = hpow(wN, N / S, f.p), wSi = hinv(wS, f.p);
        for (uint32_t k = 0; k < S; ++k) {
            c.tab.ws[k] = to_form(f, hpow(wS, k, f.p));
            c.tab.iws[k] = to_form(f, hpow(wSi, k, f.p));
        }
    }
    return c;
}

size_t noalloc_prime_words(uint32_t N, uint32_t S) {
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
    auto *kern = crt ? k_mul_ntt<true> : k_mul_ntt<false>;

    // Geometry, as for a plan.
    const uint32_t digits = crt ? nout : 2 * nout;
    const uint32_t N = next_pow2(digits < 2 ? 2 : digits);
    const uint32_t S = N > kMaxSubLength ? N / kMaxSubLength : 1;
    const uint32_t L = N / S;
    uint32_t logL = 0;
    while ((1u << logL) < L) ++logL;
    uint32_t T = L / 8;
    if (T < 32) T = 32;
    if (T > 1024) T = 1024;
    const uint32_t Lp2 = (phys_words(L) + 1) & ~1u;
    const uint32_t smem = 8u * (2u * Lp2 + T) + 4u * 32u;
    const uint64_t stride = (S > 1 ? 2ull * N : 0ull) + (crt ? (uint64_t)N : 0ull);

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
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mul_ntt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mul_ntt<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) {
            record_error("bn_mul_ntt_noalloc device set-up failed");
            return BN_ECUDA;
        }
        d.scratch = static_cast<uint64_t *>(ps);
        d.tables = static_cast<uint64_t *>(pt);
        d.ready = true;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)T, smem);
    if (e != cudaSuccess || per_sm == 0) {
        record_error("bn_mul_ntt_noalloc: kernel does not fit on this device");
        return BN_ECUDA;
    }
    uint64_t max_grid = (uint64_t)d.sms * per_sm;
    if (stride > 0 && kNoAllocScratchWords / stride < max_grid) max_grid = kNoAllocScratchWords / stride;

    const NoAllocPrime c1 = noalloc_prime(field_p1(), N, S, d.tables);
    const NoAllocPrime c2 = noalloc_prime(field_p2(), N, S, d.tables + noalloc_prime_words(N, S));
    // A captured call records its own table kernel (replays regenerate the
    // tables they read) and leaves the host's record of the table contents
    // unusable for every later call.
    if (capturing) d.captured = true;
    if (capturing || d.captured || !d.have_tables || d.crt != crt || d.N != N) {
        const uint32_t words = (uint32_t)noalloc_prime_words(N, S);
        const unsigned blocks = (words + 255) / 256 < 1024 ? (words + 255) / 256 : 1024;
        k_noalloc_tables<FieldP1><<<blocks, 256, 0, st>>>(d.tables, L, S, c1.one, c1.wL, c1.wLi,
                                                           c1.wN, c1.wNi, c1.scale);
        if (crt)
            k_noalloc_tables<FieldP2><<<blocks, 256, 0, st>>>(d.tables + words, L, S, c2.one, c2.wL,
                                                               c2.wLi, c2.wN, c2.wNi, c2.scale);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            d.have_tables = false;
            record_error("bn_mul_ntt_noalloc table kernel launch failed");
            return BN_ECUDA;
        }
        d.have_tables = !d.captured;
        d.crt = crt;
        d.N = N;
    }

    NttArgs args{};
    args.a = a;
    args.b = b;
    args.c = c;
    args.na = na;
    args.nb = nb;
    args.nout = nout;
    args.N = N;
    args.L = L;
    args.logL = logL;
    args.S = S;
    args.digit_bits = crt ? 32 : 16;
    args.batch = batch;
    args.scratch = d.scratch;
    args.scratch_stride = stride;
    args.garner_inv = to_form(field_p2(), hinv(field_p1().p % field_p2().p, field_p2().p));
    args.t1 = c1.tab;
    args.t2 = c2.tab;
    const uint64_t grid = batch < max_grid ? batch : max_grid;
    if (crt) k_mul_ntt<true><<<(unsigned)grid, T, smem, st>>>(args);
    else k_mul_ntt<false><<<(unsigned)grid, T, smem, st>>>(args);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        record_error("bn_mul_ntt_noalloc kernel launch failed");
        return BN_ECUDA;
    }
    return BN_OK;
}
