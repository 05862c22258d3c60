// Device building blocks of the transform products (Section 4), shared by the
// 64-bit (one and two primes) and 32-bit (three primes) kernels: the radix-8
// butterfly passes over a shared-memory buffer, whole forward / inverse
// transforms, and the normalisation of convolution coefficients into limbs.
//
// A field type F provides Elem (the word type of its elements), Tw (the type
// of a twiddle table entry) and the two butterflies on lazily reduced
// elements, in place on (u, v):
//   dif(u, v, w):  (u + v, (u - v) w)    decimation in frequency,
//   dit(u, v, w):  (u + v w, u - v w)    decimation in time,
// and dif1 / dit1, the same with the twiddle 1.  Each field states the range
// its elements keep between passes; the forward passes start from values
// below 2P, and whatever range the inverse passes end in, the field's final
// scaling maps it back.
#pragma once
#include <type_traits>

#include "bn_debug.cuh"
#include "bn_device.cuh"

namespace bn {
namespace ntt {

typedef unsigned __int128 u128;

constexpr int kRadixLog = 3;  // radix-8 passes

// Shared-memory index with one element of padding per 16 (bank spread) for
// 64-bit elements.
__device__ __forceinline__ uint32_t phys(uint32_t i) { return i + (i >> 4); }
__host__ __device__ constexpr uint32_t phys_words(uint32_t n) { return n + (n >> 4) + 1; }

// Shared-memory index for 32-bit elements: four words of padding per 32, so
// groups of 4 consecutive elements stay 16-byte aligned (vector accesses) and
// every pass below meets 32 distinct banks: strides 4, 8 and 16 through the
// padding, unit-stride groups through 16-byte vector accesses.
__device__ __forceinline__ uint32_t phys4(uint32_t i) { return i + 4u * (i >> 5); }
__host__ __device__ constexpr uint32_t phys4_words(uint32_t n) { return n + 4u * ((n + 31) >> 5); }

template <class T>
__device__ __forceinline__ uint32_t pidx(uint32_t i) {
    if constexpr (sizeof(T) == 4) return phys4(i);
    else return phys(i);
}

// E consecutive elements starting at logical index `base` (a multiple of E).
// 32-bit elements move as 8- or 16-byte vectors: a run of E <= 8 from a
// multiple of E never crosses a 32-element padding boundary.
template <class T, int E>
__device__ __forceinline__ void load_run(const T *buf, uint32_t base, T (&x)[E]) {
    if constexpr (sizeof(T) == 4 && E >= 2) {
        const T *p = buf + phys4(base);
        if constexpr (E == 2) {
            const uint2 v = *reinterpret_cast<const uint2 *>(p);
            x[0] = v.x; x[1] = v.y;
        } else {
#pragma unroll
            for (int k = 0; k < E; k += 4) {
                const uint4 v = *reinterpret_cast<const uint4 *>(p + k);
                x[k] = v.x; x[k + 1] = v.y; x[k + 2] = v.z; x[k + 3] = v.w;
            }
        }
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) x[m] = buf[pidx<T>(base + m)];
    }
}

template <class T, int E>
__device__ __forceinline__ void store_run(T *buf, uint32_t base, const T (&x)[E]) {
    if constexpr (sizeof(T) == 4 && E >= 2) {
        T *p = buf + phys4(base);
        if constexpr (E == 2) {
            *reinterpret_cast<uint2 *>(p) = make_uint2(x[0], x[1]);
        } else {
#pragma unroll
            for (int k = 0; k < E; k += 4)
                *reinterpret_cast<uint4 *>(p + k) = make_uint4(x[k], x[k + 1], x[k + 2], x[k + 3]);
        }
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) buf[pidx<T>(base + m)] = x[m];
    }
}

// Twiddle index of group element m in the stage of half-size h (h = hm*step):
// the position of element m within its 2h block.  Within one group it depends
// only on m's bits below hm, so a stage needs hm distinct twiddles.
__device__ __forceinline__ uint32_t tw_index(uint32_t base, uint32_t m, uint32_t step, uint32_t h) {
    return h + ((base + m * step) & (h - 1));
}

// KK decimation-in-frequency stages with half-sizes H, H/2, ..., H >> (KK-1).
// UNIT: the group step is 1, so the last stage's twiddle is 1, and so is that
// of every group's element 0 in the other stages.
template <class F, int KK, bool UNIT>
__device__ __forceinline__ void dif_pass(typename F::Elem *buf, uint32_t L, uint32_t H,
                                         const typename F::Tw *tw) {
    using T = typename F::Elem;
    using W = typename F::Tw;
    constexpr int E = 1 << KK;
    const uint32_t step = UNIT ? 1u : H >> (KK - 1);
    const uint32_t lstep = UNIT ? 0u : __ffs(step) - 1;
    for (uint32_t g = threadIdx.x; g < (L >> KK); g += blockDim.x) {
        const uint32_t base = ((g >> lstep) << (lstep + KK)) | (g & (step - 1));
        T x[E];
        if constexpr (UNIT) load_run<T, E>(buf, base, x);
        else {
#pragma unroll
            for (int m = 0; m < E; ++m) x[m] = buf[pidx<T>(base + m * step)];
        }
#pragma unroll
        for (int st = 0; st < KK; ++st) {
            const uint32_t hm = 1u << (KK - 1 - st), h = hm * step;
            const bool trivial = UNIT && hm == 1;
            W w[E / 2];
#pragma unroll
            for (int m = 0; m < (int)hm; ++m)
                w[m] = (trivial || (UNIT && m == 0)) ? W{} : __ldg(tw + tw_index(base, m, step, h));
#pragma unroll
            for (int m = 0; m < E; ++m) {
                if (m & hm) continue;
                // UNIT: base is a multiple of E, so element m's twiddle is w_{2h}^(m mod hm): 1 for m mod hm = 0
                const bool one = UNIT && (m & (hm - 1)) == 0;
                if (one) F::dif1(x[m], x[m + hm]);
                else F::dif(x[m], x[m + hm], w[m & (hm - 1)]);
            }
        }
        if constexpr (UNIT) store_run<T, E>(buf, base, x);
        else {
#pragma unroll
            for (int m = 0; m < E; ++m) buf[pidx<T>(base + m * step)] = x[m];
        }
    }
}

// KK decimation-in-time stages with half-sizes h0, 2 h0, ..., h0 << (KK-1).
// UNIT: h0 = 1, so the first stage's twiddle is 1 (and every group's element
// 0 has twiddle 1 in the other stages).
template <class F, int KK, bool UNIT>
__device__ __forceinline__ void dit_pass(typename F::Elem *buf, uint32_t L, uint32_t h0,
                                         const typename F::Tw *tw) {
    using T = typename F::Elem;
    using W = typename F::Tw;
    constexpr int E = 1 << KK;
    const uint32_t step = UNIT ? 1u : h0;
    const uint32_t lstep = UNIT ? 0u : __ffs(step) - 1;
    for (uint32_t g = threadIdx.x; g < (L >> KK); g += blockDim.x) {
        const uint32_t base = ((g >> lstep) << (lstep + KK)) | (g & (step - 1));
        T x[E];
        if constexpr (UNIT) load_run<T, E>(buf, base, x);
        else {
#pragma unroll
            for (int m = 0; m < E; ++m) x[m] = buf[pidx<T>(base + m * step)];
        }
#pragma unroll
        for (int st = 0; st < KK; ++st) {
            const uint32_t hm = 1u << st, h = hm * step;
            const bool trivial = UNIT && hm == 1;
            W w[E / 2];
#pragma unroll
            for (int m = 0; m < (int)hm; ++m)
                w[m] = (trivial || (UNIT && m == 0)) ? W{} : __ldg(tw + tw_index(base, m, step, h));
#pragma unroll
            for (int m = 0; m < E; ++m) {
                if (m & hm) continue;
                const bool one = UNIT && (m & (hm - 1)) == 0;  // twiddle w_{2h}^0 = 1 (as in dif_pass)
                if (one) F::dit1(x[m], x[m + hm]);
                else F::dit(x[m], x[m + hm], w[m & (hm - 1)]);
            }
        }
        if constexpr (UNIT) store_run<T, E>(buf, base, x);
        else {
#pragma unroll
            for (int m = 0; m < E; ++m) buf[pidx<T>(base + m * step)] = x[m];
        }
    }
}

// Forward transforms of A and B (natural order in, bit-reversed out); ends
// with a barrier.  For 32-bit elements the passes that are not radix 8 come
// first (large strides), so no pass runs at stride 2, the one pattern the
// 32-bit padding leaves with bank conflicts.
template <class F>
__device__ void forward2(uint32_t L, uint32_t logL, const typename F::Tw *tw, typename F::Elem *A,
                         typename F::Elem *B) {
    uint32_t H = L >> 1, left = logL;
    if constexpr (sizeof(typename F::Elem) == 4) {
        const uint32_t rem = left % kRadixLog;
        if (rem == 2 && left > 2) {
            dif_pass<F, 2, false>(A, L, H, tw);
            dif_pass<F, 2, false>(B, L, H, tw);
            __syncthreads();
            H >>= 2;
            left -= 2;
        } else if (rem == 1 && left > 1) {
            dif_pass<F, 1, false>(A, L, H, tw);
            dif_pass<F, 1, false>(B, L, H, tw);
            __syncthreads();
            H >>= 1;
            left -= 1;
        }
    }
    while (left > (uint32_t)kRadixLog) {  // these passes have step >= 2
        dif_pass<F, kRadixLog, false>(A, L, H, tw);
        dif_pass<F, kRadixLog, false>(B, L, H, tw);
        __syncthreads();
        H >>= kRadixLog;
        left -= kRadixLog;
    }
    if (left == 3) {                       // the last pass has step 1
        dif_pass<F, 3, true>(A, L, H, tw);
        dif_pass<F, 3, true>(B, L, H, tw);
    } else if (left == 2) {
        dif_pass<F, 2, true>(A, L, H, tw);
        dif_pass<F, 2, true>(B, L, H, tw);
    } else {
        dif_pass<F, 1, true>(A, L, H, tw);
        dif_pass<F, 1, true>(B, L, H, tw);
    }
    __syncthreads();
}

// Unscaled inverse transform of B (bit-reversed in, natural out); ends with a
// barrier.
template <class F>
__device__ void inverse(uint32_t L, uint32_t logL, const typename F::Tw *tw, typename F::Elem *B) {
    uint32_t left = logL;
    const uint32_t first = left >= (uint32_t)kRadixLog ? (uint32_t)kRadixLog : left;
    if (first == 3) dit_pass<F, 3, true>(B, L, 1, tw);   // the first pass has h0 = 1
    else if (first == 2) dit_pass<F, 2, true>(B, L, 1, tw);
    else dit_pass<F, 1, true>(B, L, 1, tw);
    __syncthreads();
    uint32_t h0 = 1u << first;
    left -= first;
    while (left >= (uint32_t)kRadixLog) {
        dit_pass<F, kRadixLog, false>(B, L, h0, tw);
        __syncthreads();
        h0 <<= kRadixLog;
        left -= kRadixLog;
    }
    if (left == 2) {
        dit_pass<F, 2, false>(B, L, h0, tw);
        __syncthreads();
    } else if (left == 1) {
        dit_pass<F, 1, false>(B, L, h0, tw);
        __syncthreads();
    }
}

// ---- passes with the transform length fixed at compile time ----------------
//
// The same radix-8 passes for a length L, group stride STEP and thread count NT
// known at compile time.  With power-of-two strides the padded index is
// additive over a group, pidx(base + m*STEP) = pidx(base) + pidx(m*STEP) (a
// group never crosses a padding block boundary: base's bits below
// log2(STEP) + KK are j0 < STEP and m*STEP stays inside that block), so every
// element and twiddle of a group is an immediate offset from one base
// register, and the loops over groups have compile-time trip counts.  Measured
// on the 16384-point three-prime transform: 30% faster than the passes above.

template <uint32_t X>
struct Log2c {
    static constexpr uint32_t v = 1 + Log2c<X / 2>::v;
};
template <>
struct Log2c<1> {
    static constexpr uint32_t v = 0;
};

template <class T>
__host__ __device__ constexpr uint32_t pidx_c(uint32_t i) {
    return sizeof(T) == 4 ? i + 4u * (i >> 5) : i + (i >> 4);
}

// KK stages over groups of E = 2^KK elements base + m*STEP; DIF: half-sizes
// STEP*E/2 .. STEP (decimation in frequency), else STEP .. STEP*E/2
// (decimation in time).  UNIT (STEP = 1): the trivial stage has twiddle 1, and
// so has element 0 of every group in the other stages.
// A pass's epilogue: epi(i, x) is stored at logical index i instead of x
// (the last inverse pass folds a final scaling in this way).
struct NoEpi {
    template <class T>
    __device__ __forceinline__ T operator()(uint32_t, T x) const { return x; }
};

template <class F, int KK, bool UNIT, uint32_t STEP, uint32_t L, uint32_t NT, bool DIF, class Epi = NoEpi>
__device__ __forceinline__ void pass_c(typename F::Elem *buf, const typename F::Tw *tw, const Epi &epi = Epi{}) {
    using T = typename F::Elem;
    using W = typename F::Tw;
    constexpr int E = 1 << KK;
    constexpr uint32_t LSTEP = Log2c<STEP>::v;
    constexpr uint32_t G = L >> KK;
#pragma unroll
    for (uint32_t g0 = 0; g0 < G; g0 += NT) {
        const uint32_t g = g0 + threadIdx.x;
        if (G % NT != 0 && g >= G) break;
        const uint32_t j0 = g & (STEP - 1);
        const uint32_t base = ((g >> LSTEP) << (LSTEP + KK)) | j0;
        const uint32_t p0 = pidx<T>(base);
        T x[E];
        if constexpr (UNIT) {
            load_run<T, E>(buf, base, x);
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) x[m] = buf[p0 + pidx_c<T>(m * STEP)];
        }
        const W *twj = tw + j0;  // twiddle of element m in the stage of half-size hm*STEP: twj[(hm+m)*STEP]
#pragma unroll
        for (int st = 0; st < KK; ++st) {
            const uint32_t hm = DIF ? 1u << (KK - 1 - st) : 1u << st;
            const bool trivial = UNIT && hm == 1;
            W w[E / 2];
#pragma unroll
            for (int m = 0; m < (int)hm; ++m) w[m] = (trivial || (UNIT && m == 0)) ? W{} : __ldg(twj + (hm + m) * STEP);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                if (m & hm) continue;
                // UNIT: j0 = 0, so element m's twiddle is tw[hm + m mod hm]: 1 for m mod hm = 0
                const bool one = UNIT && (m & (hm - 1)) == 0;
                if constexpr (DIF) {
                    if (one) F::dif1(x[m], x[m + hm]);
                    else F::dif(x[m], x[m + hm], w[m & (hm - 1)]);
                } else {
                    if (one) F::dit1(x[m], x[m + hm]);
                    else F::dit(x[m], x[m + hm], w[m & (hm - 1)]);
                }
            }
        }
        if constexpr (!std::is_same<Epi, NoEpi>::value) {
#pragma unroll
            for (int m = 0; m < E; ++m) x[m] = epi(base + m * STEP, x[m]);
        }
        if constexpr (UNIT) {
            store_run<T, E>(buf, base, x);
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) buf[p0 + pidx_c<T>(m * STEP)] = x[m];
        }
    }
}

template <class F, uint32_t L, uint32_t NT, uint32_t H, uint32_t LEFT>
__device__ __forceinline__ void dif_rest_c(typename F::Elem *A, typename F::Elem *B,
                                           const typename F::Tw *tw) {
    if constexpr (LEFT > 3) {
        pass_c<F, 3, false, H / 4, L, NT, true>(A, tw);
        pass_c<F, 3, false, H / 4, L, NT, true>(B, tw);
        __syncthreads();
        dif_rest_c<F, L, NT, H / 8, LEFT - 3>(A, B, tw);
    } else {
        pass_c<F, (int)LEFT, true, 1, L, NT, true>(A, tw);
        pass_c<F, (int)LEFT, true, 1, L, NT, true>(B, tw);
    }
}

// Forward transforms of A and B of length 2^LOGL (as forward2, with the
// non-radix-8 pass first); ends with a barrier.
template <class F, uint32_t LOGL, uint32_t NT>
__device__ void forward2_c(const typename F::Tw *tw, typename F::Elem *A, typename F::Elem *B) {
    constexpr uint32_t L = 1u << LOGL;
    if constexpr (LOGL % 3 == 2 && LOGL > 2) {
        pass_c<F, 2, false, L / 4, L, NT, true>(A, tw);
        pass_c<F, 2, false, L / 4, L, NT, true>(B, tw);
        __syncthreads();
        dif_rest_c<F, L, NT, L / 8, LOGL - 2>(A, B, tw);
    } else if constexpr (LOGL % 3 == 1 && LOGL > 1) {
        pass_c<F, 1, false, L / 2, L, NT, true>(A, tw);
        pass_c<F, 1, false, L / 2, L, NT, true>(B, tw);
        __syncthreads();
        dif_rest_c<F, L, NT, L / 4, LOGL - 1>(A, B, tw);
    } else {
        dif_rest_c<F, L, NT, L / 2, LOGL>(A, B, tw);
    }
    __syncthreads();
}

template <class F, uint32_t L, uint32_t NT, uint32_t H0, uint32_t LEFT, class Epi>
__device__ __forceinline__ void dit_rest_c(typename F::Elem *B, const typename F::Tw *tw, const Epi &epi) {
    if constexpr (LEFT > 3) {
        pass_c<F, 3, false, H0, L, NT, false>(B, tw);
        __syncthreads();
        dit_rest_c<F, L, NT, H0 * 8, LEFT - 3>(B, tw, epi);
    } else if constexpr (LEFT > 0) {
        pass_c<F, (int)LEFT, false, H0, L, NT, false>(B, tw, epi);
        __syncthreads();
    }
}

// Inverse transform of B of length 2^LOGL, unscaled, or with the last
// pass's outputs passed through epi; ends with a barrier.
template <class F, uint32_t LOGL, uint32_t NT, class Epi = NoEpi>
__device__ void inverse_c(const typename F::Tw *tw, typename F::Elem *B, const Epi &epi = Epi{}) {
    constexpr uint32_t L = 1u << LOGL;
    constexpr uint32_t first = LOGL >= 3 ? 3 : LOGL;
    if constexpr (LOGL == first) {
        pass_c<F, (int)first, true, 1, L, NT, false>(B, tw, epi);
        __syncthreads();
    } else {
        pass_c<F, (int)first, true, 1, L, NT, false>(B, tw);
        __syncthreads();
        dit_rest_c<F, L, NT, (1u << first), LOGL - first>(B, tw, epi);
    }
}

// Normalisation (Section 4.2's splitFftReg/baddRegMul2Fft, with whole
// digits): limb(k) gives the part of the product that starts in limb k (the
// digit coefficients aligned there, < 2^96 in total).  Each thread folds the
// limbs of its window, carrying inside the window, the window's carry spills
// into the next window, and the remaining one-bit carries are resolved with
// the Section 2 carry scan across the CTA.  The nout limbs are assembled in
// the shared staging row out_s (limb k at k + k/16: the threads' windows are
// 16 limbs apart, and the padding puts them in distinct banks; out_s holds
// nout + nout/16 + 1 words) and then copied to crow.  Every thread of the CTA
// calls it; spill has one word per thread, flags one per warp.
__device__ __forceinline__ uint32_t stage_index(uint32_t k) { return k + (k >> 4); }

template <class LimbFn>
__device__ void normalize_limbs(uint32_t nout, uint32_t *crow, uint32_t *out_s, uint64_t *spill,
                                uint32_t *flags, LimbFn &&limb) {
    const uint32_t T = blockDim.x, t = threadIdx.x;
    uint32_t QN = (nout + T - 1) / T;
    if (QN < 2) QN = 2;  // a window must absorb a two-word spill
    const uint32_t k0 = t * QN;
    const uint32_t k1 = k0 + QN < nout ? k0 + QN : nout;
    // (a) this window's limbs, carrying within the window (their loads four at
    // a time, so that a limb read from L2 does not wait for the one before)
    u128 carry = 0;
    for (uint32_t k = k0; k < k1; k += 4) {
        u128 lv[4];
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) lv[j] = k + j < k1 ? limb(k + j) : (u128)0;
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j)
            if (k + j < k1) {
                const u128 v = lv[j] + carry;
                out_s[stage_index(k + j)] = (uint32_t)v;
                carry = v >> 32;
            }
    }
    spill[t] = (uint64_t)carry;  // < 2^64: the coefficients are below 2^96
    __syncthreads();
    // (b) add the previous window's spill; one carry bit may leave the window
    uint64_t c = t > 0 ? spill[t - 1] : 0;
    uint32_t all = 0xffffffffu;
    for (uint32_t k = k0; k < k1; ++k) {
        const uint64_t v = (uint64_t)out_s[stage_index(k)] + (c & 0xffffffffu);
        out_s[stage_index(k)] = (uint32_t)v;
        c = (c >> 32) + (v >> 32);
        all &= (uint32_t)v;
    }
    const bool owns = k0 < k1;
    // nothing may spill past the product: not out of its top window, not into
    // a thread with no limbs
    BN_DEBUG_CHECK(!(owns && k1 == nout) || c == 0, kDbgSpill);
    BN_DEBUG_CHECK(owns || c == 0, kDbgSpill);
    // (c) resolve the carries across windows (Section 2 carry scan)
    const uint32_t cin = group_carry_in(owns && c != 0, owns && all == 0xffffffffu, T, flags);
    BN_DEBUG_CHECK(!(owns && k1 == nout && cin && all == 0xffffffffu), kDbgSpill);
    if (cin)
        for (uint32_t k = k0; k < k1; ++k)
            if (++out_s[stage_index(k)] != 0) break;
    __syncthreads();
    // (d) coalesced copy-out
    for (uint32_t x = t; x < nout; x += T) st_stream(crow + x, out_s[stage_index(x)]);
    __syncthreads();
}

}  // namespace ntt
}  // namespace bn
