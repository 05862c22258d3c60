// Device building blocks of the schoolbook product (Section 3), shared by the
// plain, batched and fused kernels: the shared-memory layout, the per-window
// multiply-accumulate chains and the window loop.  See mul_quad.cu for the
// partition they implement.
#pragma once
#include "bn_debug.cuh"
#include "bn_device.cuh"

namespace bn {
namespace quad {

constexpr uint32_t kQuadMaxThreads = 1024;

// Shared-memory word index for logical index x: a 16-byte pad after every 32
// words, which keeps 16-byte vector accesses at a stride of Q words free of
// bank conflicts.  x must be a multiple of 4 for vector accesses.
__device__ __forceinline__ uint32_t phys(uint32_t x) { return x + 4u * (x >> 5); }
__host__ __device__ constexpr uint32_t phys_size(uint32_t x) { return x + 4u * ((x + 31) >> 5); }

__host__ __device__ inline uint32_t roundup(uint32_t x, uint32_t m) { return (x + m - 1) / m * m; }

struct Geometry {
    uint32_t nap, nbp, units, group, ipb, inst_words, ab_words, l_offset, hc_offset, block, smem;
};

__host__ __device__ inline Geometry geometry(uint32_t na, uint32_t nb, uint32_t Q, uint32_t cta_target) {
    Geometry g{};
    g.nbp = roundup(nb, 2 * Q);
    g.nap = roundup(na, Q);
    if (g.nap < g.nbp) g.nap = g.nbp;
    g.units = g.nap / Q;
    if (g.units <= 32) {
        g.group = 1;
        while (g.group < g.units) g.group <<= 1;
    } else {
        g.group = roundup(g.units, 32);
    }
    g.ipb = g.group < cta_target ? cta_target / g.group : 1;
    // A at [0, phys_size(nap)), B (logical -Q .. nbp+Q) after it, then L
    // (nap + nbp words) and the H spill words (2 per window).
    const uint32_t a_words = roundup(phys_size(g.nap), 4);
    const uint32_t b_words = roundup(phys_size(g.nbp + 2 * Q), 4);
    const uint32_t l_words = roundup(phys_size(g.nap + g.nbp), 4);
    g.ab_words = a_words;
    g.l_offset = a_words + b_words;
    g.hc_offset = g.l_offset + l_words;
    const uint32_t windows = (g.nap + g.nbp) / Q;
    g.inst_words = roundup(g.hc_offset + 2 * windows, 4);
    g.block = g.group * g.ipb;
    g.smem = 4 * (g.inst_words * g.ipb + 32);
    return g;
}


// acc + cnt 2^{32Q} += a * (w[0] + w[1] 2^32 + ... + w[Q-1] 2^{32(Q-1)}): acc has Q+2
// words; the carry out of the low-half chain, which belongs at word Q, is
// counted in cnt instead of being carried through words Q and Q+1 (one
// instruction instead of two per chain); fold_count adds it in once per
// window.
template <int Q>
__device__ __forceinline__ void mac(uint32_t (&acc)[Q + 2], uint32_t &cnt, uint32_t a, const uint32_t (&w)[Q]);

template <>
__device__ __forceinline__ void mac<4>(uint32_t (&acc)[6], uint32_t &cnt, uint32_t a, const uint32_t (&w)[4]) {
    asm("mad.lo.cc.u32  %0, %7, %8,  %0;\n\t"
        "madc.lo.cc.u32 %1, %7, %9,  %1;\n\t"
        "madc.lo.cc.u32 %2, %7, %10, %2;\n\t"
        "madc.lo.cc.u32 %3, %7, %11, %3;\n\t"
        "addc.u32       %6, %6, 0;\n\t"
        "mad.hi.cc.u32  %1, %7, %8,  %1;\n\t"
        "madc.hi.cc.u32 %2, %7, %9,  %2;\n\t"
        "madc.hi.cc.u32 %3, %7, %10, %3;\n\t"
        "madc.hi.cc.u32 %4, %7, %11, %4;\n\t"
        "addc.u32       %5, %5, 0;"
        : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3]), "+r"(acc[4]), "+r"(acc[5]), "+r"(cnt)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]));
}

template <>
__device__ __forceinline__ void mac<8>(uint32_t (&acc)[10], uint32_t &cnt, uint32_t a, const uint32_t (&w)[8]) {
    asm("mad.lo.cc.u32  %0, %11, %12, %0;\n\t"
        "madc.lo.cc.u32 %1, %11, %13, %1;\n\t"
        "madc.lo.cc.u32 %2, %11, %14, %2;\n\t"
        "madc.lo.cc.u32 %3, %11, %15, %3;\n\t"
        "madc.lo.cc.u32 %4, %11, %16, %4;\n\t"
        "madc.lo.cc.u32 %5, %11, %17, %5;\n\t"
        "madc.lo.cc.u32 %6, %11, %18, %6;\n\t"
        "madc.lo.cc.u32 %7, %11, %19, %7;\n\t"
        "addc.u32       %10, %10, 0;\n\t"
        "mad.hi.cc.u32  %1, %11, %12, %1;\n\t"
        "madc.hi.cc.u32 %2, %11, %13, %2;\n\t"
        "madc.hi.cc.u32 %3, %11, %14, %3;\n\t"
        "madc.hi.cc.u32 %4, %11, %15, %4;\n\t"
        "madc.hi.cc.u32 %5, %11, %16, %5;\n\t"
        "madc.hi.cc.u32 %6, %11, %17, %6;\n\t"
        "madc.hi.cc.u32 %7, %11, %18, %7;\n\t"
        "madc.hi.cc.u32 %8, %11, %19, %8;\n\t"
        "addc.u32       %9, %9, 0;"
        : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3]), "+r"(acc[4]), "+r"(acc[5]),
          "+r"(acc[6]), "+r"(acc[7]), "+r"(acc[8]), "+r"(acc[9]), "+r"(cnt)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]),
          "r"(w[7]));
}

// acc += cnt 2^{32Q} (the low-chain carries counted by mac), then cnt = 0.
template <int Q>
__device__ __forceinline__ void fold_count(uint32_t (&acc)[Q + 2], uint32_t &cnt) {
    asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+r"(acc[Q]), "+r"(acc[Q + 1]) : "r"(cnt));
    cnt = 0;
}

// Partial carry chains for the triangular blocks of the lane form:
// x[0..M) += the low (lo_chain) or high (hi_chain) words of a * w[0..M), the
// chain's carry out added to c.  One asm statement per chain (the carry flag
// does not survive between statements).
template <int M>
__device__ __forceinline__ void lo_chain(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w);
template <int M>
__device__ __forceinline__ void hi_chain(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w);

template <>
__device__ __forceinline__ void lo_chain<1>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\t"
        "addc.u32 %1, %1, 0;"
        : "+r"(x[0]), "+r"(c)
        : "r"(a), "r"(w[0]));
}

template <>
__device__ __forceinline__ void lo_chain<2>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.lo.cc.u32 %1, %3, %5, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]));
}

template <>
__device__ __forceinline__ void lo_chain<3>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.lo.cc.u32 %0, %4, %5, %0;\n\t"
        "madc.lo.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]));
}

template <>
__device__ __forceinline__ void lo_chain<4>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.lo.cc.u32 %0, %5, %6, %0;\n\t"
        "madc.lo.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %8, %2;\n\t"
        "madc.lo.cc.u32 %3, %5, %9, %3;\n\t"
        "addc.u32 %4, %4, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]));
}

template <>
__device__ __forceinline__ void lo_chain<5>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.lo.cc.u32 %0, %6, %7, %0;\n\t"
        "madc.lo.cc.u32 %1, %6, %8, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %9, %2;\n\t"
        "madc.lo.cc.u32 %3, %6, %10, %3;\n\t"
        "madc.lo.cc.u32 %4, %6, %11, %4;\n\t"
        "addc.u32 %5, %5, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]));
}

template <>
__device__ __forceinline__ void lo_chain<6>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.lo.cc.u32 %0, %7, %8, %0;\n\t"
        "madc.lo.cc.u32 %1, %7, %9, %1;\n\t"
        "madc.lo.cc.u32 %2, %7, %10, %2;\n\t"
        "madc.lo.cc.u32 %3, %7, %11, %3;\n\t"
        "madc.lo.cc.u32 %4, %7, %12, %4;\n\t"
        "madc.lo.cc.u32 %5, %7, %13, %5;\n\t"
        "addc.u32 %6, %6, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]));
}

template <>
__device__ __forceinline__ void lo_chain<7>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.lo.cc.u32 %0, %8, %9, %0;\n\t"
        "madc.lo.cc.u32 %1, %8, %10, %1;\n\t"
        "madc.lo.cc.u32 %2, %8, %11, %2;\n\t"
        "madc.lo.cc.u32 %3, %8, %12, %3;\n\t"
        "madc.lo.cc.u32 %4, %8, %13, %4;\n\t"
        "madc.lo.cc.u32 %5, %8, %14, %5;\n\t"
        "madc.lo.cc.u32 %6, %8, %15, %6;\n\t"
        "addc.u32 %7, %7, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(x[6]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]));
}

template <>
__device__ __forceinline__ void lo_chain<8>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.lo.cc.u32 %0, %9, %10, %0;\n\t"
        "madc.lo.cc.u32 %1, %9, %11, %1;\n\t"
        "madc.lo.cc.u32 %2, %9, %12, %2;\n\t"
        "madc.lo.cc.u32 %3, %9, %13, %3;\n\t"
        "madc.lo.cc.u32 %4, %9, %14, %4;\n\t"
        "madc.lo.cc.u32 %5, %9, %15, %5;\n\t"
        "madc.lo.cc.u32 %6, %9, %16, %6;\n\t"
        "madc.lo.cc.u32 %7, %9, %17, %7;\n\t"
        "addc.u32 %8, %8, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(x[6]), "+r"(x[7]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]));
}

template <>
__device__ __forceinline__ void hi_chain<1>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.hi.cc.u32 %0, %2, %3, %0;\n\t"
        "addc.u32 %1, %1, 0;"
        : "+r"(x[0]), "+r"(c)
        : "r"(a), "r"(w[0]));
}

template <>
__device__ __forceinline__ void hi_chain<2>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.hi.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %5, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]));
}

template <>
__device__ __forceinline__ void hi_chain<3>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.hi.cc.u32 %0, %4, %5, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]));
}

template <>
__device__ __forceinline__ void hi_chain<4>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.hi.cc.u32 %0, %5, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %8, %2;\n\t"
        "madc.hi.cc.u32 %3, %5, %9, %3;\n\t"
        "addc.u32 %4, %4, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]));
}

template <>
__device__ __forceinline__ void hi_chain<5>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.hi.cc.u32 %0, %6, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %6, %8, %1;\n\t"
        "madc.hi.cc.u32 %2, %6, %9, %2;\n\t"
        "madc.hi.cc.u32 %3, %6, %10, %3;\n\t"
        "madc.hi.cc.u32 %4, %6, %11, %4;\n\t"
        "addc.u32 %5, %5, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]));
}

template <>
__device__ __forceinline__ void hi_chain<6>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.hi.cc.u32 %0, %7, %8, %0;\n\t"
        "madc.hi.cc.u32 %1, %7, %9, %1;\n\t"
        "madc.hi.cc.u32 %2, %7, %10, %2;\n\t"
        "madc.hi.cc.u32 %3, %7, %11, %3;\n\t"
        "madc.hi.cc.u32 %4, %7, %12, %4;\n\t"
        "madc.hi.cc.u32 %5, %7, %13, %5;\n\t"
        "addc.u32 %6, %6, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]));
}

template <>
__device__ __forceinline__ void hi_chain<7>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.hi.cc.u32 %0, %8, %9, %0;\n\t"
        "madc.hi.cc.u32 %1, %8, %10, %1;\n\t"
        "madc.hi.cc.u32 %2, %8, %11, %2;\n\t"
        "madc.hi.cc.u32 %3, %8, %12, %3;\n\t"
        "madc.hi.cc.u32 %4, %8, %13, %4;\n\t"
        "madc.hi.cc.u32 %5, %8, %14, %5;\n\t"
        "madc.hi.cc.u32 %6, %8, %15, %6;\n\t"
        "addc.u32 %7, %7, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(x[6]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]));
}

template <>
__device__ __forceinline__ void hi_chain<8>(uint32_t *x, uint32_t &c, uint32_t a, const uint32_t *w) {
    asm("mad.hi.cc.u32 %0, %9, %10, %0;\n\t"
        "madc.hi.cc.u32 %1, %9, %11, %1;\n\t"
        "madc.hi.cc.u32 %2, %9, %12, %2;\n\t"
        "madc.hi.cc.u32 %3, %9, %13, %3;\n\t"
        "madc.hi.cc.u32 %4, %9, %14, %4;\n\t"
        "madc.hi.cc.u32 %5, %9, %15, %5;\n\t"
        "madc.hi.cc.u32 %6, %9, %16, %6;\n\t"
        "madc.hi.cc.u32 %7, %9, %17, %7;\n\t"
        "addc.u32 %8, %8, 0;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(x[6]), "+r"(x[7]), "+r"(c)
        : "r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]));
}

// acc[1..8] += pend[1..8], the carry out into acc[9].
__device__ __forceinline__ void fold_pending8(uint32_t (&acc)[10], const uint32_t (&pend)[9]) {
    asm("add.cc.u32  %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.cc.u32 %2, %2, %11;\n\t"
        "addc.cc.u32 %3, %3, %12;\n\t"
        "addc.cc.u32 %4, %4, %13;\n\t"
        "addc.cc.u32 %5, %5, %14;\n\t"
        "addc.cc.u32 %6, %6, %15;\n\t"
        "addc.cc.u32 %7, %7, %16;\n\t"
        "addc.u32    %8, %8, 0;"
        : "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3]), "+r"(acc[4]), "+r"(acc[5]), "+r"(acc[6]),
          "+r"(acc[7]), "+r"(acc[8]), "+r"(acc[9])
        : "r"(pend[1]), "r"(pend[2]), "r"(pend[3]), "r"(pend[4]), "r"(pend[5]), "r"(pend[6]),
          "r"(pend[7]), "r"(pend[8]));
}

// Column form (Section 3.2's accumulate step): column q keeps a 64-bit sum
// and a carry count.  One mad.wide adds the full 64-bit product; the sum
// wrapped exactly when its high word decreased, since a product's high word
// is at most 2^32 - 2.
template <int Q>
__device__ __forceinline__ void mac_cols(uint64_t (&acc)[Q], uint32_t (&car)[Q], uint32_t a,
                                         const uint32_t (&w)[Q]) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint32_t old_hi = (uint32_t)(acc[q] >> 32);
        asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[q]) : "r"(a), "r"(w[q]));
        car[q] += (uint32_t)(acc[q] >> 32) < old_hi;
    }
}

// Window value sum_q (acc[q] + car[q] 2^64) 2^{32q} as Q+2 words.
template <int Q>
__device__ __forceinline__ void cols_to_words(const uint64_t (&acc)[Q], const uint32_t (&car)[Q],
                                              uint32_t (&out)[Q + 2]) {
    uint64_t c = 0;
#pragma unroll
    for (int q = 0; q < Q + 2; ++q) {
        uint64_t v = c;
        if (q < Q) v += (uint32_t)acc[q];
        if (q >= 1 && q <= Q) v += (uint32_t)(acc[q - 1] >> 32);
        if (q >= 2) v += car[q - 2];
        out[q] = (uint32_t)v;
        c = v >> 32;
    }
}

template <int Q>
__device__ __forceinline__ void ld_words(const uint32_t *S, uint32_t x, uint32_t (&v)[Q]) {
#pragma unroll
    for (int j = 0; j < Q / 4; ++j) {
        const uint4 t = *reinterpret_cast<const uint4 *>(S + phys(x + 4 * j));
        v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
    }
}

template <int Q>
__device__ __forceinline__ void st_words(uint32_t *S, uint32_t x, const uint32_t *v) {
#pragma unroll
    for (int j = 0; j < Q / 4; ++j)
        *reinterpret_cast<uint4 *>(S + phys(x + 4 * j)) =
            make_uint4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}

// Q steps i = i0 .. i0+Q-1 of a window: the B window for step s is
// B[k-i0-s .. k-i0-s+Q), taken from the chunk pair (lo, hi) = B[k-i0-Q .. k-i0+Q).
template <int Q, bool COLS>
__device__ __forceinline__ void window_block(const uint32_t *As, uint32_t i0, const uint32_t (&lo)[Q],
                                             const uint32_t (&hi)[Q], uint32_t (&acc)[Q + 2], uint32_t &cnt,
                                             uint64_t (&cacc)[Q], uint32_t (&ccar)[Q]) {
    uint32_t av[4];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        if (s % 4 == 0) ld_words<4>(As, i0 + s, av);  // A four words at a time
        uint32_t w[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int idx = Q - s + q;
            w[q] = idx < Q ? lo[idx] : hi[idx - Q];
        }
        if constexpr (COLS) mac_cols<Q>(cacc, ccar, av[s % 4], w);
        else mac<Q>(acc, cnt, av[s % 4], w);
    }
}

// Window starting at column k: sum over i in [ilo, ilo + steps) of
// A_i * B[k-i .. k-i+Q).  B's logical index x lives at phys(x + Q).
// ilo, k and steps are multiples of Q.  Blocks alternate between two chunk
// buffers, so the chunk that moves from "lower" to "upper" is never copied.
template <int Q, bool COLS>
__device__ __forceinline__ void conv_window(const uint32_t *As, const uint32_t *Bs, uint32_t k,
                                            uint32_t ilo, uint32_t steps, uint32_t (&acc)[Q + 2]) {
    uint64_t cacc[Q];
    uint32_t ccar[Q];
    uint32_t cnt = 0;
#pragma unroll
    for (int q = 0; q < Q + 2; ++q) acc[q] = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        cacc[q] = 0;
        ccar[q] = 0;
    }
    // xb = (k - i0) + Q: the offset-Q index of the current block's upper chunk.
    uint32_t xb = k - ilo + Q, i0 = ilo;
    const uint32_t nblk = steps / Q;
    uint32_t c0[Q], c1[Q];
    ld_words<Q>(Bs, xb, c1);
    for (uint32_t b = 0; b + 1 < nblk; b += 2) {
        ld_words<Q>(Bs, xb - Q, c0);
        window_block<Q, COLS>(As, i0, c0, c1, acc, cnt, cacc, ccar);
        ld_words<Q>(Bs, xb - 2 * Q, c1);
        window_block<Q, COLS>(As, i0 + Q, c1, c0, acc, cnt, cacc, ccar);
        xb -= 2 * Q;
        i0 += 2 * Q;
    }
    if (nblk & 1) {
        ld_words<Q>(Bs, xb - Q, c0);
        window_block<Q, COLS>(As, i0, c0, c1, acc, cnt, cacc, ccar);
    }
    if constexpr (COLS) cols_to_words<Q>(cacc, ccar, acc);
    else fold_count<Q>(acc, cnt);
}

// A unit of work: up to two windows run back to back as ONE loop of n0 + n1
// blocks.  Window w starts at column k_w with first step ilo_w and takes n_w
// blocks (n1 = 0: one window).  Every unit of the partition has the same
// total (R + 1 blocks), so the lanes of a warp share one trip count whatever
// their windows; only the hand-over between the windows diverges.  Each
// finished window goes to publish(k, acc).
struct Unit {
    uint32_t k0, ilo0, n0, k1, ilo1, n1;
};

template <int Q, class Publish>
__device__ __forceinline__ void conv_unit(const uint32_t *As, const uint32_t *Bs, const Unit &u,
                                          Publish &&publish) {
    uint32_t acc[Q + 2];
    uint32_t cnt = 0;
    uint64_t cacc[Q];  // unused by the chain form
    uint32_t ccar[Q];
#pragma unroll
    for (int q = 0; q < Q + 2; ++q) acc[q] = 0;
    uint32_t k = u.k0, i0 = u.ilo0, left = u.n0, second = u.n1;
    const uint32_t total = u.n0 + u.n1;
    uint32_t c0[Q], c1[Q];
    ld_words<Q>(Bs, k - i0 + Q, c1);  // upper chunk of the first block
    // After a window's last block: publish it and start the next one, whose
    // upper chunk goes to the buffer the next block reads as "upper".
    auto finish = [&](uint32_t (&next_hi)[Q]) {
        fold_count<Q>(acc, cnt);
        publish(k, acc);
#pragma unroll
        for (int q = 0; q < Q + 2; ++q) acc[q] = 0;
        if (second) {
            k = u.k1;
            i0 = u.ilo1;
            left = second;
            second = 0;
            ld_words<Q>(Bs, k - i0 + Q, next_hi);
        }
    };
    for (uint32_t b = 0; b < total; b += 2) {
        ld_words<Q>(Bs, k - i0, c0);
        window_block<Q, false>(As, i0, c0, c1, acc, cnt, cacc, ccar);
        i0 += Q;
        if (--left == 0) finish(c0);
        if (b + 1 == total) break;
        ld_words<Q>(Bs, k - i0, c1);
        window_block<Q, false>(As, i0, c1, c0, acc, cnt, cacc, ccar);
        i0 += Q;
        if (--left == 0) finish(c1);
    }
}

// Copies n words of a global row into shared memory at logical offset `off`
// (layout phys), zero-filling logical [off + n, off + n_pad).
__device__ __forceinline__ void stage_row(uint32_t *S, const uint32_t *row, uint32_t n,
                                          uint32_t off, uint32_t n_pad, bool vec, bool live,
                                          uint32_t t, uint32_t group) {
    if (vec && live) {
        for (uint32_t x = 4 * t; x < n; x += 4 * group) {
            const uint4 v = ld_stream_v4(row + x);
            *reinterpret_cast<uint4 *>(S + phys(off + x)) = v;
        }
        for (uint32_t x = n + t; x < n_pad; x += group) S[phys(off + x)] = 0;
    } else {
        for (uint32_t x = t; x < n_pad; x += group)
            S[phys(off + x)] = (live && x < n) ? ld_stream(row + x) : 0u;
    }
}


}  // namespace quad
}  // namespace bn
