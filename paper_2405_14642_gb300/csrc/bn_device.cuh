// Device building blocks shared by the kernels: carry chains on u32 limbs and
// the carry-propagation scan of Section 2 at warp and block level.
//
// Carry scan (Section 2).  Each thread owns a contiguous chunk of limbs whose
// partial sum s = a + b is known.  The chunk "generates" a carry (g) if s
// overflowed and "propagates" one (p) if s is all ones; g and p exclude each
// other.  The carries entering the chunks are the exclusive scan of (g, p)
// under the paper's carry operator.  Within a warp this scan is one binary
// addition: with G = ballot(g) and P = ballot(p), the sum X + Y of X = G and
// Y = G | P carries out of lane l exactly when the operator says so (g: 1+1,
// p: 0+1, neither: 0+0), so the carries INTO the lanes are (X + Y + cin) ^ P
// and bit 32 of the 64-bit sum is the warp's carry-out.  Warps are chained
// through shared memory the same way (footnote on hierarchical scans).
#pragma once
#include <cstdint>

namespace bn {

constexpr unsigned FULL_MASK = 0xffffffffu;

// (g, p) of a whole row of 32 lanes: carry-out with carry-in 0, and whether a
// carry-in would pass through every lane.
struct RowFlags {
    uint32_t G, P;
};

// Carries into each lane (bit l) and the carry out of the row, for carry-in cin.
__device__ __forceinline__ uint32_t row_carries(RowFlags f, uint32_t cin, uint32_t &cout) {
    uint64_t s = (uint64_t)f.G + (uint64_t)(f.G | f.P) + cin;
    cout = (uint32_t)(s >> 32);
    return (uint32_t)s ^ f.P;
}

// Carry operator on (g, p) pairs: the prefix x followed by y.
__device__ __forceinline__ void carry_compose(uint32_t &g, uint32_t &p, uint32_t g2, uint32_t p2) {
    g = g2 | (p2 & g);
    p = p & p2;
}

// Bit l set at every lane l that ends a group of `group` lanes (group a power
// of two <= 32): the carry leaving such a lane must not enter the next group.
__device__ __forceinline__ uint32_t group_end_mask(uint32_t group) {
    uint32_t m = 0;
    for (uint32_t l = group - 1; l < 32; l += group) m |= 1u << l;
    return m;
}

// Exclusive carry scan over groups of `group` consecutive threads of the CTA,
// thread t of a group owning chunk t (in memory order).  Returns the carry
// into this thread's chunk.  `group` is a power of two <= 32 or a multiple of
// 32; for whole-warp groups the warps meet once in shared memory (`flags`:
// one word per warp of the CTA) and every thread of the CTA must call this.
__device__ __forceinline__ uint32_t group_carry_in(uint32_t g, uint32_t p, uint32_t group,
                                                   uint32_t *flags) {
    const uint32_t lane = threadIdx.x & 31;
    const RowFlags f{__ballot_sync(FULL_MASK, g), __ballot_sync(FULL_MASK, p)};
    if (group <= 32) {
        const uint32_t keep = ~group_end_mask(group);
        const uint64_t X = f.G & keep, Y = (f.G | f.P) & keep;
        return (((uint32_t)(X + Y) ^ (f.P & keep)) >> lane) & 1u;
    }
    const uint32_t warp = threadIdx.x >> 5, wpg = group >> 5;
    const uint32_t gi = warp / wpg, w = warp - gi * wpg;
    uint32_t wc;
    row_carries(f, 0, wc);
    if (lane == 0) flags[warp] = wc | ((f.P == FULL_MASK) << 1);
    __syncthreads();
    const uint32_t sw = lane < wpg ? flags[gi * wpg + lane] : 0u;
    const RowFlags fw{__ballot_sync(FULL_MASK, sw & 1u), __ballot_sync(FULL_MASK, (sw >> 1) & 1u)};
    uint32_t unused;
    const uint32_t wcin = (row_carries(fw, 0, unused) >> w) & 1u;
    return (row_carries(f, wcin, unused) >> lane) & 1u;
}

// ---- chunk arithmetic on VEC consecutive limbs --------------------------

// s = a + b over VEC limbs; returns the carry out.
template <int VEC>
__device__ __forceinline__ uint32_t chunk_add(const uint32_t (&a)[VEC], const uint32_t (&b)[VEC],
                                              uint32_t (&s)[VEC]);

template <>
__device__ __forceinline__ uint32_t chunk_add<1>(const uint32_t (&a)[1], const uint32_t (&b)[1],
                                                 uint32_t (&s)[1]) {
    uint32_t c;
    asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, 0, 0;" : "=r"(s[0]), "=r"(c) : "r"(a[0]), "r"(b[0]));
    return c;
}

template <>
__device__ __forceinline__ uint32_t chunk_add<4>(const uint32_t (&a)[4], const uint32_t (&b)[4],
                                                 uint32_t (&s)[4]) {
    uint32_t c;
    asm("add.cc.u32 %0, %5, %9;\n\t"
        "addc.cc.u32 %1, %6, %10;\n\t"
        "addc.cc.u32 %2, %7, %11;\n\t"
        "addc.cc.u32 %3, %8, %12;\n\t"
        "addc.u32 %4, 0, 0;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(c)
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]));
    return c;
}

// s += cin (cin in {0,1}) over VEC limbs.
template <int VEC>
__device__ __forceinline__ void chunk_inc(uint32_t (&s)[VEC], uint32_t cin);

template <>
__device__ __forceinline__ void chunk_inc<1>(uint32_t (&s)[1], uint32_t cin) {
    s[0] += cin;
}

template <>
__device__ __forceinline__ void chunk_inc<4>(uint32_t (&s)[4], uint32_t cin) {
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3])
        : "r"(cin));
}

template <int VEC>
__device__ __forceinline__ uint32_t chunk_all_ones(const uint32_t (&s)[VEC]) {
    uint32_t x = s[0];
#pragma unroll
    for (int k = 1; k < VEC; ++k) x &= s[k];
    return x == 0xffffffffu;
}

// ---- streaming global memory access -------------------------------------

__device__ __forceinline__ uint4 ld_stream_v4(const uint32_t *p) {
    return __ldcs(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(uint32_t *p, uint32_t v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream_v4(uint32_t *p, uint4 v) {
    __stcs(reinterpret_cast<uint4 *>(p), v);
}

}  // namespace bn
