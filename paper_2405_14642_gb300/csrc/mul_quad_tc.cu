// Schoolbook product on the tensor cores (BN_OP_MUL_QUAD_TC).
//
// The product of Section 3 sums every word product A_i B_j into column i + j
// (Eq. 1).  This kernel computes the same column sums one level down, on
// bytes, as an exact contraction on the fifth-generation tensor cores: a byte
// is an exact fp16 integer, a byte product is below 2^16, and 128 of them sum
// below 2^23, where f32 arithmetic is exact whatever the order of the sums.
//
// Cut both operands into blocks of 128 bytes (a: blocks I < ma, b: J < mb) and
// let W_J be the 128 x 128 Toeplitz matrix W_J[r][c] = b-byte (128 J + r - c)
// (zero outside b).  Byte column 128 s + r of the product is then
//     sum_J  sum_c  W_J[r][c] * a-byte (128 (s - J) + c),
// so for each J the contribution to the output blocks s is D_J = W_J X^T,
// where row I of X is block I of a: one MMA chain with M = 128 (r), K = 128
// (c) and N = the output blocks s with 0 <= s - J < ma.  D_J is read from
// tensor memory, turned into integers and added into per-thread integer
// column sums (below 2^31: no rounding anywhere); the column sums are folded
// into limbs by the transform products' normalisation (carry scan included).
//
// Per CTA and instance: X is staged once in shared memory as fp16 in the
// tensor core's core-matrix layout (the longer operand, with 32 zero blocks on
// each side); b stays as raw bytes.  The output is processed in tiles of 128
// blocks, each tile in steps J.  Three roles run as a pipeline linked by
// mbarriers: four warps build W_J (one row per thread) into one of four W
// slots in tensor memory, one thread issues the step's 8 MMAs of K = 16 into
// one of two D slots and commits them, and eight warps (two per group of 32
// lanes) add each finished D into their integer column sums and publish them
// at the end of the tile.
#include <cuda_runtime.h>

#include <new>

#include "bn_internal.h"
#include "ntt_device.cuh"
#include "tc_device.cuh"

namespace bn {

__device__ uint32_t g_tc_fault;  // set when an MMA wait timed out

namespace {

constexpr uint32_t kThreads = 640;   // warp 0 issues the MMAs, 1-3 build W, 4-19 read D
constexpr uint32_t kBuilders = 3, kEpiWarps = 16;
constexpr uint32_t kBlk = 128;       // bytes per block: rows of W, K of a step
constexpr uint32_t kTile = 256;      // output blocks per tile (D columns, the MMA's N)
constexpr uint32_t kPad = 32;        // zero blocks on each side of X
constexpr uint32_t kTmemCols = 512;  // two D slots of 256 columns
constexpr uint32_t kDSlots = 2;      // D slots in tensor memory (256 columns each)
constexpr uint32_t kWSlots = 3;      // W slots in shared memory
constexpr uint32_t kWBytes = 128 * 128 * 2;  // one W_J in fp16: 16 K-chunks x 16 row groups x 128 B
constexpr uint32_t kWLbo = 2048, kWSbo = 128;  // W: K-chunk stride, 8-row-group stride
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s per wait
constexpr uint32_t kMinSmem = 116 * 1024;     // one CTA per SM (the whole tensor memory each)

struct TcArgs {
    const uint32_t *a, *b;  // na >= nb (the host orders the operands)
    uint32_t *c;
    uint32_t na, nb, nout, ma, mb, tiles;
    uint64_t batch;
    uint32_t *scratch;        // per CTA: 128 (ma + mb) byte-column sums
    uint64_t scratch_stride;  // words per CTA
    uint32_t xs;              // bytes per chunk row of X: (ma + 2 kPad) * 16
    uint32_t w_off, braw_off, spill_off, flags_off, bar_off;  // shared-memory byte offsets
};

__device__ __forceinline__ int jlo(const TcArgs &g, int t) {
    const int v = (int)(kTile * t) - (int)g.ma + 1;
    return v > 0 ? v : 0;
}
__device__ __forceinline__ int jhi(const TcArgs &g, int t) {
    const int v = (int)(kTile * t + kTile - 1);
    return v < (int)g.mb ? v : (int)g.mb;
}

// D chunks (32 columns each) of tile t that step J writes: the columns s with
// 0 <= s - J < ma, rounded out to whole chunks (X's zero blocks cover the rest).
__device__ __forceinline__ void chunk_range(const TcArgs &g, int t, int J, int &clo, int &chi) {
    const int s0 = (int)(kTile * t);
    const int lo = (J > s0 ? J : s0) - s0;
    const int e = J + (int)g.ma, hi = (e < s0 + (int)kTile ? e : s0 + (int)kTile) - s0;
    clo = lo >> 5;
    chi = (hi + 31) >> 5;
}

__device__ __forceinline__ bool step_next(const TcArgs &g, int &t, int &J) {
    if (J < jhi(g, t)) {
        ++J;
        return true;
    }
    if (t + 1 < (int)g.tiles) {
        ++t;
        J = jlo(g, t);
        return true;
    }
    return false;
}

// Row r of W_J, words 32 h .. 32 h + 31, into the W slot at
// `w` (shared memory, the MMA's A operand: K-major without swizzle, the 16-byte
// piece of row r and K-chunk q at (r / 8) * 128 + q * 2048 + (r % 8) * 16).
// Word k of row r holds the fp16 pair (W_J[r][2k], W_J[r][2k+1]) =
// (b-byte (v - 2k), b-byte (v - 2k - 1)), v = 128 J + r; braw holds b's bytes
// at offset 128 + index, zero outside b.
__device__ __forceinline__ void build_w(const uint32_t *braw, int J, uint32_t r, uint32_t h, uint8_t *w) {
    const int e = 65 + 128 * J + (int)r - 64 * (int)h;  // lowest byte offset this thread reads
    const uint32_t *bw = braw + (e >> 2);
    const uint32_t sh = (uint32_t)e & 3u;
    uint32_t wv[17];
#pragma unroll
    for (int j = 0; j < 17; ++j) wv[j] = bw[j];
    // bytes at offsets e + 63 - 4g, e + 62 - 4g, e + 61 - 4g, e + 60 - 4g
    const uint32_t sel = (sh + 3) | ((sh + 2) << 4) | ((sh + 1) << 8) | (sh << 12);
    uint8_t *row = w + (r >> 3) * kWSbo + (r & 7) * 16 + 8 * h * kWLbo;
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // K-chunk 8 h + q: words 4 q .. 4 q + 3 of this half
        const uint32_t r0 = __byte_perm(wv[15 - 2 * q], wv[16 - 2 * q], sel);
        const uint32_t r1 = __byte_perm(wv[14 - 2 * q], wv[15 - 2 * q], sel);
        *reinterpret_cast<uint4 *>(row + q * kWLbo) =
            make_uint4(tc::bytes01_f16x2(r0), tc::bytes23_f16x2(r0), tc::bytes01_f16x2(r1), tc::bytes23_f16x2(r1));
    }
}

// Exact integer of an f32 holding an integer v in [0, 2^23): v + 2^23 has
// exponent 23, so its mantissa bits are v.
__device__ __forceinline__ uint32_t f32_int(uint32_t bits) {
    return __float_as_uint(__fadd_rn(__uint_as_float(bits), 8388608.0f)) - 0x4b000000u;
}

__global__ void __launch_bounds__(kThreads, 1) k_mul_quad_tc(TcArgs g) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *X = sm;  // X and the W slots double as the normalisation's staging row
    uint8_t *W = sm + g.w_off;
    uint32_t *braw = reinterpret_cast<uint32_t *>(sm + g.braw_off);
    uint64_t *spill = reinterpret_cast<uint64_t *>(sm + g.spill_off);
    uint32_t *flags = reinterpret_cast<uint32_t *>(sm + g.flags_off);
    uint64_t *wfull = reinterpret_cast<uint64_t *>(sm + g.bar_off);  // [kWSlots], builder arrivals
    uint64_t *wempty = wfull + kWSlots;                                 // [kWSlots], MMA commits
    uint64_t *dfull = wempty + kWSlots;                                 // [kDSlots], MMA commits
    uint64_t *dempty = dfull + kDSlots;                                 // [kDSlots], epilogue arrivals
    uint32_t *slot = reinterpret_cast<uint32_t *>(dempty + kDSlots);
    volatile uint32_t *abortf = slot + 1;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lq = warp & 3;  // the tensor-memory lanes this warp may move
    if (warp == 0) tc::tmem_alloc(slot, kTmemCols);
    if (tid == 0) {
        for (uint32_t k = 0; k < kWSlots; ++k) {
            tc::mbar_init(&wfull[k], 32 * kBuilders);
            tc::mbar_init(&wempty[k], 1);
        }
        for (uint32_t k = 0; k < kDSlots; ++k) {
            tc::mbar_init(&dfull[k], 1);
            tc::mbar_init(&dempty[k], 32 * kEpiWarps);
        }
        *abortf = 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot;
    const uint32_t lane_off = (32 * lq) << 16;
    const uint32_t x_s = tc::smem_u32(X), w_s = tc::smem_u32(W);
    const uint32_t out_blocks = g.ma + g.mb;
    uint32_t *cols = g.scratch + blockIdx.x * g.scratch_stride;
    uint32_t gs = 0;  // this thread's step count over all instances (slots and phases)
    bool fail = false;

    for (uint64_t inst = blockIdx.x; inst < g.batch; inst += gridDim.x) {
        const uint32_t *arow = g.a + inst * g.na, *brow = g.b + inst * g.nb;
        // ---- stage X (fp16, core-matrix layout) and b's bytes
        for (uint32_t x = tid; x < 16 * g.ma; x += kThreads) {
            const uint32_t I = x >> 4, q = x & 15, w0 = 32 * I + 2 * q;
            const uint32_t u = w0 < g.na ? __ldg(arow + w0) : 0u;
            const uint32_t v = w0 + 1 < g.na ? __ldg(arow + w0 + 1) : 0u;
            const uint4 f = make_uint4(tc::bytes01_f16x2(u), tc::bytes23_f16x2(u), tc::bytes01_f16x2(v),
                                       tc::bytes23_f16x2(v));
            *reinterpret_cast<uint4 *>(X + q * g.xs + (I + kPad) * 16) = f;
        }
        for (uint32_t x = tid; x < 16 * 2 * kPad; x += kThreads) {
            const uint32_t q = x / (2 * kPad), p = x % (2 * kPad);
            const uint32_t I = p < kPad ? p : g.ma + p;  // padded index (kPad offset included)
            *reinterpret_cast<uint4 *>(X + q * g.xs + I * 16) = make_uint4(0, 0, 0, 0);
        }
        const uint32_t bwords = 32 * (g.mb + 2) + 4;
        for (uint32_t x = tid; x < bwords; x += kThreads)
            braw[x] = (x >= 32 && x - 32 < g.nb) ? __ldg(brow + x - 32) : 0u;
        tc::fence_proxy_async();
        __syncthreads();

        // ---- the steps (tile, J), one role per warp group
        int t = 0, J = jlo(g, 0);
        if (warp == 0) {
            // one thread issues each step's 8 MMAs (K = 16 each) and commits them
            do {
                const uint32_t k = gs % kWSlots, d = gs % kDSlots, ud = gs / kDSlots;
                if (lane == 0) {
                    bool ok = tc::mbar_wait(&wfull[k], (gs / kWSlots) & 1u, kWaitNs, abortf);
                    if (ok && ud > 0) ok = tc::mbar_wait(&dempty[d], (ud - 1) & 1u, kWaitNs, abortf);
                    if (ok) {
                        tc::fence_after_sync();
                        int clo, chi;
                        chunk_range(g, t, J, clo, chi);
                        const uint32_t idesc = tc::idesc_f16_f32(128, 32u * (uint32_t)(chi - clo));
                        const int i0 = (int)(kTile * t) + 32 * clo - J + (int)kPad;  // padded block of column 0
                        const uint32_t dt = tbase + kTile * d + 32 * (uint32_t)clo;
                        const uint32_t ws = w_s + k * kWBytes;
#pragma unroll
                        for (uint32_t kk = 0; kk < 8; ++kk) {
                            const uint64_t bd = tc::smem_desc(x_s + 2 * kk * g.xs + (uint32_t)i0 * 16, g.xs, 128);
                            const uint64_t ad = tc::smem_desc(ws + 2 * kk * kWLbo, kWLbo, kWSbo);
                            tc::mma_f16_ss(dt, ad, bd, idesc, kk > 0);
                        }
                        tc::mma_commit(&dfull[d]);
                        tc::mma_commit(&wempty[k]);
                    } else {
                        *abortf = 1;
                    }
                }
                ++gs;
                if (__shfl_sync(FULL_MASK, (uint32_t)*abortf, 0)) break;
            } while (step_next(g, t, J));
        } else if (warp <= kBuilders) {
            // builders: W_J into a W slot once the MMA that last read it is done;
            // the 256 pieces (row, half) are spread over the 96 builder threads
            const uint32_t bt = tid - 32;
            do {
                const uint32_t k = gs % kWSlots, use = gs / kWSlots;
                if (use > 0 &&
                    !__all_sync(FULL_MASK, tc::mbar_wait(&wempty[k], (use - 1) & 1u, kWaitNs, abortf))) {
                    *abortf = 1;
                    break;
                }
                uint8_t *wk = W + k * kWBytes;
                for (uint32_t i = bt; i < 256; i += 32 * kBuilders) build_w(braw, J, i & 127, i >> 7, wk);
                tc::fence_proxy_async();
                tc::mbar_arrive(&wfull[k]);
                ++gs;
            } while (step_next(g, t, J));
        } else {
            // epilogue: D of each step into the integer column sums of the tile
            // (the 4 warps of lane group lq own chunks 2m, 2m + 1, m = 0..3)
            const uint32_t m = (warp - 1 - kBuilders) >> 2;  // warps 4..19: m = 0..3
            uint32_t acc[2][32];
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int i = 0; i < 32; ++i) acc[c][i] = 0;
            do {
                const uint32_t d = gs % kDSlots;
                if (!__all_sync(FULL_MASK, tc::mbar_wait(&dfull[d], (gs / kDSlots) & 1u, kWaitNs, abortf))) {
                    *abortf = 1;
                    break;
                }
                tc::fence_after_sync();
                int clo, chi;
                chunk_range(g, t, J, clo, chi);
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int ch = 2 * (int)m + c;
                    if (ch >= clo && ch < chi) {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            uint32_t v[16];
                            tc::tmem_ld16(tbase + lane_off + kTile * d + 32 * (uint32_t)ch + 16 * hh, v);
#pragma unroll
                            for (int i = 0; i < 16; ++i) acc[c][16 * hh + i] += f32_int(v[i]);
                        }
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&dempty[d]);
                ++gs;
                if (J == jhi(g, t)) {  // tile complete: publish its column sums
                    const uint32_t s0 = kTile * (uint32_t)t, r = 32 * lq + lane;
#pragma unroll
                    for (int c = 0; c < 2; ++c)
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const uint32_t s = s0 + 32 * (2 * m + c) + i;
                            if (s < out_blocks) cols[kBlk * s + r] = acc[c][i];
                            acc[c][i] = 0;
                        }
                }
            } while (step_next(g, t, J));
        }
        __syncthreads();
        fail = *abortf != 0;
        if (fail) break;
        // ---- column sums -> limbs (Section 2 carry scan inside)
        ntt::normalize_limbs(g.nout, g.c + inst * g.nout, reinterpret_cast<uint32_t *>(X), spill, flags,
                             [&](uint32_t k) {
                                 const uint4 q = *reinterpret_cast<const uint4 *>(cols + 4 * k);
                                 return (ntt::u128)((uint64_t)q.x + ((uint64_t)q.y << 8) +
                                                    ((uint64_t)q.z << 16) + ((uint64_t)q.w << 24));
                             });
    }
    if (fail && tid == 0) {
        // wind down: give the MMAs issued last a bounded time to finish
        if (gs > 0) {
            const uint32_t last = gs - 1;
            tc::mbar_wait(&dfull[last % kDSlots], (last / kDSlots) & 1u, kWaitNs);
        }
        atomicOr(&g_tc_fault, 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

struct TcGeometry {
    uint32_t na, nb, ma, mb, tiles, xs, w_off, braw_off, spill_off, flags_off, bar_off, smem;
    bool swap;
};

TcGeometry geometry(uint32_t na, uint32_t nb) {
    TcGeometry q{};
    q.swap = na < nb;
    q.na = q.swap ? nb : na;
    q.nb = q.swap ? na : nb;
    q.ma = (q.na + 31) / 32;
    q.mb = (q.nb + 31) / 32;
    q.tiles = (q.ma + q.mb + kTile - 1) / kTile;
    q.xs = (q.ma + 2 * kPad) * 16;
    const uint32_t nout = q.na + q.nb;
    const uint32_t stage_bytes = 4 * ((nout - 1) + ((nout - 1) >> 4) + 1);
    q.w_off = 16 * q.xs;  // a multiple of 16
    uint32_t off = q.w_off + kWSlots * kWBytes;
    if (off < stage_bytes) off = stage_bytes;
    off = (off + 15) & ~15u;
    q.braw_off = off;
    off += 4 * (32 * (q.mb + 2) + 4);
    off = (off + 15) & ~15u;
    q.spill_off = off;
    off += 8 * kThreads;
    q.flags_off = off;
    off += 4 * (kThreads / 32);
    q.bar_off = (off + 15) & ~15u;
    off = q.bar_off + 8 * (2 * kWSlots + 2 * kDSlots) + 8;
    q.smem = off > kMinSmem ? off : kMinSmem;
    return q;
}

}  // namespace

struct QuadTcPlan {
    TcGeometry geo;
    uint32_t nout = 0, ctas = 0;
    uint32_t *scratch = nullptr;
    uint64_t stride = 0;
};

bn_status quad_tc_create(QuadTcPlan **out, uint32_t na, uint32_t nb) {
    *out = nullptr;
    if (na == 0 || nb == 0) return BN_EINVAL;
    if (na > BN_MUL_MAX_LIMBS || nb > BN_MUL_MAX_LIMBS) return BN_EUNSUPPORTED;
    QuadTcPlan *p = new (std::nothrow) QuadTcPlan();
    if (!p) return BN_ENOMEM;
    p->geo = geometry(na, nb);
    p->nout = na + nb;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = allow_max_smem((const void *)k_mul_quad_tc);
    if (e != cudaSuccess) {
        delete p;
        return BN_ECUDA;
    }
    p->ctas = (uint32_t)sms;
    p->stride = (uint64_t)kBlk * (p->geo.ma + p->geo.mb);
    e = cudaMalloc(&p->scratch, p->stride * 4ull * p->ctas);
    if (e != cudaSuccess) {
        delete p;
        return e == cudaErrorMemoryAllocation ? BN_ENOMEM : BN_ECUDA;
    }
    *out = p;
    return BN_OK;
}

void quad_tc_destroy(QuadTcPlan *p) {
    if (!p) return;
    cudaFree(p->scratch);
    delete p;
}

size_t quad_tc_scratch_bytes(const QuadTcPlan *p) { return p ? p->stride * 4ull * p->ctas : 0; }

cudaError_t quad_tc_launch(QuadTcPlan *p, const uint32_t *a, const uint32_t *b, uint32_t *c, uint64_t batch,
                           cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    const TcGeometry &q = p->geo;
    TcArgs g{};
    g.a = q.swap ? b : a;
    g.b = q.swap ? a : b;
    g.c = c;
    g.na = q.na;
    g.nb = q.nb;
    g.nout = p->nout;
    g.ma = q.ma;
    g.mb = q.mb;
    g.tiles = q.tiles;
    g.batch = batch;
    g.scratch = p->scratch;
    g.scratch_stride = p->stride;
    g.xs = q.xs;
    g.w_off = q.w_off;
    g.braw_off = q.braw_off;
    g.spill_off = q.spill_off;
    g.flags_off = q.flags_off;
    g.bar_off = q.bar_off;
    const uint32_t grid = batch < p->ctas ? (uint32_t)batch : p->ctas;
    k_mul_quad_tc<<<grid, kThreads, q.smem, st>>>(g);
    return cudaGetLastError();
}

// Reads and clears the flag that a tensor-core kernel sets when an MMA wait
// timed out (synchronises the device).
cudaError_t tc_fault_take(uint32_t *flag) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyFromSymbol(flag, g_tc_fault, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    const uint32_t zero = 0;
    return cudaMemcpyToSymbol(g_tc_fault, &zero, sizeof(uint32_t));
}

}  // namespace bn
