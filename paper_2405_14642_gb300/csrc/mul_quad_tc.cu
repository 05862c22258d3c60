// Schoolbook product on the tensor cores (BN_OP_MUL_QUAD_TC).
//
// The product of Section 3 sums every word product A_i B_j into column i + j
// (Eq. 1).  This kernel computes the same column sums one level down, on
// bytes, as an exact contraction on the fifth-generation tensor cores: a byte
// is an exact fp16 integer, a byte product is below 2^16, and 128 of them sum
// below 2^23, where f32 arithmetic is exact whatever the order of the sums.
//
// Cut both operands into blocks of 128 bytes (a, the longer: blocks I < ma;
// b: J < mb) and let W_J be the 128 x 128 Toeplitz matrix W_J[r][c] =
// b-byte (128 J + r - c) (zero outside b).  Byte column 128 s + r of the
// product is then
//     sum_J  sum_c  W_J[r][c] * a-byte (128 (s - J) + c),
// J = 0..mb (block mb carries the top of b's last block).  Step J computes
// D_J = W_J X^T, one MMA chain with M = 128 (r), K = 128 (c) and N = ma:
// D's columns are circular, column n holding output block n while J <= n and
// block n + ma afterwards, so that D_J's column n is a-block n - J, or
// n - J + ma below J.  X is staged twice in a row (XX[I] = a-block I mod ma),
// which makes step J's B operand the window of XX starting at block ma - J.
// D_J is read from tensor memory, turned into integers and added into
// per-thread integer column sums (below 2^31: no rounding anywhere); once step
// J is added, column J holds all of block J, which is stored before the
// column starts over as block J + ma.  The column sums are folded into limbs
// by the transform products' normalisation (carry scan included).
//
// Per CTA (one per SM, persistent over the products) and product: XX in
// shared memory as fp16 in the tensor core's core-matrix layout, b as raw
// bytes.  Each step is a bias MMA (2048 x 4096 into every element, so D
// starts at 2^23; its constant operands are one core matrix each, repeated
// over the rows by a zero stride) and 8 MMAs of K = 16 over the block's 128
// bytes.  D = 2^23 + v with v < 2^23, so its bit pattern minus 0x4b000000 is
// v, which the epilogue warps add into per-thread integer column sums (four
// warps per group of 32 tensor-memory lanes, each a quarter of D's columns)
// and publish to a per-CTA scratch row.  Three kernels, by the width of D:
//  * k_mul_quad_tc (ma > 128): two D slots of 256 columns; warps 1-7 build
//    each step's Toeplitz rows (below) in shared memory, whose windows are the
//    MMAs' A operands, into one of two slots; warps 8-23 read D, warp 0 issues
//    the MMAs;
//  * k_mul_quad_tc_tw (64 < ma16 <= 128): W in tensor memory, built by the 16
//    epilogue warps; three D slots of 128 columns and two W slots;
//  * k_mul_quad_tc_tall (ma16 <= 64): every MMA's A operand is a window of
//    one Toeplitz matrix in shared memory, D takes all of tensor memory in
//    slots of 32 or 64 columns in two halves, three buffers of Toeplitz rows,
//    no bias MMA (a step's first MMA overwrites D and the epilogue adds the
//    2^23 in f32), and the staging and the carry into limbs overlap the MMAs
//    (see there).
// Warp 0 polls its mbarriers without sleeping (its wake-up is on the
// critical path).  Every wait is bounded; a timeout raises a device flag
// (bn_tc_check).
#include <cuda_runtime.h>

#include <new>
#include <type_traits>

#include "bn_internal.h"
#include "ntt_device.cuh"
#include "tc_device.cuh"

namespace bn {

__device__ uint32_t g_tc_fault;  // set when an MMA wait timed out

namespace {

constexpr uint32_t kThreads = 768;   // warp 0 issues the MMAs, warps 1-7 build W, warps 8-23 read D
constexpr uint32_t kBuildWarps = 7;
constexpr uint32_t kEpiWarps = 16;   // four per group of 32 tensor-memory lanes
constexpr uint32_t kBlk = 128;       // bytes per block: rows of W, K of a step
constexpr uint32_t kTmemCols = 512;  // the D slots
constexpr uint32_t kWSlotsMax = 4, kDSlotsMax = 4;  // mbarrier room for any of the kernels
constexpr uint32_t kTSlotBytes = 8192;          // one step's 240 Toeplitz rows (7.5 KB) in k_mul_quad_tc
constexpr uint64_t kWaitNs = 1000000000ull;     // 1 s per wait
constexpr uint32_t kMinSmem = 116 * 1024;       // one CTA per SM (the whole tensor memory each)

struct TcArgs {
    const uint32_t *a, *b;  // na >= nb (the host orders the operands)
    uint32_t *c;
    uint32_t na, nb, nout, ma, mb;
    uint32_t ma16;            // ma rounded up to 16: D's width (the MMA's N)
    uint64_t batch;
    uint32_t *scratch;        // per CTA: 128 (ma + mb) byte-column sums
    uint64_t scratch_stride;  // words per CTA
    uint32_t xs;              // bytes per K-chunk row of XX: (2 ma + ma16 - ma) * 16
    // shared-memory offsets (ca_off, cb_off: the bias MMA's operands; in k_mul_quad_tc_tall
    // ca_off holds a's words of the next product)
    uint32_t w_off, ca_off, cb_off, braw_off, spill_off, flags_off, bar_off;
    uint32_t x1_off;          // k_mul_quad_tc_tall: the second XX buffer
    uint32_t t_off, t_bytes;  // k_mul_quad_tc_tall: the kTBufs T buffers
};

// Quarter u of row r of W_J (words 16 u .. 16 u + 15) into registers, for a
// store to tensor memory.  Word k of row r holds the fp16 pair (W_J[r][2k],
// W_J[r][2k+1]) = (b-byte (v - 2k), b-byte (v - 2k - 1)), v = 128 J + r; braw
// holds b's bytes at offset 128 + index, zero outside b.
__device__ __forceinline__ void build_w_regs(const uint32_t *braw, uint32_t J, uint32_t r, uint32_t u,
                                             uint32_t (&out)[16]) {
    const uint32_t e = 97 + 128 * J + r - 32 * u;  // lowest byte offset this thread reads
    const uint32_t *bw = braw + (e >> 2);
    const uint32_t sh = e & 3u;
    uint32_t wv[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) wv[j] = bw[j];
    const uint32_t sel = (sh + 3) | ((sh + 2) << 4) | ((sh + 1) << 8) | (sh << 12);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t r0 = __byte_perm(wv[7 - 2 * q], wv[8 - 2 * q], sel);
        const uint32_t r1 = __byte_perm(wv[6 - 2 * q], wv[7 - 2 * q], sel);
        out[4 * q] = tc::bytes01_f16x2(r0);
        out[4 * q + 1] = tc::bytes23_f16x2(r0);
        out[4 * q + 2] = tc::bytes01_f16x2(r1);
        out[4 * q + 3] = tc::bytes23_f16x2(r1);
    }
}

// Every D starts at 2^23 (a first MMA multiplies 2048 by 4096 into each
// element); the byte products add an integer v < 2^23, so D = 2^23 + v is
// exact in f32 and, having exponent 23, its bit pattern is 0x4b000000 + v.
constexpr uint32_t kBiasBits = 0x4b000000u;
constexpr uint16_t kF16_2048 = 0x6800u, kF16_4096 = 0x6c00u;
constexpr uint32_t kBiasBytes = 256;  // each bias operand: one core matrix per K-chunk (8 rows, then zeros)

// Column f (warp-uniform, f < N of the M accumulators) stored to dst[stride f]
// and started over at zero, by a tree of uniform branches on f: a switch
// compiles to an indirect jump, which measured slower in these epilogues.
template <uint32_t LO, uint32_t N, uint32_t M>
__device__ __forceinline__ void flush_tree(uint32_t (&acc)[M], uint32_t f, uint32_t *dst, uint32_t stride) {
    if constexpr (N == 1) {
        dst[stride * LO] = acc[LO];
        acc[LO] = 0;
    } else {
        if (f < LO + N / 2) flush_tree<LO, N / 2, M>(acc, f, dst, stride);
        else flush_tree<LO + N / 2, N / 2, M>(acc, f, dst, stride);
    }
}
template <uint32_t M>
__device__ __forceinline__ void flush_column(uint32_t (&acc)[M], uint32_t f, uint32_t *dst, uint32_t stride) {
    flush_tree<0, M, M>(acc, f, dst, stride);
}

// ---- Toeplitz rows ----------------------------------------------------------
//
// K-chunk kk of W_J (its columns 16 kk .. 16 kk + 15) is the 128-row window
// starting at row R0 = 128 J - 16 kk of one tall matrix T[R][c] = b-byte (R - c),
// c < 16:  W_J[r][16 kk + c] = b-byte (128 J + r - 16 kk - c) = T[R0 + r][c].
// An MMA can therefore take its A operand from a window of T in shared memory
// (a descriptor offset) instead of a whole W_J: a step needs T's 240 rows
// 128 J - 112 .. 128 J + 127 (7.5 KB) where W_J takes 32 KB, and consecutive
// K-chunks' windows overlap by 7/8.  Layout of the A operand (K-major, no
// swizzle): row i, K-half h at (i / 8) * 256 + h * 128 + (i % 8) * 16, i.e.
// LBO = 128, SBO = 256.
constexpr uint32_t kTallRowBytes = 32;  // 16 fp16
constexpr uint32_t kTallLbo = 128, kTallSbo = 256;
constexpr uint32_t kTallLead = 112;     // rows of T below 128 J that step J's window reaches

// Row R of T (words k = 0..7: the fp16 pair (b-byte (R - 2k), b-byte (R - 2k - 1)))
// from braw (b's bytes at offset 128 + index, zero outside b; R >= -112).
__device__ __forceinline__ void tall_row(const uint32_t *braw, int32_t R, uint32_t (&w)[8]) {
    const uint32_t e = (uint32_t)(113 + R);  // braw byte of b-byte (R - 15)
    const uint32_t *bw = braw + (e >> 2);
    const uint32_t sh = e & 3u;
    uint32_t wv[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) wv[j] = bw[j];
    // x_m holds b-bytes R - 4m, R - 4m - 1, R - 4m - 2, R - 4m - 3 (bytes 0..3)
    const uint32_t sel = (sh + 3) | ((sh + 2) << 4) | ((sh + 1) << 8) | (sh << 12);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t x = __byte_perm(wv[3 - m], wv[4 - m], sel);
        w[2 * m] = tc::bytes01_f16x2(x);
        w[2 * m + 1] = tc::bytes23_f16x2(x);
    }
}

// Products whose longer operand has more than 128 blocks: two D slots of
// SLOTC = 256 columns; an epilogue warp owns 64 columns of its 32 lanes.
__global__ void __launch_bounds__(kThreads, 1) k_mul_quad_tc(TcArgs g) {
    constexpr uint32_t SLOTC = 256;
    constexpr uint32_t kDS = kTmemCols / SLOTC;  // D slots
    constexpr uint32_t kCPW = SLOTC / 128;       // 32-column chunks per epilogue warp
    constexpr uint32_t kWS = 2;                  // slots of Toeplitz rows
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *X = sm;  // XX and the T slots double as the normalisation's staging row
    uint8_t *W = sm + g.w_off;  // two slots of Toeplitz rows
    uint32_t *braw = reinterpret_cast<uint32_t *>(sm + g.braw_off);
    uint64_t *spill = reinterpret_cast<uint64_t *>(sm + g.spill_off);
    uint32_t *flags = reinterpret_cast<uint32_t *>(sm + g.flags_off);
    uint64_t *wfull = reinterpret_cast<uint64_t *>(sm + g.bar_off);  // [kWS], one arrival per builder warp
    uint64_t *wempty = wfull + kWSlotsMax;                              // [kWS], MMA commits
    uint64_t *dfull = wempty + kWSlotsMax;                              // [kDS], MMA commits
    uint64_t *dempty = dfull + kDSlotsMax;                              // [kDS], one arrival per warp
    uint32_t *slot = reinterpret_cast<uint32_t *>(dempty + kDSlotsMax);
    volatile uint32_t *abortf = slot + 1;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lq = warp & 3;  // the tensor-memory lanes this warp may move
    if (warp == 0) tc::tmem_alloc(slot, kTmemCols);
    if (tid < kBiasBytes / 2) {  // the bias MMA's operands: A[r][0] = 2048, B[n][0] = 4096, zero elsewhere
        reinterpret_cast<uint16_t *>(sm + g.ca_off)[tid] = (tid % 8 == 0 && tid < 64) ? kF16_2048 : 0;
        reinterpret_cast<uint16_t *>(sm + g.cb_off)[tid] = (tid % 8 == 0 && tid < 64) ? kF16_4096 : 0;
    }
    tc::fence_proxy_async();
    if (tid == 0) {
        for (uint32_t k = 0; k < kWS; ++k) {
            tc::mbar_init(&wfull[k], kBuildWarps);
            tc::mbar_init(&wempty[k], 1);
        }
        for (uint32_t k = 0; k < kDS; ++k) {
            tc::mbar_init(&dfull[k], 1);
            tc::mbar_init(&dempty[k], kEpiWarps);
        }
        *abortf = 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot, S = g.mb + 1;  // steps J = 0..mb
    const uint32_t lane_off = (32 * lq) << 16;
    const uint32_t x_s = tc::smem_u32(X), w_s = tc::smem_u32(W);
    uint32_t *cols = g.scratch + blockIdx.x * g.scratch_stride;
    uint32_t gs = 0;  // steps done by this CTA over all instances (slots and phases)
    bool fail = false;

    for (uint64_t inst = blockIdx.x; inst < g.batch; inst += gridDim.x) {
        const uint32_t *arow = g.a + inst * g.na, *brow = g.b + inst * g.nb;
        // ---- stage XX (fp16, core-matrix layout: a-block I at blocks I and
        // I + ma), its zero blocks up to D's width, and b's bytes
        for (uint32_t x = tid; x < 16 * g.ma; x += kThreads) {
            const uint32_t I = x >> 4, q = x & 15, w0 = 32 * I + 2 * q;
            const uint32_t u = w0 < g.na ? __ldg(arow + w0) : 0u;
            const uint32_t v = w0 + 1 < g.na ? __ldg(arow + w0 + 1) : 0u;
            const uint4 f = make_uint4(tc::bytes01_f16x2(u), tc::bytes23_f16x2(u), tc::bytes01_f16x2(v),
                                       tc::bytes23_f16x2(v));
            *reinterpret_cast<uint4 *>(X + q * g.xs + I * 16) = f;
            *reinterpret_cast<uint4 *>(X + q * g.xs + (I + g.ma) * 16) = f;
        }
        const uint32_t zb = g.ma16 - g.ma;
        for (uint32_t x = tid; x < 16 * zb; x += kThreads)
            *reinterpret_cast<uint4 *>(X + (x / zb) * g.xs + (2 * g.ma + x % zb) * 16) = make_uint4(0, 0, 0, 0);
        const uint32_t bwords = 32 * (g.mb + 2) + 4;
        for (uint32_t x = tid; x < bwords; x += kThreads)
            braw[x] = (x >= 32 && x - 32 < g.nb) ? __ldg(brow + x - 32) : 0u;
        tc::fence_proxy_async();
        __syncthreads();

        if (warp == 0) {
            // the warp waits and computes each step's descriptors together (so
            // they stay in uniform registers); one elected lane issues the
            // MMAs and commits them
            const uint32_t idesc = tc::idesc_f16_f32(128, g.ma16);
            const uint64_t bstep = (2 * g.xs) >> 4;
            for (uint32_t J = 0; J < S; ++J, ++gs) {
                const uint32_t k = gs % kWS, d = gs % kDS, ud = gs / kDS;
                bool ok = tc::mbar_wait_spin(&wfull[k], (gs / kWS) & 1u, kWaitNs, abortf);
                if (ok && ud > 0) ok = tc::mbar_wait_spin(&dempty[d], (ud - 1) & 1u, kWaitNs, abortf);
                if (!__all_sync(FULL_MASK, ok)) {
                    *abortf = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t dt = tbase + SLOTC * d;
                // T's rows of step J in slot k; K-chunk kk's window from row 112 - 16 kk
                const uint64_t ad = tc::smem_desc(w_s + k * kTSlotBytes + kTallLead * kTallRowBytes, kTallLbo, kTallSbo);
                const uint64_t bd = tc::smem_desc(x_s + (g.ma - J) * 16, g.xs, 128);  // XX from block ma - J
                // the bias operands' core matrix repeats over all row groups (stride 0)
                const uint64_t cad = tc::smem_desc(x_s + g.ca_off, 128, 0);
                const uint64_t cbd = tc::smem_desc(x_s + g.cb_off, 128, 0);
                if (tc::elect_one()) {
                    tc::mma_f16_ss(dt, cad, cbd, idesc, 0);  // D = 2^23
                    // K-chunks descending: each window sits 16 rows above the previous one
#pragma unroll
                    for (int kk = 7; kk >= 0; --kk)
                        tc::mma_f16_ss(dt, ad - kk * (16 * kTallRowBytes / 16), bd + kk * bstep, idesc, 1);
                    tc::mma_commit(&dfull[d]);
                    tc::mma_commit(&wempty[k]);
                }
                __syncwarp();
            }
        } else if (warp <= kBuildWarps) {
            // builders: T's 240 rows of each step (128 J - 112 .. 128 J + 127) into a
            // slot once the MMAs that last read it are done
            const uint32_t bt = tid - 32;
            for (uint32_t J = 0; J < S; ++J, ++gs) {
                const uint32_t k = gs % kWS, use = gs / kWS;
                if (use > 0 &&
                    !__all_sync(FULL_MASK, tc::mbar_wait(&wempty[k], (use - 1) & 1u, kWaitNs, abortf))) {
                    *abortf = 1;
                    break;
                }
                uint8_t *wk = W + k * kTSlotBytes;
                const int32_t Rbase = (int32_t)(kBlk * J) - (int32_t)kTallLead;
                for (uint32_t i = bt; i < kBlk + kTallLead; i += 32 * kBuildWarps) {
                    uint32_t w[8];
                    tall_row(braw, Rbase + (int32_t)i, w);
                    uint8_t *row = wk + (i >> 3) * kTallSbo + (i & 7) * 16;
                    *reinterpret_cast<uint4 *>(row) = make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4 *>(row + kTallLbo) = make_uint4(w[4], w[5], w[6], w[7]);
                }
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&wfull[k]);
            }
        } else {
            // epilogue: each finished D into the integer column sums; the 4 warps
            // of lane group lq own the columns [n0, n0 + SLOTC / 4)
            const uint32_t m = (warp - 1 - kBuildWarps) >> 2, n0 = 32 * kCPW * m;
            const uint32_t chi = (g.ma + 31) >> 5;        // chunks that hold D's ma columns
            uint32_t *const colr = cols + 32 * lq + lane;  // this thread's row of every column block
            uint32_t acc[kCPW * 32];
#pragma unroll
            for (int i = 0; i < (int)(kCPW * 32); ++i) acc[i] = 0;
            for (uint32_t J = 0; J < S; ++J, ++gs) {
                const uint32_t d = gs % kDS;
                if (!__all_sync(FULL_MASK, tc::mbar_wait(&dfull[d], (gs / kDS) & 1u, kWaitNs, abortf))) {
                    *abortf = 1;
                    break;
                }
                tc::fence_after_sync();
#pragma unroll
                for (int c = 0; c < (int)kCPW; ++c) {
                    const uint32_t ch = kCPW * m + c;
                    if (ch < chi) {
                        const uint32_t ta = tbase + lane_off + SLOTC * d + 32 * ch;
#pragma unroll
                        for (int hh = 0; hh < 4; ++hh) {  // 8 columns at a time: the register cap is 80
                            uint32_t v[8];
                            tc::tmem_ld8(ta + 8 * hh, v);
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[32 * c + 8 * hh + j] += v[j] - kBiasBits;
                        }
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&dempty[d]);
                // column J now holds all of block J: store it and start the column
                // over as block J + ma (after the last step, J = mb, every column
                // is published below instead)
                const uint32_t f = J - n0;  // warp-uniform
                if (J < g.mb && f < 32 * kCPW) flush_column(acc, f, colr + kBlk * n0, kBlk);
            }
            // publish: column n < mb went on to block n + ma after step n
#pragma unroll
            for (int c = 0; c < (int)kCPW; ++c)
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const uint32_t n = n0 + 32 * c + j;
                    if (n < g.ma) colr[kBlk * (n < g.mb ? n + g.ma : n)] = acc[32 * c + j];
                }
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
            tc::mbar_wait(&dfull[last % kDS], (last / kDS) & 1u, kWaitNs);
        }
        atomicOr(&g_tc_fault, 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

// Products whose longer operand has at most 128 blocks (up to 128K bits): D is
// at most 128 columns wide, so tensor memory holds three D slots and, beside
// them, two W slots (W_J as the MMA's A operand: 128 lanes x 64 columns of
// fp16 pairs).  The epilogue warps build W themselves: W_J's slot is free
// exactly when the step that read it last (J - 2) has delivered its D, which
// those warps wait for anyway.  No W goes through shared memory, which then
// only carries XX (the MMAs' B operand) and b's bytes.  17 warps: warp 0
// issues the MMAs; warps 1-16, four per group of 32 tensor-memory lanes, each
// build a quarter of their lanes' W rows (16 columns), read 32 columns of D
// (one load) and keep those columns' sums.
constexpr uint32_t kThreadsTw = 544;
constexpr uint32_t kWColsTw = 64;  // tensor-memory columns per W slot

__global__ void __launch_bounds__(kThreadsTw, 1) k_mul_quad_tc_tw(TcArgs g) {
    constexpr uint32_t kDSlotsTw = 3, kWSlotsTw = 2;
    constexpr uint32_t kDColsTw = 128;      // tensor-memory columns per D slot
    constexpr uint32_t kCW = kDColsTw / 4;  // D columns per epilogue warp
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *X = sm;  // XX doubles as the normalisation's staging row
    uint32_t *braw = reinterpret_cast<uint32_t *>(sm + g.braw_off);
    uint64_t *spill = reinterpret_cast<uint64_t *>(sm + g.spill_off);
    uint32_t *flags = reinterpret_cast<uint32_t *>(sm + g.flags_off);
    uint64_t *wfull = reinterpret_cast<uint64_t *>(sm + g.bar_off);  // [kWSlotsTw], one arrival per epilogue warp
    uint64_t *dfull = wfull + kWSlotsMax;                               // [kDSlotsTw], MMA commits
    uint64_t *dempty = dfull + kDSlotsMax;                              // [kDSlotsTw], one arrival per epilogue warp
    uint32_t *slot = reinterpret_cast<uint32_t *>(dempty + kDSlotsMax);
    volatile uint32_t *abortf = slot + 1;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lq = warp & 3;  // the tensor-memory lanes this warp may move
    if (warp == 0) tc::tmem_alloc(slot, kTmemCols);
    if (tid < kBiasBytes / 2) {  // the bias MMA's operands: A[r][0] = 2048, B[n][0] = 4096, zero elsewhere
        reinterpret_cast<uint16_t *>(sm + g.ca_off)[tid] = (tid % 8 == 0 && tid < 64) ? kF16_2048 : 0;
        reinterpret_cast<uint16_t *>(sm + g.cb_off)[tid] = (tid % 8 == 0 && tid < 64) ? kF16_4096 : 0;
    }
    tc::fence_proxy_async();
    if (tid == 0) {
        for (uint32_t k = 0; k < kWSlotsTw; ++k) tc::mbar_init(&wfull[k], kEpiWarps);
        for (uint32_t k = 0; k < kDSlotsTw; ++k) {
            tc::mbar_init(&dfull[k], 1);
            tc::mbar_init(&dempty[k], kEpiWarps);
        }
        *abortf = 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot, S = g.mb + 1;  // steps J = 0..mb
    const uint32_t wbase = tbase + kDSlotsTw * kDColsTw;  // W slot k at column wbase + 64 k (ends at 512)
    const uint32_t lane_off = (32 * lq) << 16;
    const uint32_t x_s = tc::smem_u32(X);
    uint32_t *cols = g.scratch + blockIdx.x * g.scratch_stride;
    uint32_t gs = 0;  // steps done by this CTA over all instances (slots and phases)
    bool fail = false;

    for (uint64_t inst = blockIdx.x; inst < g.batch; inst += gridDim.x) {
        const uint32_t *arow = g.a + inst * g.na, *brow = g.b + inst * g.nb;
        // ---- stage XX (a-block I at blocks I and I + ma), its zero blocks up
        // to D's width, and b's bytes
        for (uint32_t x = tid; x < 16 * g.ma; x += kThreadsTw) {
            const uint32_t I = x >> 4, q = x & 15, w0 = 32 * I + 2 * q;
            const uint32_t u = w0 < g.na ? __ldg(arow + w0) : 0u;
            const uint32_t v = w0 + 1 < g.na ? __ldg(arow + w0 + 1) : 0u;
            const uint4 f = make_uint4(tc::bytes01_f16x2(u), tc::bytes23_f16x2(u), tc::bytes01_f16x2(v),
                                       tc::bytes23_f16x2(v));
            *reinterpret_cast<uint4 *>(X + q * g.xs + I * 16) = f;
            *reinterpret_cast<uint4 *>(X + q * g.xs + (I + g.ma) * 16) = f;
        }
        const uint32_t zb = g.ma16 - g.ma;
        for (uint32_t x = tid; x < 16 * zb; x += kThreadsTw)
            *reinterpret_cast<uint4 *>(X + (x / zb) * g.xs + (2 * g.ma + x % zb) * 16) = make_uint4(0, 0, 0, 0);
        const uint32_t bwords = 32 * (g.mb + 2) + 4;
        for (uint32_t x = tid; x < bwords; x += kThreadsTw)
            braw[x] = (x >= 32 && x - 32 < g.nb) ? __ldg(brow + x - 32) : 0u;
        tc::fence_proxy_async();
        __syncthreads();

        if (warp == 0) {
            const uint32_t idesc = tc::idesc_f16_f32(128, g.ma16);
            const uint64_t bstep = (2 * g.xs) >> 4;
            const uint64_t cad = tc::smem_desc(x_s + g.ca_off, 128, 0), cbd = tc::smem_desc(x_s + g.cb_off, 128, 0);
            for (uint32_t J = 0; J < S; ++J) {
                const uint32_t ud = gs / kDSlotsTw;
                bool ok = tc::mbar_wait_spin(&wfull[gs % kWSlotsTw], (gs / kWSlotsTw) & 1u, kWaitNs, abortf);
                if (ok && ud > 0) ok = tc::mbar_wait_spin(&dempty[gs % kDSlotsTw], (ud - 1) & 1u, kWaitNs, abortf);
                if (!__all_sync(FULL_MASK, ok)) {
                    *abortf = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t dt = tbase + kDColsTw * (gs % kDSlotsTw);
                const uint32_t at = wbase + kWColsTw * (gs % kWSlotsTw);
                const uint64_t bd = tc::smem_desc(x_s + (g.ma - J) * 16, g.xs, 128);  // XX from block ma - J
                if (tc::elect_one()) {
                    tc::mma_f16_ss(dt, cad, cbd, idesc, 0);  // D = 2^23
#pragma unroll
                    for (uint32_t kk = 0; kk < 8; ++kk) tc::mma_f16_ts(dt, at + 8 * kk, bd + kk * bstep, idesc, 1);
                    tc::mma_commit(&dfull[gs % kDSlotsTw]);
                }
                __syncwarp();
                ++gs;
            }
        } else {
            // column quarter m: D columns [kCW m, kCW m + kCW), W columns [16 m, 16 m + 16)
            const uint32_t m = (warp - 1) >> 2, n0 = kCW * m, r = 32 * lq + lane;
            uint32_t *const colr = cols + r;  // this thread's row of every column block
            uint32_t acc[1][kCW];
#pragma unroll
            for (int i = 0; i < (int)kCW; ++i) acc[0][i] = 0;
            // W_0 .. W_{kWSlotsTw - 1} (their slots are free: every earlier MMA
            // has delivered its D)
            for (uint32_t J = 0; J < kWSlotsTw && J < S; ++J) {
                uint32_t w16[16];
                build_w_regs(braw, J, r, m, w16);
                tc::tmem_st16(wbase + lane_off + kWColsTw * ((gs + J) % kWSlotsTw) + 16 * m, w16);
                tc::tmem_st_wait();
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&wfull[(gs + J) % kWSlotsTw]);
            }
            for (uint32_t J = 0; J < S; ++J, ++gs) {
                const uint32_t d = gs % kDSlotsTw;
                if (!__all_sync(FULL_MASK, tc::mbar_wait(&dfull[d], (gs / kDSlotsTw) & 1u, kWaitNs, abortf))) {
                    *abortf = 1;
                    break;
                }
                tc::fence_after_sync();
                // W_{J+kWSlotsTw} into the slot step J has finished reading,
                // released to the MMA warp before D is read (it gates later MMAs)
                if (J + kWSlotsTw < S) {
                    uint32_t w16[16];
                    build_w_regs(braw, J + kWSlotsTw, r, m, w16);
                    tc::tmem_st16(wbase + lane_off + kWColsTw * (gs % kWSlotsTw) + 16 * m, w16);
                    tc::tmem_st_wait();
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&wfull[gs % kWSlotsTw]);
                }
                if (n0 < g.ma) {  // the warp's kCW columns of D in one load
                    uint32_t v[kCW];
                    tc::tmem_ld32(tbase + lane_off + kDColsTw * d + n0, v);
#pragma unroll
                    for (int j = 0; j < (int)kCW; ++j) acc[0][j] += v[j] - kBiasBits;
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&dempty[d]);
                // column J now holds all of block J: store it and start the column
                // over as block J + ma
                const uint32_t f = J - n0;  // warp-uniform
                if (J < g.mb && f < kCW) flush_column(acc[0], f, colr + kBlk * n0, kBlk);
            }
            // publish: column n < mb went on to block n + ma after step n (two
            // loops with one destination each: this form compiles without spills)
#pragma unroll
            for (int j = 0; j < (int)kCW; ++j)
                if (n0 + j >= g.mb && n0 + j < g.ma) colr[kBlk * (n0 + j)] = acc[0][j];
            uint32_t *const colr_hi = colr + kBlk * g.ma;
#pragma unroll
            for (int j = 0; j < (int)kCW; ++j)
                if (n0 + j < g.mb) colr_hi[kBlk * (n0 + j)] = acc[0][j];
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
            tc::mbar_wait(&dfull[last % kDSlotsTw], (last / kDSlotsTw) & 1u, kWaitNs);
        }
        atomicOr(&g_tc_fault, 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}
// ---- up to 64K bits: the Toeplitz rows in shared memory --------------------
//
// At N = ma16 <= 64 one MMA carries little work (128 x N x 16 products) and its
// cost is set by the operands it reads from shared memory.  Every MMA takes
// its A operand from a window of T (the Toeplitz rows above): no W is built
// per step, a step's eight MMAs run back to back with K-chunks descending so
// that each window sits 16 rows above the previous one (also from one step to
// the next), and all of tensor memory holds D: 512 / DW slots in two halves,
// group g of steps (half as many steps as slots) writing half g % 2 while the
// other half is read.  The first MMA of a step overwrites its slot, so D holds
// that step's column sums v < 2^23 exactly; the epilogue takes the integer
// from the bit pattern of v + 2^23 (0x4b000000 + v).
//
// Roles, so that nothing but MMAs sits on the tensor pipe's critical path:
//  * warp 0 issues the MMAs (group g reads T buffer g % 3 and D half g % 2,
//    product p reads XX buffer p % 2) and commits once per group;
//  * warps 1-8 (epilogue) read each group's D half once the group has
//    completed, keep the column sums, store each finished column, publish the
//    rest per product into one of two column-sum rows, and free the half;
//  * warps 9-16 (producer) stage each product's XX and b's bytes from a copy
//    of the product's rows fetched (cp.async) while the previous product ran,
//    and build each group's rows of T: R in [128 J - 112, 128 (J + n)), in
//    the A operand's layout (K-major, no swizzle: row i, K-half h at
//    (i / 8) * 256 + h * 128 + (i % 8) * 16, i.e. LBO = 128, SBO = 256), up to
//    three groups ahead of the tensor pipe;
//  * the column sums of each product are carried into limbs by four more
//    warps at DW = 64 (17-20), or by the producer once three groups of the
//    next product are built at DW = 32.
// mbarriers link them (tfull/tempty per T buffer, the latter also telling the
// epilogue that the group's D half is complete; dempty per D half; xfull/
// xempty per XX buffer; cfull/cempty per column-sum row; the producer's and
// the normalising warps' own barriers are mbarriers too), and every wait is
// bounded and watches the CTA's abort flag.
constexpr uint32_t kEpiTall = 8;    // two per group of 32 tensor-memory lanes
constexpr uint32_t kProdWarps = 8;
constexpr uint32_t kTBufs = 3;      // T buffers: the producer builds up to three groups ahead
template <uint32_t DW>
constexpr uint32_t norm_warps() { return DW == 64 ? 4u : 0u; }
template <uint32_t DW>
constexpr uint32_t threads_tall() { return 32 * (1 + kEpiTall + kProdWarps + norm_warps<DW>()); }

// A barrier among the warps of one role: each warp's lane 0 arrives on an
// mbarrier counting those warps (release: the warp's earlier writes, shared
// or global, are visible to a thread that sees the phase complete), then
// every thread waits for the phase (bounded, watching the abort flag).
__device__ __forceinline__ bool role_sync(uint64_t *bar, uint32_t &phase, volatile uint32_t *abortf) {
    __threadfence_block();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(bar);
    const bool ok = __all_sync(FULL_MASK, tc::mbar_wait(bar, phase, kWaitNs, abortf));
    phase ^= 1u;
    if (!ok) *abortf = 1;
    return ok;
}

// normalize_limbs for the NW warps of one role (thread t of NT = 32 NW),
// synchronised by role_sync: column sums -> limbs, carry scan, copy-out.  A
// byte column holds at most 8192 byte products (64K bits), so its sum is
// below 2^29 and a limb (four columns) below 2^54: a 64-bit running carry
// suffices.  The limbs' loads go out eight at a time.
template <uint32_t NW, class LimbFn>
__device__ bool normalize_role(uint32_t nout, uint32_t *crow, uint32_t *out_s, uint64_t *spill, uint32_t *flags,
                               uint32_t t, uint64_t *bar, uint32_t &phase, volatile uint32_t *abortf,
                               LimbFn &&limb) {
    constexpr uint32_t NT = 32 * NW;
    const uint32_t lane = t & 31, w = t >> 5;
    uint32_t QN = (nout + NT - 1) / NT;
    if (QN < 2) QN = 2;  // a window must absorb a two-word spill
    const uint32_t k0 = t * QN;
    const uint32_t k1 = k0 + QN < nout ? k0 + QN : nout;
    // (a) this window's limbs, carrying within the window
    uint64_t carry = 0;
    for (uint32_t k = k0; k < k1; k += 8) {
        uint64_t lv[8];
#pragma unroll
        for (uint32_t j = 0; j < 8; ++j) lv[j] = k + j < k1 ? limb(k + j) : 0;
#pragma unroll
        for (uint32_t j = 0; j < 8; ++j)
            if (k + j < k1) {
                const uint64_t v = lv[j] + carry;
                out_s[ntt::stage_index(k + j)] = (uint32_t)v;
                carry = v >> 32;
            }
    }
    spill[t] = carry;
    if (!role_sync(bar, phase, abortf)) return false;
    // (b) add the previous window's spill
    uint64_t c = t > 0 ? spill[t - 1] : 0;
    uint32_t all = 0xffffffffu;
    for (uint32_t k = k0; k < k1; ++k) {
        const uint64_t v = (uint64_t)out_s[ntt::stage_index(k)] + (c & 0xffffffffu);
        out_s[ntt::stage_index(k)] = (uint32_t)v;
        c = (c >> 32) + (v >> 32);
        all &= (uint32_t)v;
    }
    const bool owns = k0 < k1;
    BN_DEBUG_CHECK(!(owns && k1 == nout) || c == 0, kDbgSpill);
    BN_DEBUG_CHECK(owns || c == 0, kDbgSpill);
    // (c) carry scan over the NT windows in memory order (Section 2)
    const RowFlags f{__ballot_sync(FULL_MASK, owns && c != 0), __ballot_sync(FULL_MASK, owns && all == 0xffffffffu)};
    uint32_t wc;
    row_carries(f, 0, wc);
    if (lane == 0) flags[w] = wc | ((f.P == FULL_MASK) << 1);
    if (!role_sync(bar, phase, abortf)) return false;
    const uint32_t sw = lane < NW ? flags[lane] : 0u;
    const RowFlags fw{__ballot_sync(FULL_MASK, sw & 1u), __ballot_sync(FULL_MASK, (sw >> 1) & 1u)};
    uint32_t unused;
    const uint32_t wcin = (row_carries(fw, 0, unused) >> w) & 1u;
    const uint32_t cin = (row_carries(f, wcin, unused) >> lane) & 1u;
    BN_DEBUG_CHECK(!(owns && k1 == nout && cin && all == 0xffffffffu), kDbgSpill);
    if (cin)
        for (uint32_t k = k0; k < k1; ++k)
            if (++out_s[ntt::stage_index(k)] != 0) break;
    if (!role_sync(bar, phase, abortf)) return false;
    // (d) coalesced copy-out; the staging row and flags are free again after the barrier
    for (uint32_t x = t; x < nout; x += NT) st_stream(crow + x, out_s[ntt::stage_index(x)]);
    return role_sync(bar, phase, abortf);
}

// Limb k of a column-sum row (four byte columns per limb).
__device__ __forceinline__ uint64_t limb_of(const uint32_t *cols, uint32_t k) {
    const uint4 v = *reinterpret_cast<const uint4 *>(cols + 4 * k);
    return (uint64_t)v.x + ((uint64_t)v.y << 8) + ((uint64_t)v.z << 16) + ((uint64_t)v.w << 24);
}

// Four-byte asynchronous copy global -> shared (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <uint32_t DW>
__global__ void __launch_bounds__(threads_tall<DW>(), 1) k_mul_quad_tc_tall(TcArgs g) {
    constexpr uint32_t kDS = kTmemCols / DW;  // D slots
    constexpr uint32_t kC = kDS / 2;          // steps per group: one D half
    constexpr uint32_t kCW = DW / 2;          // D columns per epilogue warp
    constexpr uint32_t kNW = norm_warps<DW>();
    extern __shared__ __align__(1024) uint8_t sm[];
    // XX buffers at 0 and g.x1_off, T buffers from g.t_off (g.t_bytes each), a's
    // words of the next product at g.ca_off, b's bytes (two copies) at g.braw_off,
    // the normalisation's staging row at g.spill_off followed by its spill words
    uint8_t *const X0 = sm, *const X1 = sm + g.x1_off;
    uint32_t *const araw = reinterpret_cast<uint32_t *>(sm + g.ca_off);
    uint32_t *const braw0 = reinterpret_cast<uint32_t *>(sm + g.braw_off);
    uint32_t *const braw1 = braw0 + (32 * (g.mb + 2) + 4);
    uint32_t *out_s = reinterpret_cast<uint32_t *>(sm + g.spill_off);
    uint64_t *spill = reinterpret_cast<uint64_t *>(sm + g.spill_off + ((4 * ntt::stage_index(g.nout) + 16 + 15) & ~15u));
    uint32_t *flags = reinterpret_cast<uint32_t *>(sm + g.flags_off);
    uint64_t *tfull = reinterpret_cast<uint64_t *>(sm + g.bar_off);  // [kTBufs] one arrival per producer warp
    uint64_t *tempty = tfull + kTBufs;  // [kTBufs] MMA commits: the group has completed
    uint64_t *dempty = tempty + kTBufs; // [2] one arrival per epilogue warp: the D half is free
    uint64_t *xfull = dempty + 2;       // [2] one arrival per producer warp
    uint64_t *xempty = xfull + 2;       // [2] MMA commits
    uint64_t *cfull = xempty + 2;       // [2] one arrival per epilogue warp
    uint64_t *cempty = cfull + 2;       // [2] one arrival per normalising warp
    uint64_t *pbar = cempty + 2;        // the producer warps' own barrier
    uint64_t *nbar = pbar + 1;          // the normalising warps' own barrier
    uint32_t *slot = reinterpret_cast<uint32_t *>(nbar + 1);
    volatile uint32_t *abortf = slot + 1;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(slot, kTmemCols);
    if (tid == 0) {
        for (uint32_t k = 0; k < kTBufs; ++k) {
            tc::mbar_init(&tfull[k], kProdWarps);
            tc::mbar_init(&tempty[k], 1);
        }
        for (uint32_t k = 0; k < 2; ++k) {
            tc::mbar_init(&dempty[k], kEpiTall);
            tc::mbar_init(&xfull[k], kProdWarps);
            tc::mbar_init(&xempty[k], 1);
            tc::mbar_init(&cfull[k], kEpiTall);
            tc::mbar_init(&cempty[k], kNW ? kNW : kProdWarps);
        }
        tc::mbar_init(pbar, kProdWarps);
        tc::mbar_init(nbar, kNW ? kNW : 1);
        *abortf = 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot, S = g.mb + 1;  // steps J = 0..mb of a product
    // this CTA's two column-sum rows (product p uses row p % 2)
    uint32_t *const cols0 = g.scratch + blockIdx.x * g.scratch_stride;
    uint32_t *const cols1 = cols0 + g.scratch_stride / 2;
    // column sums of product q (instance inst) -> limbs, by the NW warps of a role
    auto finish = [&](uint32_t q, uint64_t inst, uint32_t t, uint64_t *bar, uint32_t &ph, auto nw) -> bool {
        const uint32_t cb = q & 1u;
        const uint32_t *cols = cb ? cols1 : cols0;
        if (!__all_sync(FULL_MASK, tc::mbar_wait(&cfull[cb], (q >> 1) & 1u, kWaitNs, abortf))) return false;
        const bool done = normalize_role<decltype(nw)::value>(g.nout, g.c + inst * g.nout, out_s, spill, flags, t,
                                                               bar, ph, abortf,
                                                               [&](uint32_t k) { return limb_of(cols, k); });
        __syncwarp();
        if (done && lane == 0) tc::mbar_arrive(&cempty[cb]);
        return done;
    };

    if (warp == 0) {
        // ---- MMA warp
        const uint32_t idesc = tc::idesc_f16_f32(128, g.ma16);
        const uint64_t bstep = (2 * g.xs) >> 4;
        const uint32_t s0 = tc::smem_u32(sm);
        uint32_t gg = 0, pi = 0;  // groups, products issued by this CTA
        bool ok = true;
        for (uint64_t inst = blockIdx.x; inst < g.batch && ok; inst += gridDim.x, ++pi) {
            const uint32_t xb = pi & 1u, x_s = s0 + (xb ? g.x1_off : 0u);
            ok = __all_sync(FULL_MASK, tc::mbar_wait_spin(&xfull[xb], (pi >> 1) & 1u, kWaitNs, abortf));
            for (uint32_t J = 0; J < S && ok; J += kC, ++gg) {
                const uint32_t n = J + kC <= S ? kC : S - J;  // steps of this group
                const uint32_t tb = gg % kTBufs, dh = gg & 1u, t_s = s0 + g.t_off + tb * g.t_bytes;
                if (gg >= 2) ok = tc::mbar_wait_spin(&dempty[dh], ((gg - 2) >> 1) & 1u, kWaitNs, abortf);
                if (ok) ok = tc::mbar_wait_spin(&tfull[tb], (gg / kTBufs) & 1u, kWaitNs, abortf);
                ok = __all_sync(FULL_MASK, ok);
                if (!ok) break;
                tc::fence_after_sync();
                if (tc::elect_one()) {
                    // step J + h: D slot kC dh + h, its T window at K-chunk 0 (row 128 h + 112
                    // of the group's rows) and its XX window (block ma - J - h); K-chunk kk
                    // moves T 16 rows up and XX two K-chunks on
                    uint32_t dt[kC];
                    uint64_t ad[kC], bd[kC];
#pragma unroll
                    for (uint32_t h = 0; h < kC; ++h) {
                        const uint32_t hh = h < n ? h : 0;  // (unused beyond n)
                        dt[h] = tbase + DW * (kC * dh + hh);
                        ad[h] = tc::smem_desc(t_s + (kBlk * hh + kTallLead) * kTallRowBytes, kTallLbo, kTallSbo);
                        bd[h] = tc::smem_desc(x_s + (g.ma - J - hh) * 16, g.xs, 128);
                    }
                    // step by step, K-chunks from 7 down to 0: each MMA's T window sits 16 rows
                    // above the one before, also from one step to the next, so consecutive MMAs
                    // share 7/8 of their A operand; a step's first MMA overwrites its slot
#pragma unroll
                    for (uint32_t h = 0; h < kC; ++h) {
                        if (h >= n) break;
#pragma unroll
                        for (int kk = 7; kk >= 0; --kk)
                            tc::mma_f16_ss(dt[h], ad[h] - kk * (16 * kTallRowBytes / 16), bd[h] + kk * bstep, idesc,
                                           kk != 7);
                    }
                    tc::mma_commit(&tempty[tb]);                // the group's D half is complete, T buffer tb free
                    if (J + n == S) tc::mma_commit(&xempty[xb]);  // XX buffer xb may be restaged
                }
                __syncwarp();
            }
        }
        if (!ok) *abortf = 1;
        // the MMAs issued last finish before tensor memory is freed (bounded; at once
        // when the epilogue has already seen them)
        if (lane == 0 && gg > 0) tc::mbar_wait(&tempty[(gg - 1) % kTBufs], ((gg - 1) / kTBufs) & 1u, kWaitNs);
        __syncwarp();
    } else if (kNW && warp > kEpiTall + kProdWarps) {
        // ---- normalising warps: each product's column sums -> limbs
        const uint32_t nt = tid - 32 * (1 + kEpiTall + kProdWarps);
        uint32_t nph = 0, pi = 0;
        bool ok = true;
        for (uint64_t inst = blockIdx.x; inst < g.batch && ok; inst += gridDim.x, ++pi)
            ok = finish(pi, inst, nt, nbar, nph, std::integral_constant<uint32_t, (kNW ? kNW : 1)>{});
        if (!ok) *abortf = 1;
    } else if (warp > kEpiTall) {
        // ---- producer warps: XX and b's bytes of each product, T's rows of each
        // group (and, at DW = 32, the previous product's limbs)
        const uint32_t pt = tid - 32 * (1 + kEpiTall);
        constexpr uint32_t PT = 32 * kProdWarps;
        const uint32_t bwords = 32 * (g.mb + 2) + 4;
        uint32_t gg = 0, pi = 0, pph = 0;
        bool ok = true;
        // a's and b's words of product inst into araw and braw (asynchronously)
        auto prefetch = [&](uint64_t inst, uint32_t *braw) {
            const uint32_t *arow = g.a + inst * g.na, *brow = g.b + inst * g.nb;
            for (uint32_t x = pt; x < g.na; x += PT) cp_async4(araw + x, arow + x);
            for (uint32_t x = pt; x < g.nb; x += PT) cp_async4(braw + 32 + x, brow + x);
            cp_async_commit();
        };
        // araw beyond na and braw outside b stay zero
        for (uint32_t x = pt; x < 32 * g.ma; x += PT) araw[x] = 0;
        for (uint32_t x = pt; x < bwords; x += PT) braw0[x] = braw1[x] = 0;
        ok = role_sync(pbar, pph, abortf);
        if (ok && blockIdx.x < g.batch) prefetch(blockIdx.x, braw0);
        for (uint64_t inst = blockIdx.x; inst < g.batch && ok; inst += gridDim.x, ++pi) {
            const uint32_t xb = pi & 1u;
            uint8_t *const X = xb ? X1 : X0;
            uint32_t *const braw = xb ? braw1 : braw0;
            if (pi >= 2) ok = __all_sync(FULL_MASK, tc::mbar_wait(&xempty[xb], ((pi - 2) >> 1) & 1u, kWaitNs, abortf));
            cp_async_wait_all();
            if (!ok || !role_sync(pbar, pph, abortf)) {  // every thread's copies have landed
                ok = false;
                break;
            }
            // XX: a-block I at blocks I and I + ma, zero blocks up to D's width
            for (uint32_t x = pt; x < 16 * g.ma; x += PT) {
                const uint32_t I = x >> 4, q = x & 15, w0 = 32 * I + 2 * q;
                const uint32_t u = araw[w0], v = araw[w0 + 1];
                const uint4 f = make_uint4(tc::bytes01_f16x2(u), tc::bytes23_f16x2(u), tc::bytes01_f16x2(v),
                                           tc::bytes23_f16x2(v));
                *reinterpret_cast<uint4 *>(X + q * g.xs + I * 16) = f;
                *reinterpret_cast<uint4 *>(X + q * g.xs + (I + g.ma) * 16) = f;
            }
            const uint32_t zb = g.ma16 - g.ma;
            for (uint32_t x = pt; x < 16 * zb; x += PT)
                *reinterpret_cast<uint4 *>(X + (x / zb) * g.xs + (2 * g.ma + x % zb) * 16) = make_uint4(0, 0, 0, 0);
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&xfull[xb]);
            // araw has been read by every thread, and the other braw copy (the product
            // before this one) is no longer read: fetch the next product's rows
            if (!role_sync(pbar, pph, abortf)) {
                ok = false;
                break;
            }
            if (inst + gridDim.x < g.batch) prefetch(inst + gridDim.x, xb ? braw0 : braw1);
            uint32_t k = 0;  // group of this product
            for (uint32_t J = 0; J < S && ok; J += kC, ++gg, ++k) {
                const uint32_t n = J + kC <= S ? kC : S - J, tb = gg % kTBufs;
                uint8_t *const Tb = sm + g.t_off + tb * g.t_bytes;
                if (gg >= kTBufs)
                    ok = __all_sync(FULL_MASK,
                                    tc::mbar_wait(&tempty[tb], ((gg - kTBufs) / kTBufs) & 1u, kWaitNs, abortf));
                if (!ok) break;
                const int32_t Rbase = (int32_t)(kBlk * J) - (int32_t)kTallLead;
                const uint32_t nrows = kBlk * n + kTallLead;
                for (uint32_t i = pt; i < nrows; i += PT) {
                    uint32_t w[8];
                    tall_row(braw, Rbase + (int32_t)i, w);
                    uint8_t *row = Tb + (i >> 3) * kTallSbo + (i & 7) * 16;
                    *reinterpret_cast<uint4 *>(row) = make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4 *>(row + kTallLbo) = make_uint4(w[4], w[5], w[6], w[7]);
                }
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&tfull[tb]);
                // every T buffer holds this product's work: finish the previous product
                if (!kNW && pi > 0 && (k == kTBufs - 1 || (J + n == S && k < kTBufs - 1)))
                    ok = finish(pi - 1, inst - gridDim.x, pt, pbar, pph, std::integral_constant<uint32_t, kProdWarps>{});
            }
        }
        cp_async_wait_all();  // nothing in flight into shared memory at exit
        if (!kNW && ok && pi > 0)
            ok = finish(pi - 1, blockIdx.x + (uint64_t)(pi - 1) * gridDim.x, pt, pbar, pph,
                        std::integral_constant<uint32_t, kProdWarps>{});
        if (!ok) *abortf = 1;
    } else {
        // ---- epilogue warps: column half m, D columns [kCW m, kCW m + kCW)
        const uint32_t lq = warp & 3;  // the tensor-memory lanes this warp may move
        const uint32_t m = (warp - 1) >> 2, n0 = kCW * m, r = 32 * lq + lane;
        const uint32_t lane_off = (32 * lq) << 16;
        uint32_t eg = 0, pi = 0;  // groups read, products
        bool ok = true;
        for (uint64_t inst = blockIdx.x; inst < g.batch && ok; inst += gridDim.x, ++pi) {
            const uint32_t cb = pi & 1u;
            uint32_t *const colr = (cb ? cols1 : cols0) + r;  // this thread's row of every column block
            if (pi >= 2) ok = __all_sync(FULL_MASK, tc::mbar_wait(&cempty[cb], ((pi - 2) >> 1) & 1u, kWaitNs, abortf));
            if (!ok) break;
            uint32_t acc[kCW];
#pragma unroll
            for (uint32_t i = 0; i < kCW; ++i) acc[i] = 0;
            // step J: wait for its group at the group's first step, add the step's D
            // columns, free the D half after the group's last step
            auto step = [&](uint32_t J) -> bool {
                const uint32_t jh = J % kC;
                if (jh == 0 && !__all_sync(FULL_MASK, tc::mbar_wait(&tempty[eg % kTBufs], (eg / kTBufs) & 1u,
                                                                    kWaitNs, abortf)))
                    return false;
                tc::fence_after_sync();
                if (n0 < g.ma) {
                    uint32_t v[kCW];
                    const uint32_t ta = tbase + lane_off + DW * (kC * (eg & 1u) + jh) + n0;
                    tc::tmem_ld16_async(ta, v);
                    if constexpr (kCW == 32) tc::tmem_ld16_async(ta + 16, v + 16);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (uint32_t j = 0; j < kCW; ++j)
                        acc[j] += __float_as_uint(__uint_as_float(v[j]) + 8388608.0f) - kBiasBits;
                }
                if (jh == kC - 1 || J == S - 1) {  // the group's D half may be overwritten
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&dempty[eg & 1u]);
                    ++eg;
                }
                return true;
            };
            // three runs of steps: before this warp's columns, the run in which step J
            // completes column J - n0 of this warp (unrolled, so that the column is a
            // register: store it and start it over as block J + ma), and the rest
            const uint32_t jb = n0 < g.mb ? n0 : g.mb;
            const uint32_t je = n0 + kCW < g.mb ? n0 + kCW : g.mb;
            uint32_t J = 0;
            for (; J < jb && ok; ++J) ok = step(J);
#pragma unroll
            for (uint32_t x = 0; x < kCW; ++x) {
                if (!ok || n0 + x >= je) break;
                ok = step(n0 + x);
                colr[kBlk * (n0 + x)] = acc[x];
                acc[x] = 0;
            }
            if (J < je) J = je;
            for (; J < S && ok; ++J) ok = step(J);
            if (!ok) break;
            // publish: column n < mb went on to block n + ma after step n
#pragma unroll
            for (uint32_t j = 0; j < kCW; ++j)
                if (n0 + j >= g.mb && n0 + j < g.ma) colr[kBlk * (n0 + j)] = acc[j];
            uint32_t *const colr_hi = colr + kBlk * g.ma;
#pragma unroll
            for (uint32_t j = 0; j < kCW; ++j)
                if (n0 + j < g.mb) colr_hi[kBlk * (n0 + j)] = acc[j];
            __threadfence_block();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&cfull[cb]);  // the normalising warps carry them into limbs
        }
        if (!ok) *abortf = 1;
    }
    if (tid == 0 && *abortf) atomicOr(&g_tc_fault, 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

struct TcGeometry {
    uint32_t na, nb, ma, mb, ma16, xs, w_off, ca_off, cb_off, braw_off, spill_off, flags_off, bar_off, smem;
    bool swap, tw;  // tw: W in tensor memory (k_mul_quad_tc_tw, 64 < ma16 <= 128)
    bool tall;      // the rows of T in shared memory (k_mul_quad_tc_tall, ma16 <= 64)
    uint32_t dw;    // D slot width: 32 or 64 (tall), 128 (tw)
    uint32_t x1_off, t_off, t_bytes;
};

constexpr uint32_t kSmemMax = 227 * 1024;  // dynamic shared memory per CTA (opt-in)

// k_mul_quad_tc_tall's layout: two XX buffers, three T buffers (one group of
// steps each), the normalisation's staging row and spill words, a's words of
// the next product, two copies of b's bytes, the flags and the mbarriers.
void tall_geometry(TcGeometry &q, uint32_t nout) {
    q.tall = true;
    q.tw = false;
    q.dw = q.ma16 <= 32 ? 32 : 64;
    const uint32_t group = kTmemCols / q.dw / 2;
    const uint32_t xbytes = (16 * q.xs + 1023) & ~1023u;
    q.x1_off = xbytes;
    q.t_off = 2 * xbytes;
    q.t_bytes = ((kBlk * group + kTallLead) * kTallRowBytes + 1023) & ~1023u;
    uint32_t off = q.t_off + kTBufs * q.t_bytes;
    q.spill_off = off;  // staging row (stage_index(nout) words + 16 bytes), then 8 bytes per normalising thread
    off += ((4 * (nout + (nout >> 4)) + 16 + 15) & ~15u) + 8 * 32 * kProdWarps;
    q.ca_off = off;  // a's words of the next product: 32 per block, zero from na on
    off += 128 * q.ma;
    q.cb_off = 0;
    q.braw_off = off;
    off += 2 * 4 * (32 * (q.mb + 2) + 4);
    off = (off + 15) & ~15u;
    q.flags_off = off;
    off += 4 * kEpiWarps;
    q.bar_off = (off + 15) & ~15u;
    q.smem = q.bar_off + 8 * (2 * kTBufs + 12) + 16;  // mbarriers, then the tensor-memory slot and abort flag
    if (q.smem < kMinSmem) q.smem = kMinSmem;  // one CTA per SM: each takes all of tensor memory
    q.w_off = 0;
}

TcGeometry geometry(uint32_t na, uint32_t nb) {
    TcGeometry q{};
    q.swap = na < nb;
    q.na = q.swap ? nb : na;
    q.nb = q.swap ? na : nb;
    q.ma = (q.na + 31) / 32;
    q.mb = (q.nb + 31) / 32;
    q.ma16 = (q.ma + 15) & ~15u;
    q.tw = q.ma16 <= 128;
    q.dw = q.ma16 <= 64 ? 64 : 128;
    q.xs = (2 * q.ma + (q.ma16 - q.ma)) * 16;
    const uint32_t nout = q.na + q.nb;
    const uint32_t stage_bytes = 4 * ((nout - 1) + ((nout - 1) >> 4) + 1);
    if (q.ma16 <= 64) {
        tall_geometry(q, nout);
        return q;
    }
    q.w_off = 16 * q.xs;  // a multiple of 256
    uint32_t off;
    if (q.tw) {  // no W in shared memory; the spill words after the staging row
        off = q.w_off > stage_bytes ? q.w_off : stage_bytes;
        off = (off + 15) & ~15u;
        q.spill_off = off;
        off += 8 * kThreadsTw;
    } else {
        q.spill_off = q.w_off;  // the normalisation's spill words reuse the T slots
        off = q.w_off + 2 * kTSlotBytes;
        if (off < stage_bytes) off = stage_bytes;
    }
    off = (off + 15) & ~15u;
    q.ca_off = off;
    off += kBiasBytes;
    q.cb_off = off;
    off += kBiasBytes;
    q.braw_off = off;
    off += 4 * (32 * (q.mb + 2) + 4);
    off = (off + 15) & ~15u;
    q.flags_off = off;
    off += 4 * (kThreads / 32);  // at least one word per warp of either kernel
    q.bar_off = (off + 15) & ~15u;
    off = q.bar_off + 8 * (2 * kWSlotsMax + 2 * kDSlotsMax) + 16;
    q.smem = off > kMinSmem ? off : kMinSmem;
    return q;
}

}  // namespace

BN_DEBUG_ACCESSOR(debug_word_quad_tc)

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
    if (p->geo.smem > kSmemMax) {
        delete p;
        return BN_EUNSUPPORTED;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = allow_max_smem((const void *)k_mul_quad_tc);
    if (e == cudaSuccess) e = allow_max_smem((const void *)k_mul_quad_tc_tw);
    if (e == cudaSuccess) e = allow_max_smem((const void *)k_mul_quad_tc_tall<32>);
    if (e == cudaSuccess) e = allow_max_smem((const void *)k_mul_quad_tc_tall<64>);
    if (e != cudaSuccess) {
        delete p;
        return BN_ECUDA;
    }
    p->ctas = (uint32_t)sms;
    // column sums per CTA: one row, or two for k_mul_quad_tc_tall (one product's
    // sums are carried into limbs while the next product's accumulate)
    p->stride = (uint64_t)kBlk * (p->geo.ma + p->geo.mb) * (p->geo.tall ? 2 : 1);
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
    g.ma16 = q.ma16;
    g.batch = batch;
    g.scratch = p->scratch;
    g.scratch_stride = p->stride;
    g.xs = q.xs;
    g.w_off = q.w_off;
    g.ca_off = q.ca_off;
    g.cb_off = q.cb_off;
    g.braw_off = q.braw_off;
    g.spill_off = q.spill_off;
    g.flags_off = q.flags_off;
    g.bar_off = q.bar_off;
    g.x1_off = q.x1_off;
    g.t_off = q.t_off;
    g.t_bytes = q.t_bytes;
    const uint32_t grid = batch < p->ctas ? (uint32_t)batch : p->ctas;
    if (q.tall && q.dw == 32)
        k_mul_quad_tc_tall<32><<<grid, threads_tall<32>(), q.smem, st>>>(g);
    else if (q.tall)
        k_mul_quad_tc_tall<64><<<grid, threads_tall<64>(), q.smem, st>>>(g);
    else if (q.tw)
        k_mul_quad_tc_tw<<<grid, kThreadsTw, q.smem, st>>>(g);
    else
        k_mul_quad_tc<<<grid, kThreads, q.smem, st>>>(g);
    return cudaGetLastError();
}

namespace {

// The bounded-wait machinery on its own: warp 0 waits for an mbarrier that
// nobody arrives on, gives up after limit_ns and raises the abort flag; warp 1
// waits on it with a 10 s limit but watches the abort flag, so it gives up as
// soon as warp 0 does.  Either giving up raises the device flag.
__global__ void k_tc_wait_selftest(uint64_t limit_ns) {
    __shared__ uint64_t bar;
    __shared__ uint32_t abortf;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        abortf = 0;
        tc::fence_mbar_init();
    }
    __syncthreads();
    const bool w0 = threadIdx.x < 32;
    const bool ok = tc::mbar_wait(&bar, 0, w0 ? limit_ns : 10000000000ull, &abortf);
    if (!__all_sync(FULL_MASK, ok)) {
        if (w0) *(volatile uint32_t *)&abortf = 1;
        if ((threadIdx.x & 31) == 0) atomicOr(&g_tc_fault, 1u);
    }
}

}  // namespace

cudaError_t tc_wait_selftest(uint32_t limit_us) {
    k_tc_wait_selftest<<<1, 64>>>(1000ull * limit_us);
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
