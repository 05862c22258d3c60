// Throughput probes (include/bn_probe.h): register-only integer multiply-adds,
// and chains of small tensor-core MMAs.
#include <cuda_runtime.h>

#include "../../include/bn_probe.h"
#include "tc_device.cuh"

namespace {

template <int KIND>
__global__ void __launch_bounds__(1024) k_probe(uint32_t iters, uint32_t *out) {
    uint32_t x[8];
    const uint32_t seed = threadIdx.x * 0x9E3779B9u + blockIdx.x;
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = seed + 0x01000193u * k;
    const uint32_t y = seed | 1u, z = seed ^ 0x5bd1e995u;
    if constexpr (KIND == 0 || KIND == 1) {
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (KIND == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(y), "r"(z));
                else asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(y), "r"(z));
            }
        }
    } else if constexpr (KIND == 2) {
        uint64_t w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = x[k];
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[k]) : "r"((uint32_t)w[k]), "r"(y));
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = (uint32_t)w[k] ^ (uint32_t)(w[k] >> 32);
    } else {
        uint32_t acc[2][10];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 10; ++k) acc[j][k] = seed + j * 10 + k;
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint32_t a = y + i + j;
                asm volatile(
                    "mad.lo.cc.u32  %0, %10, %11, %0;\n\t"
                    "madc.lo.cc.u32 %1, %10, %12, %1;\n\t"
                    "madc.lo.cc.u32 %2, %10, %13, %2;\n\t"
                    "madc.lo.cc.u32 %3, %10, %14, %3;\n\t"
                    "madc.lo.cc.u32 %4, %10, %15, %4;\n\t"
                    "madc.lo.cc.u32 %5, %10, %16, %5;\n\t"
                    "madc.lo.cc.u32 %6, %10, %17, %6;\n\t"
                    "madc.lo.cc.u32 %7, %10, %18, %7;\n\t"
                    "addc.cc.u32    %8, %8, 0;\n\t"
                    "addc.u32       %9, %9, 0;\n\t"
                    "mad.hi.cc.u32  %1, %10, %11, %1;\n\t"
                    "madc.hi.cc.u32 %2, %10, %12, %2;\n\t"
                    "madc.hi.cc.u32 %3, %10, %13, %3;\n\t"
                    "madc.hi.cc.u32 %4, %10, %14, %4;\n\t"
                    "madc.hi.cc.u32 %5, %10, %15, %5;\n\t"
                    "madc.hi.cc.u32 %6, %10, %16, %6;\n\t"
                    "madc.hi.cc.u32 %7, %10, %17, %7;\n\t"
                    "madc.hi.cc.u32 %8, %10, %18, %8;\n\t"
                    "addc.u32       %9, %9, 0;"
                    : "+r"(acc[j][0]), "+r"(acc[j][1]), "+r"(acc[j][2]), "+r"(acc[j][3]),
                      "+r"(acc[j][4]), "+r"(acc[j][5]), "+r"(acc[j][6]), "+r"(acc[j][7]),
                      "+r"(acc[j][8]), "+r"(acc[j][9])
                    : "r"(a), "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]),
                      "r"(x[6]), "r"(x[7]));
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] ^= acc[0][k] + acc[1][k + 2];
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s ^= x[k];
    // One word per block; a reduction keeps the result live.
    s = __reduce_xor_sync(0xffffffffu, s);
    if ((threadIdx.x & 31) == 0) atomicXor(out + blockIdx.x, s);
}


// One CTA per SM; one elected thread of warp 0 issues `iters` MMAs of
// kind::f16, M = 128, K = 16, N = n over `chains` accumulators of n columns
// (MMA i goes to accumulator i % chains and restarts it, accumulate = 0,
// every chain_len MMAs of that accumulator), A and B from shared memory
// windows that move with every MMA as the tensor-core schoolbook's do (A: a
// 128-row window of a tall K-major matrix stepping 512 bytes; B: an n-row
// window stepping 16 bytes with a 1 KB K-chunk stride).  The operands are
// zero: only the time matters.  One commit at the end; the wait for it is
// bounded, and a timeout sets *status.
constexpr uint32_t kProbeA = 98304, kProbeB = 32768, kProbeSmem = kProbeA + kProbeB + 128;

__global__ void __launch_bounds__(128, 1) k_probe_mma(uint32_t n, uint32_t chains, uint32_t chain_len,
                                                      uint32_t iters, uint32_t ncols, uint32_t *status) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kProbeA + kProbeB);
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + kProbeA + kProbeB + 64);
    for (uint32_t i = threadIdx.x; i < (kProbeA + kProbeB) / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    const uint32_t warp = threadIdx.x >> 5;
    if (warp == 0) bn::tc::tmem_alloc(slot, ncols);
    if (threadIdx.x == 0) {
        bn::tc::mbar_init(bar, 1);
        bn::tc::fence_mbar_init();
    }
    bn::tc::fence_proxy_async();
    bn::tc::fence_before_sync();
    __syncthreads();
    bn::tc::fence_after_sync();
    const uint32_t taddr = *slot;
    if (warp == 0) {
        if (bn::tc::elect_one()) {
            const uint32_t s0 = bn::tc::smem_u32(sm);
            const uint64_t ad = bn::tc::smem_desc(s0, 128, 256), bd = bn::tc::smem_desc(s0 + kProbeA, 1024, 128);
            const uint32_t idesc = bn::tc::idesc_f16_f32(128, n);
            // counters stepped without divisions, so that issuing stays well ahead of the pipe:
            // A window ia of 185 positions x 512 bytes (the last ends at 94208 + 4096 = kProbeA),
            // B window ib of 32 positions x 16 bytes (n <= 256 rows: 4 KB per K-chunk, ends below
            // kProbeB), accumulator c, and r = this MMA's place in its chain
            uint32_t c = 0, r = 0, ia = 0, ib = 0;
            for (uint32_t i = 0; i < iters; ++i) {
                bn::tc::mma_f16_ss(taddr + n * c, ad + 32 * ia, bd + ib, idesc, r != 0);
                ia = ia == 184 ? 0 : ia + 1;
                ib = (ib + 1) & 31;
                if (++c == chains) {
                    c = 0;
                    r = r + 1 == chain_len ? 0 : r + 1;
                }
            }
            bn::tc::mma_commit(bar);
            if (!bn::tc::mbar_wait(bar, 0, 2000000000ull)) {
                atomicExch(status, 1u);
                bn::tc::mbar_wait(bar, 0, 2000000000ull);  // the MMAs in flight, bounded again
            }
        }
        __syncwarp();
    }
    bn::tc::fence_before_sync();
    __syncthreads();
    bn::tc::fence_after_sync();
    if (warp == 0) bn::tc::tmem_dealloc(taddr, ncols);
}
}  // namespace

extern "C" bn_status bn_probe_int_throughput(int kind, uint32_t blocks, uint32_t threads,
                                             uint32_t iters, uint32_t *out,
                                             uint64_t *ops_per_thread, void *stream) {
    if (!out || !ops_per_thread || blocks == 0 || threads == 0 || threads > 1024 || threads % 32)
        return BN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    switch (kind) {
    case BN_PROBE_MAD_LO: k_probe<0><<<blocks, threads, 0, st>>>(iters, out); break;
    case BN_PROBE_MAD_HI: k_probe<1><<<blocks, threads, 0, st>>>(iters, out); break;
    case BN_PROBE_MAD_WIDE: k_probe<2><<<blocks, threads, 0, st>>>(iters, out); break;
    case BN_PROBE_MAC_CHAIN: k_probe<3><<<blocks, threads, 0, st>>>(iters, out); break;
    default: return BN_EINVAL;
    }
    *ops_per_thread = (uint64_t)iters * (kind == BN_PROBE_MAC_CHAIN ? 32u : 8u);
    return cudaGetLastError() == cudaSuccess ? BN_OK : BN_ECUDA;
}

extern "C" bn_status bn_probe_mma_throughput(uint32_t n, uint32_t chains, uint32_t chain_len, uint32_t iters,
                                             uint32_t ctas, uint32_t *status, void *stream) {
    if (!status || ctas == 0 || iters == 0 || chains == 0 || chain_len == 0) return BN_EINVAL;
    if (n < 16 || n > 256 || n % 16 || n * chains > 512) return BN_EINVAL;
    uint32_t ncols = 32;
    while (ncols < n * chains) ncols <<= 1;
    if (cudaFuncSetAttribute(k_probe_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeSmem) != cudaSuccess)
        return BN_ECUDA;
    k_probe_mma<<<ctas, 128, kProbeSmem, (cudaStream_t)stream>>>(n, chains, chain_len, iters, ncols, status);
    return cudaGetLastError() == cudaSuccess ? BN_OK : BN_ECUDA;
}
