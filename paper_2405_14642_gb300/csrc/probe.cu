// Register-only integer multiply-add throughput probe (include/bn_probe.h).
#include <cuda_runtime.h>

#include "../../include/bn_probe.h"

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
