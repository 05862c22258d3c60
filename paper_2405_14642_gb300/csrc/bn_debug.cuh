// Checks compiled into the debug build only (-DBN_DEBUG).  A failed check
// sets bits in an error word of its translation unit (atomicOr, never a
// trap), read and cleared from the host through bn_debug_word() (api.cu).
// Checks cover what a correct kernel must never see: words of a product at
// or beyond na + nb that are not zero (the exact product has na + nb limbs,
// Section 3.2, Fig. 5), a carry leaving the product, and shared-memory
// indices outside the region they address.  In the regular build every check
// compiles to nothing.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace bn {

enum DebugBits : uint32_t {
    kDbgSpill = 1u,   // a word or carry beyond the product's length is not zero
    kDbgIndex = 2u,   // a shared-memory index outside its region
};

}  // namespace bn

#ifdef BN_DEBUG
// One error word per translation unit; BN_DEBUG_ACCESSOR(name) defines the
// host function name() that returns and clears this unit's word.
static __device__ uint32_t g_bn_debug_word;
#define BN_DEBUG_CHECK(cond, bit) \
    do {                          \
        if (!(cond)) atomicOr(&g_bn_debug_word, (uint32_t)(bit)); \
    } while (0)
#define BN_DEBUG_ACCESSOR(name)                                              \
    uint32_t name() {                                                        \
        uint32_t v = 0, z = 0;                                               \
        if (cudaMemcpyFromSymbol(&v, g_bn_debug_word, sizeof v) != cudaSuccess) return ~0u; \
        cudaMemcpyToSymbol(g_bn_debug_word, &z, sizeof z);                   \
        return v;                                                            \
    }
#else
#define BN_DEBUG_CHECK(cond, bit) \
    do {                          \
    } while (0)
#define BN_DEBUG_ACCESSOR(name) \
    uint32_t name() { return 0; }
#endif
