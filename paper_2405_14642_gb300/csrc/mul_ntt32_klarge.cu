// Three-prime transform kernels for log2 N = 13 .. 14 (see ntt3_device.cuh);
// the lengths are split over several files so that they compile in parallel.
#include "ntt3_device.cuh"

namespace bn {

BN_DEBUG_ACCESSOR(debug_word_ntt3_large)

ntt3::Kernels3 ntt3_kernels_large(uint32_t log_n) {
    switch (log_n) {
    case 13: return ntt3::kernels3<13>();
    case 14: return ntt3::kernels3<14>();
    default: return {nullptr, nullptr};
    }
}

}  // namespace bn
