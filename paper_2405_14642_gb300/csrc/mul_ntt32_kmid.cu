// Three-prime transform kernels for log2 N = 11 .. 12 (see ntt3_device.cuh);
// the lengths are split over several files so that they compile in parallel.
#include "ntt3_device.cuh"

namespace bn {

BN_DEBUG_ACCESSOR(debug_word_ntt3_mid)

ntt3::Kernels3 ntt3_kernels_mid(uint32_t log_n) {
    switch (log_n) {
    case 11: return ntt3::kernels3<11>();
    case 12: return ntt3::kernels3<12>();
    default: return {nullptr, nullptr};
    }
}

}  // namespace bn
