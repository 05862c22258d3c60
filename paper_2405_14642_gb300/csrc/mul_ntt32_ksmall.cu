// Three-prime transform kernels for log2 N = 1 .. 10 (see ntt3_device.cuh);
// the lengths are split over several files so that they compile in parallel.
#include "ntt3_device.cuh"

namespace bn {

BN_DEBUG_ACCESSOR(debug_word_ntt3_small)

ntt3::Kernels3 ntt3_kernels_small(uint32_t log_n) {
    switch (log_n) {
    case 1: return ntt3::kernels3<1>();
    case 2: return ntt3::kernels3<2>();
    case 3: return ntt3::kernels3<3>();
    case 4: return ntt3::kernels3<4>();
    case 5: return ntt3::kernels3<5>();
    case 6: return ntt3::kernels3<6>();
    case 7: return ntt3::kernels3<7>();
    case 8: return ntt3::kernels3<8>();
    case 9: return ntt3::kernels3<9>();
    case 10: return ntt3::kernels3<10>();
    default: return {nullptr, nullptr};
    }
}

}  // namespace bn
