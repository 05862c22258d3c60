// Internal host-side interface between the C ABI (api.cu) and the kernel
// translation units.  Not installed; the public interface is include/bn.h.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/bn.h"

namespace bn {

// Raises a kernel's dynamic shared-memory cap to the device's opt-in maximum,
// once per (kernel, device).  The cap is a property of the function, so
// lowering it for one plan would break larger plans of the same kernel.
cudaError_t allow_max_smem(const void *kernel);

// Records `what` as this host thread's bn_last_error() text.
void record_error(const char *what);

// ---- addition (Section 2) -------------------------------------------------
struct AddConfig {
    uint32_t na = 0, nb = 0, n = 0, nout = 0;
    uint32_t limbs_per_thread = 0;  // requested (0 = default)
    uint32_t cta_threads = 0;       // requested (0 = default)
};
// Validates tuning against the size; BN_OK or BN_EINVAL/BN_EUNSUPPORTED.
bn_status add_configure(AddConfig &cfg, uint32_t na, uint32_t nb, const bn_tuning *t);
cudaError_t add_launch(const AddConfig &cfg, const uint32_t *a, const uint32_t *b, uint32_t *c,
                       uint64_t batch, cudaStream_t stream);
// Number of kernel launches one add_launch issues (for launch accounting).
inline int add_launch_count() { return 1; }

// ---- quadratic multiplication (Section 3) ---------------------------------
struct QuadConfig {
    uint32_t na = 0, nb = 0, nout = 0;
    uint32_t q = 0;        // result limbs per window
    bool cols = false;     // per-column 64-bit sums instead of carry chains
    uint32_t threads = 0;  // threads per instance group
    uint32_t cta_threads = 0;
};
bn_status quad_configure(QuadConfig &cfg, uint32_t na, uint32_t nb, const bn_tuning *t);
cudaError_t quad_launch(const QuadConfig &cfg, const uint32_t *a, const uint32_t *b, uint32_t *c,
                        uint64_t batch, cudaStream_t stream);

// ---- NTT multiplication (Section 4) ---------------------------------------
struct NttPlan;  // opaque; defined in mul_ntt.cu
bn_status ntt_create(NttPlan **out, bool crt, uint32_t na, uint32_t nb, const bn_tuning *t);
void ntt_destroy(NttPlan *p);
cudaError_t ntt_launch(NttPlan *p, const uint32_t *a, const uint32_t *b, uint32_t *c,
                       uint64_t batch, cudaStream_t stream);
size_t ntt_scratch_bytes(const NttPlan *p);
uint32_t ntt_length(const NttPlan *p);

}  // namespace bn
