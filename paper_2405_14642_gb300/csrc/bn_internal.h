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

// Debug build (-DBN_DEBUG): each kernel translation unit's check bits, read
// and cleared (bn_debug.cuh); 0 in the regular build.
uint32_t debug_word_quad();
uint32_t debug_word_quad_tc();
uint32_t debug_word_ntt();
uint32_t debug_word_ntt3_small();
uint32_t debug_word_ntt3_mid();
uint32_t debug_word_ntt3_large();

// ---- mixed-size batches ----------------------------------------------------
// One operation of a batch: operands at the given limb offsets of the flat
// a and b buffers, result at off_c of the flat c buffer.
struct BatchItem {
    uint64_t off_a, off_b, off_c;
    uint32_t na, nb;
};
// Base pointers of the flat buffers, read by the batched kernels from device
// memory so a captured graph can run on new buffers.
struct BatchBinding {
    const uint32_t *a, *b;
    uint32_t *c;
};

// ---- cost model (cost_model.cu) -------------------------------------------
double default_quad_rate(uint32_t key);              // word products / us
double default_ntt_us(bool crt, uint32_t log_n);     // us per product
struct MulChoice {
    uint32_t kind = 1;  // 1 schoolbook, 2 one-prime, 3 two-prime, 4 three-prime transform
    uint32_t quad_key = 0, log_n64 = 0, log_ncrt = 0;  // log_ncrt is also the three-prime length
    double est_us = 0;
};
double default_ntt3_us(uint32_t log_n);               // us per product, three 32-bit primes
MulChoice choose_mul(uint32_t na, uint32_t nb);

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

// Batched additions of one size class (both operands <= n_max limbs).
struct AddClass {
    uint32_t n_max = 0, rows = 1, warps_per_team = 1, teams_per_cta = 1, block = 32;
};
bn_status add_batch_class(AddClass &ac, uint32_t n_max);
cudaError_t add_batch_launch(const AddClass &ac, const BatchItem *items, uint32_t count,
                             const BatchBinding *bind, cudaStream_t stream);

// ---- quadratic multiplication (Section 3) ---------------------------------
struct QuadConfig {
    uint32_t na = 0, nb = 0, nout = 0;
    uint32_t q = 0;        // result limbs per window
    bool cols = false;     // per-column 64-bit sums instead of carry chains
    bool lane = false;     // one product per thread (operands up to 128 limbs)
    bool lane_auto = false;  // the lane form for batches of at least a warp per SM
    uint32_t threads = 0;  // threads per instance group
    uint32_t cta_threads = 0;
};
bn_status quad_configure(QuadConfig &cfg, uint32_t na, uint32_t nb, const bn_tuning *t);
cudaError_t quad_launch(const QuadConfig &cfg, const uint32_t *a, const uint32_t *b, uint32_t *c,
                        uint64_t batch, cudaStream_t stream);

// Batched schoolbook products of one size class (longer operand <= n_max):
// a persistent kernel whose CTAs take `ipb` items at a time from a work queue.
struct QuadClass {
    uint32_t q = 8, n_max = 0;
    uint32_t group = 0, ipb = 0, block = 0, inst_words = 0, smem = 0, grid = 0;
};
bn_status quad_batch_class(QuadClass &qc, uint32_t q, uint32_t n_max, uint32_t cta_target);
cudaError_t quad_batch_launch(const QuadClass &qc, const BatchItem *items, uint32_t count,
                              uint32_t *queue, const BatchBinding *bind, cudaStream_t stream);

// ---- NTT multiplication (Section 4) ---------------------------------------
struct NttPlan;  // opaque; defined in mul_ntt.cu
bn_status ntt_create(NttPlan **out, bool crt, uint32_t na, uint32_t nb, const bn_tuning *t);
void ntt_destroy(NttPlan *p);
cudaError_t ntt_launch(NttPlan *p, const uint32_t *a, const uint32_t *b, uint32_t *c,
                       uint64_t batch, cudaStream_t stream);
size_t ntt_scratch_bytes(const NttPlan *p);
// Plan for a mixed-size batch class: transform length exactly N; the batched
// kernel takes each item's sizes from its descriptor (digits(a)+digits(b) must
// lie in (N/2, N]).
bn_status ntt_batch_plan(NttPlan **out, bool crt, uint32_t N);
cudaError_t ntt_batch_launch(NttPlan *p, const BatchItem *items, uint32_t count, uint32_t *queue,
                             const BatchBinding *bind, cudaStream_t stream);
// One product of na x nb limbs with the tables of plan p (same transform length).
cudaError_t ntt_launch_sized(NttPlan *p, uint32_t na, uint32_t nb, const uint32_t *a,
                             const uint32_t *b, uint32_t *c, cudaStream_t stream);
uint32_t ntt_length(const NttPlan *p);

// Three 32-bit primes (mul_ntt32.cu).
struct Ntt3Plan;  // opaque
bn_status ntt3_create(Ntt3Plan **out, uint32_t na, uint32_t nb, const bn_tuning *t);
void ntt3_destroy(Ntt3Plan *p);
cudaError_t ntt3_launch(Ntt3Plan *p, const uint32_t *a, const uint32_t *b, uint32_t *c, uint64_t batch,
                        cudaStream_t st);
size_t ntt3_scratch_bytes(const Ntt3Plan *p);
uint32_t ntt3_length(const Ntt3Plan *p);
// Batch form: a plan of transform length exactly N (items with na + nb <= N).
bn_status ntt3_batch_plan(Ntt3Plan **out, uint32_t N);
cudaError_t ntt3_batch_launch(Ntt3Plan *p, const BatchItem *items, uint32_t count, uint32_t *queue,
                              const BatchBinding *bind, cudaStream_t st);
cudaError_t ntt3_launch_sized(Ntt3Plan *p, uint32_t na, uint32_t nb, const uint32_t *a, const uint32_t *b,
                              uint32_t *c, cudaStream_t st);

// Schoolbook product on the tensor cores (mul_quad_tc.cu).
struct QuadTcPlan;  // opaque
bn_status quad_tc_create(QuadTcPlan **out, uint32_t na, uint32_t nb);
void quad_tc_destroy(QuadTcPlan *p);
cudaError_t quad_tc_launch(QuadTcPlan *p, const uint32_t *a, const uint32_t *b, uint32_t *c, uint64_t batch,
                           cudaStream_t st);
size_t quad_tc_scratch_bytes(const QuadTcPlan *p);
// Reads and clears the tensor-core kernels' timeout flag (synchronises the device).
cudaError_t tc_fault_take(uint32_t *flag);
// One launch whose mbarrier wait must time out after limit_us (raises the flag).
cudaError_t tc_wait_selftest(uint32_t limit_us);

}  // namespace bn
