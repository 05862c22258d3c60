/*
 * bn.h - batched exact addition and multiplication of midsize unsigned
 * integers (1K to about 256K bits) on one NVIDIA GB300 (sm_103a) GPU.
 *
 * Method: Oancea & Watt, "GPU Implementations for Midsize Integer Addition
 * and Multiplication" (arXiv 2405.14642).  Each integer is handled by one CTA
 * (or by part of a CTA for small sizes), as in the paper.
 *
 * Representation (Section 2): an integer is an array of little-endian u32
 * limbs, a = a_0 + a_1 x + ... + a_{n-1} x^{n-1} with x = 2^32.  A batch of
 * `batch` integers of n limbs is one contiguous array: instance i starts at
 * limb i*n.  Results are full width (the paper keeps the input length; its
 * result is the low limbs of the result here):
 *     add: max(na, nb) + 1 limbs      mul: na + nb limbs
 * The shorter operand of an addition is zero-extended.
 *
 * Ownership and memory: every a/b/c pointer of the device entry points is
 * caller-owned DEVICE memory that stays valid until the enqueued work has
 * finished.  Plans own their tables and scratch until bn_plan_destroy.
 * c must not overlap a or b (BN_EINVAL).  No alignment is required; 16-byte
 * aligned rows (base 16-byte aligned and a limb count that is a multiple of 4)
 * take the vectorised load path.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Device entry points only enqueue work and return; results
 * are ready when the stream reaches that point.  Errors from the work itself
 * surface as BN_ECUDA on a later call or on stream synchronisation.
 *
 * Errors: every entry point returns a bn_status and throws nothing.  On
 * BN_ECUDA the CUDA error text is available from bn_last_error().
 * batch == 0 is a no-op returning BN_OK (pointers are not checked then).
 *
 * Thread safety: distinct plans may be used from different host threads.  One
 * plan must not be executed concurrently from two host threads.  The one-shot
 * forms keep an internal, mutex-protected cache of plans per size.
 */
#ifndef BN_GB300_H
#define BN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bn_status {
    BN_OK = 0,
    BN_EINVAL = 1,        /* null pointer, zero size, overlap, bad option */
    BN_ENOMEM = 2,        /* a device or host allocation failed */
    BN_ECUDA = 3,         /* a CUDA runtime call or launch failed */
    BN_EUNSUPPORTED = 4,  /* size outside what the variant holds */
    BN_ETIMEOUT = 5       /* a bounded device-side wait gave up */
} bn_status;

typedef enum bn_op {
    /* Section 2: three-step addition, carries by an exclusive scan with the
     * carry operator (here a warp-ballot carry-lookahead plus a cross-warp
     * step through shared memory).  na, nb <= BN_ADD_MAX_LIMBS. */
    BN_OP_ADD = 0,
    /* Section 3: classical product, Eq. (1), each thread owning whole result
     * windows under the load-balanced partition of Fig. 3 (extended to full,
     * unequal-length products), per-thread windows recombined by the L/H
     * addition of Fig. 4/5.  na, nb <= BN_MUL_MAX_LIMBS. */
    BN_OP_MUL_QUAD = 1,
    /* Section 4: product through a number-theoretic transform over the
     * prime field PrimeField64 (p = 29*2^57 + 1, Section 4.1) with 16-bit
     * digits, transform length the next power of two >= 2(na + nb). */
    BN_OP_MUL_NTT64 = 2,
    /* Section 4 with 32-bit digits over two primes (29*2^57 + 1 and
     * 27*2^56 + 1), recombined by the Chinese remainder theorem. */
    BN_OP_MUL_NTT_CRT = 3,
    /* Multiplication by whichever of the schoolbook and transform products
     * (BN_OP_MUL_NTT3 included) the cost model finds fastest for the sizes:
     * per item in a mixed-size batch; for a plan (and bn_mul) once, at
     * creation (bn_plan_op reports the choice; tuning applies only when the
     * choice is the schoolbook product). */
    BN_OP_MUL_AUTO = 4,
    /* Section 4's transform product over three 32-bit good primes
     * (7*2^26 + 1, 45*2^24 + 1, 119*2^23 + 1; roots by the Section 4.1
     * search) with 32-bit digits, recombined by Garner's mixed-radix CRT
     * (coefficients < 2^78 < the primes' product).  Transform length the next
     * power of two >= na + nb, at most 16384 (na + nb <= 16384).  Field
     * elements are single 32-bit words.  Plans and one-shot calls only (not a
     * batch item op). */
    BN_OP_MUL_NTT3 = 5,
    /* Section 3's classical product (every word product, summed by column,
     * Eq. (1)) computed one level down on bytes as an exact contraction on
     * the tensor cores: fp16 byte digits, f32 sums of at most 128 byte
     * products (below 2^23, exact), per-thread integer column sums, then the
     * normalisation into limbs with the Section 2 carry scan.  Operands cut
     * into 128-byte blocks; per block J of the shorter operand one MMA chain
     * of M = 128, K = 128 against all blocks of the longer one.
     * na, nb <= BN_MUL_MAX_LIMBS; no tuning fields.  Plans and one-shot
     * calls only (not a batch item op). */
    BN_OP_MUL_QUAD_TC = 6
} bn_op;

/* Largest limb counts per operand (256K bits for the products, 512K bits for
 * the sum). */
#define BN_ADD_MAX_LIMBS 16384u
#define BN_MUL_MAX_LIMBS 8192u

/* Optional launch tuning; a zero field takes the built-in default. */
typedef struct bn_tuning {
    uint32_t limbs_per_thread;  /* add: limbs per thread (multiple of the vector width);
                                   quad: result limbs per window (4 or 8) */
    uint32_t cta_threads;       /* threads per CTA (multiple of 32, <= 1024); the three-prime
                                   transform's kernels are compiled for one count per
                                   length (N/8 within 32..1024) and refuse any other */
    uint32_t variant;           /* quad: 1 = carry-chain accumulation by thread groups,
                                   2 = per-column 64-bit sums with carry counts, 3 = one
                                   product per thread (operands up to 128 limbs, no
                                   other tuning field); 0 = 3 for operands up to 96
                                   limbs and batches of at least 4864, else 1;
                                   other ops: 0 */
    uint32_t reserved;          /* must be zero */
} bn_tuning;

typedef struct bn_plan_s *bn_plan;

/* Create a plan for `batch` instances of an na-limb by nb-limb operation.
 * NTT plans build their twiddle tables and device scratch here (the only
 * place the library allocates device memory besides the host-buffer staging
 * of bn_plan_execute_host).  tuning may be NULL.
 * Errors: BN_EINVAL (null out, zero size, bad tuning), BN_EUNSUPPORTED (size
 * above the op's limit), BN_ENOMEM, BN_ECUDA. */
bn_status bn_plan_create(bn_plan *out, bn_op op, uint32_t na, uint32_t nb,
                         uint64_t batch, const bn_tuning *tuning);

/* Enqueue the plan on `stream` over device arrays a (batch x na), b (batch x nb)
 * and c (batch x bn_plan_out_limbs).  Errors: BN_EINVAL, BN_ECUDA. */
bn_status bn_plan_execute(bn_plan plan, const uint32_t *a, const uint32_t *b,
                          uint32_t *c, void *stream);

/* Same over HOST arrays: copies a and b to plan-owned device staging buffers
 * (allocated on first use), runs the plan, copies c back and synchronises
 * `stream` before returning, so c is filled on BN_OK.  Pinned host memory
 * makes the copies asynchronous and faster; pageable memory also works. */
bn_status bn_plan_execute_host(bn_plan plan, const uint32_t *a, const uint32_t *b,
                               uint32_t *c, void *stream);

/* Same copies and kernel, enqueued on `stream` without the final
 * synchronisation, so that the copies and kernels of several plans on
 * several streams overlap (the copy engines run beside the kernels).  a and b
 * must stay unchanged and c untouched until `stream` reaches the end of the
 * call; with pinned host memory the copies are asynchronous (pageable memory
 * makes them partly synchronous).  The plan's staging buffers are reused by
 * every call on the plan, so calls on one plan must be on one stream (or
 * otherwise ordered).  Errors as bn_plan_execute_host; errors of the queued
 * work surface on stream synchronisation. */
bn_status bn_plan_execute_host_async(bn_plan plan, const uint32_t *a, const uint32_t *b,
                                     uint32_t *c, void *stream);

/* Free the plan's device resources (synchronises the device first). */
bn_status bn_plan_destroy(bn_plan plan);

/* Result limbs per instance: max(na,nb)+1 for add, na+nb for products. */
uint32_t bn_plan_out_limbs(bn_plan plan);

/* The plan's concrete op (a BN_OP_MUL_AUTO plan reports the product it
 * chose); -1 for a null plan. */
int bn_plan_op(bn_plan plan);

/* Device scratch the plan holds (bytes; 0 for add and quad). */
size_t bn_plan_scratch_bytes(bn_plan plan);

/* Transform length N of an NTT plan (0 for other ops). */
uint32_t bn_plan_transform_length(bn_plan plan);

/* One-shot forms over device arrays: create (or reuse a cached) plan for the
 * size, enqueue on `stream`, return.  bn_mul_ntt: crt == 0 selects
 * BN_OP_MUL_NTT64, crt != 0 selects BN_OP_MUL_NTT_CRT. */
bn_status bn_add(const uint32_t *a, const uint32_t *b, uint32_t *c,
                 uint32_t na, uint32_t nb, uint64_t batch, void *stream);
bn_status bn_mul_quad(const uint32_t *a, const uint32_t *b, uint32_t *c,
                      uint32_t na, uint32_t nb, uint64_t batch, void *stream);
bn_status bn_mul_ntt(const uint32_t *a, const uint32_t *b, uint32_t *c,
                     uint32_t na, uint32_t nb, uint64_t batch, int crt, void *stream);
/* One-shot BN_OP_MUL_NTT3 (three 32-bit primes): same arguments, layout,
 * result (na + nb limbs) and errors as bn_mul_ntt. */
bn_status bn_mul_ntt3(const uint32_t *a, const uint32_t *b, uint32_t *c,
                      uint32_t na, uint32_t nb, uint64_t batch, void *stream);
/* One-shot BN_OP_MUL_QUAD_TC (schoolbook on the tensor cores): same
 * arguments, layout, ownership and errors as bn_mul_quad. */
bn_status bn_mul_quad_tc(const uint32_t *a, const uint32_t *b, uint32_t *c,
                         uint32_t na, uint32_t nb, uint64_t batch, void *stream);

/* Tensor-core kernels wait for their MMAs with a time limit (1 s per wait);
 * one that gives up skips the rest of its work, leaves its results
 * incomplete and raises a device flag.  This call synchronises the device,
 * reads and clears the flag: BN_ETIMEOUT if it was raised since the last
 * call, BN_ECUDA on a CUDA error, else BN_OK. */
bn_status bn_tc_check(void);

/* Diagnostic of the bounded waits above: launches one small kernel whose
 * mbarrier wait has no arrival coming, so it must give up after limit_us
 * microseconds (a second waiter watching the shared abort flag must give up
 * with it), and reads the device flag.  Returns BN_ETIMEOUT when the waits
 * gave up as designed (the flag is left clear), BN_OK if they did not,
 * BN_ECUDA on a CUDA error.  Synchronises the device. */
bn_status bn_tc_wait_selftest(uint32_t limit_us);

/* One-shot BN_OP_MUL_AUTO: c = a * b by the fastest product for the sizes
 * (schoolbook for small operands, the three-prime transform from about 8K
 * bits on GB300); arguments, layout, result and errors as bn_mul_quad. */
bn_status bn_mul(const uint32_t *a, const uint32_t *b, uint32_t *c,
                 uint32_t na, uint32_t nb, uint64_t batch, void *stream);

/* Transform multiplication that allocates nothing, for callers that cannot
 * call cudaMalloc: code whose device memory is wholly owned by another
 * allocator (a framework's memory pool, a fixed budget reserved at start-up)
 * and latency-sensitive loops that must not take cudaMalloc/cudaFree's
 * implicit device-wide synchronisation.  The paper has no counterpart.
 *
 * Same operation, arguments, layout and results as bn_mul_ntt (a, b, c are
 * caller-owned device memory; crt selects the two-prime form).  Instead of
 * plan-owned memory it uses two file-scope device arrays that every GPU which
 * loads the library holds until the process exits:
 *   scratch   BN_NOALLOC_SCRATCH_BYTES (32 MiB): the first prime's
 *             coefficients of two-prime products short enough to run on
 *             one CTA (longer transforms keep everything in shared memory);
 *             large enough for a full grid at every size, and
 *   tables    1.5 MiB of twiddle tables (Shoup pairs), regenerated on the
 *             device (on `stream`) whenever the transform length or field
 *             changes.
 * Operand sizes above BN_NOALLOC_MAX_LIMBS return BN_EUNSUPPORTED with a
 * bn_last_error() text saying so.  No call allocates host or device memory.
 *
 * The first call on a device sets that device up (looks up the arrays'
 * device addresses, raises the kernel's shared-memory cap), so make that
 * first call before any stream capture: a first call made while `stream` is
 * capturing returns BN_EINVAL.  Every call shares the arrays and they keep
 * the last call's contents (nothing in them has to start at zero: each call
 * writes every scratch and table word before reading it), so calls that
 * overlap on the GPU (different streams, other host threads) race and give
 * wrong results: serialise them on one stream.  Eager calls skip the table
 * kernel when the tables already hold their (field, length); a call made
 * while `stream` is capturing always records the table kernel, and after
 * the first such call every later call on that device regenerates its
 * tables too (a replay may have rewritten them).  The per-device set-up is
 * never redone: after cudaDeviceReset use a fresh process. */
#define BN_NOALLOC_SCRATCH_BYTES (32ull << 20)
#define BN_NOALLOC_MAX_LIMBS 8192u
bn_status bn_mul_ntt_noalloc(const uint32_t *a, const uint32_t *b, uint32_t *c,
                             uint32_t na, uint32_t nb, uint64_t batch, int crt, void *stream);

/* ---- same-length arithmetic and fused programs (Sections 2 and 6) ------
 * The paper's own benchmarks keep every result at the operands' length n,
 * i.e. compute modulo 2^(32 n) (Section 2), and Section 6 measures two
 * programs fused into one kernel each.  All three entry points take a, b, c
 * as row-major device arrays of batch x n u32 limbs (little-endian limb
 * order, instance i at offset i*n), write c only, and return once the kernel
 * is enqueued on `stream`.  c must not overlap a or b; a == b is allowed.
 * Errors: BN_EINVAL (n == 0, null pointer with batch > 0, overlap),
 * BN_EUNSUPPORTED (n > BN_MUL_MAX_LIMBS), BN_ECUDA (launch failure,
 * bn_last_error() has the CUDA text).  batch == 0 is a no-op.
 *
 * bn_mul_low  c = a*b mod 2^(32n): the schoolbook product restricted to its
 *             low n columns (Section 3, Fig. 3: the rising triangle, each
 *             thread taking a window and its mirror so all do equal work);
 *             half the word products of bn_mul_quad.
 * bn_poly     c = (a*a + b)*(b*b + b) + a*b mod 2^(32n) (Section 6's
 *             polynomial program): four low products and three additions in
 *             one kernel, every intermediate kept in shared memory.
 * bn_add6     six dependent additions x_{k+1} = x_k + x_{k-1} from x_0 = a,
 *             x_1 = b, c = x_7 = 8a + 13b mod 2^(32n) (Section 6's repeated
 *             addition program; the paper does not spell out the chain, this
 *             is the library's reading), intermediates in registers. */
bn_status bn_mul_low(const uint32_t *a, const uint32_t *b, uint32_t *c,
                     uint32_t n, uint64_t batch, void *stream);
bn_status bn_poly(const uint32_t *a, const uint32_t *b, uint32_t *c,
                  uint32_t n, uint64_t batch, void *stream);
bn_status bn_add6(const uint32_t *a, const uint32_t *b, uint32_t *c,
                  uint32_t n, uint64_t batch, void *stream);

/* ---- mixed-size batches ------------------------------------------------
 * Many independent operations of different sizes and kinds in one call.  The
 * paper evaluates one size per kernel launch (Section 6); this form runs a
 * whole mixed workload as one CUDA graph: items are grouped into size classes,
 * each class is one persistent kernel whose CTAs take items from a device
 * work queue (largest first), and the classes run concurrently.  A cost
 * model, calibrated at creation when BN_BATCH_AUTOTUNE is set (otherwise
 * built-in GB300 timings), picks the window size and CTA size of each
 * schoolbook class and, for BN_OP_MUL_AUTO items, schoolbook or transform.
 *
 * Layout: all a operands live in one flat u32 array, likewise b and c; item
 * i reads a[a_offset .. a_offset+na) and b[b_offset .. b_offset+nb) and
 * writes c[c_offset .. c_offset + out) with out = max(na,nb)+1 (add) or
 * na+nb (products).  Result ranges must not overlap each other or the
 * operands (not checked).  Sizes: 1..BN_ADD_MAX_LIMBS for add,
 * 1..BN_MUL_MAX_LIMBS for products.
 * bn_batch_create copies the item list, allocates device memory for it,
 * the work queues and the transform tables/scratch, and captures the graph
 * (on internal streams); it must not be called during stream capture.
 * bn_batch_execute binds the flat arrays and enqueues the graph on `stream`;
 * it must not overlap another execution of the same batch.
 * BN_BATCH_PLAIN executes the same item list as one ordinary launch per
 * item (same kernel choices, no graph).  BN_BATCH_PLAIN_CLASSES executes it
 * the way the paper's per-size launches would (Section 6 runs one size per
 * launch): per size class, in turn, a gather kernel copies the items'
 * operands into contiguous rows zero-padded to the class's largest sizes
 * (longer operand first for products), one ordinary batched launch of the
 * class's kernel computes all of them, and a scatter kernel copies each
 * item's result limbs back; three launches per class and device buffers for
 * the padded rows, allocated at creation.  Both are baselines the batched
 * form is measured against; they give bit-identical results and exclude
 * each other (BN_EINVAL). */
typedef struct bn_batch_item {
    uint32_t op;         /* bn_op */
    uint32_t na, nb;     /* limb counts */
    uint32_t reserved;   /* must be zero */
    uint64_t a_offset, b_offset, c_offset;  /* limb offsets into the flat arrays */
} bn_batch_item;

typedef struct bn_batch_info {
    uint32_t classes;        /* size classes (kernel launches in the graph) */
    uint32_t launches;       /* kernel launches per execution (plain: one per item) */
    uint64_t items_add, items_quad, items_ntt64, items_crt;  /* after BN_OP_MUL_AUTO */
    double tune_ms;          /* time spent calibrating at creation */
    uint64_t items_ntt3;     /* BN_OP_MUL_AUTO items on the three-prime transform */
} bn_batch_info;

typedef struct bn_batch_s *bn_batch;

#define BN_BATCH_AUTOTUNE 1u
#define BN_BATCH_PLAIN 2u
#define BN_BATCH_PLAIN_CLASSES 4u

bn_status bn_batch_create(bn_batch *out, const bn_batch_item *items, uint64_t count,
                          uint32_t flags);
bn_status bn_batch_execute(bn_batch batch, const uint32_t *a, const uint32_t *b, uint32_t *c,
                           void *stream);
bn_status bn_batch_get_info(bn_batch batch, bn_batch_info *info);
bn_status bn_batch_destroy(bn_batch batch);

/* ---- serving loop ---------------------------------------------------------
 * A request server for products (and sums) of mixed sizes whose operands are
 * already in device memory.  A scheduler thread owned by the server batches
 * requests continuously: whenever one of `max_inflight` slots is free it
 * admits pending requests in arrival order while their results fit in the
 * device result pool (first-fit, at most BN_SERVER_MAX_POOL bytes), groups
 * them into size classes (cost model as for batches) and launches the class
 * kernels on that slot's stream; requests that arrive meanwhile wait for the
 * next free slot, so their work overlaps the work already on the GPU.
 * BN_SERVER_SEQUENTIAL instead runs one request at a time with an ordinary
 * launch (the per-request baseline).  Results are bit-identical either way.
 *
 * Time: the server clock counts microseconds from creation
 * (bn_server_now_us); a request's arrival time is given at submission (or
 * taken from the clock if negative) and its completion time is when the
 * scheduler sees its micro-batch finish.
 * Memory: operands a, b stay caller-owned and must remain valid until the
 * request completes; results live in the pool until bn_server_release.
 * Transform tables and scratch (per slot) are allocated at creation, outside
 * the pool.  Threads: the submit/poll/release calls may come from any host
 * thread; the scheduler runs on its own thread. */
#define BN_SERVER_MAX_POOL (8ull << 30)
#define BN_SERVER_SEQUENTIAL 1u

typedef struct bn_server_config {
    uint64_t pool_bytes;      /* device result pool; 0 = 1 GiB; <= BN_SERVER_MAX_POOL */
    uint32_t max_inflight;    /* micro-batches on the GPU at once; 0 = 4 */
    uint32_t max_batch;       /* requests per micro-batch; 0 = 4096 */
    uint32_t flags;           /* BN_SERVER_SEQUENTIAL or 0 */
    uint32_t reserved;        /* must be zero */
} bn_server_config;

typedef struct bn_request {
    uint32_t op;              /* BN_OP_ADD or a multiplication op (BN_OP_MUL_AUTO recommended) */
    uint32_t na, nb;          /* limb counts (as for batch items) */
    uint32_t reserved;        /* must be zero */
    const uint32_t *a, *b;    /* device operands */
    double arrival_us;        /* server-clock arrival time; < 0 = now */
} bn_request;

typedef struct bn_completion {
    uint64_t ticket;
    uint32_t *c;              /* device result (pool memory) */
    uint32_t limbs;           /* result limbs */
    uint32_t reserved;
    double arrival_us, done_us;
} bn_completion;

typedef struct bn_server_stats {
    uint64_t submitted, completed, batches, pool_high_water;
    uint32_t max_inflight_seen, reserved;
} bn_server_stats;

typedef struct bn_server_s *bn_server;

bn_status bn_server_create(bn_server *out, const bn_server_config *cfg);
/* Enqueue `count` requests; tickets[i] receives request i's ticket.  Returns
 * immediately (BN_EINVAL for a bad request, none of the batch enqueued). */
bn_status bn_server_submit(bn_server s, const bn_request *reqs, uint32_t count, uint64_t *tickets);
/* Move up to `max` completions into out; *n receives how many. */
bn_status bn_server_poll(bn_server s, bn_completion *out, uint32_t max, uint32_t *n);
/* Free the result memory of `count` completed requests (unknown tickets are
 * skipped and reported as BN_EINVAL). */
bn_status bn_server_release(bn_server s, const uint64_t *tickets, uint32_t count);
/* Wait until nothing is pending or in flight (BN_ETIMEOUT after timeout_s). */
bn_status bn_server_drain(bn_server s, double timeout_s);
double bn_server_now_us(bn_server s);
bn_status bn_server_get_stats(bn_server s, bn_server_stats *out);
/* Stop the scheduler (after draining) and free everything. */
bn_status bn_server_destroy(bn_server s);

/* Static description of a status code. */
const char *bn_status_str(bn_status s);

/* Text of the last error recorded on this host thread ("" if none). */
const char *bn_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int bn_version(void);

/* ---- debug build -----------------------------------------------------------
 * The library also builds as a debug variant (compiled with BN_DEBUG) in
 * which the kernels check what a correct run never sees, without trapping:
 * a word of a product at or beyond na + nb that is not zero, or a carry
 * leaving the product (the exact product has na + nb limbs, Section 3.2,
 * Fig. 5; BN_DEBUG_SPILL), and a shared-memory index outside its region
 * (BN_DEBUG_INDEX).  Schoolbook, tensor-core schoolbook and transform
 * products are checked.
 * bn_debug_word synchronises the device and returns the OR of the bits set
 * since the last call, clearing them; ~0u if the synchronisation failed.
 * The regular build compiles the checks out and always returns 0.
 * bn_debug_build returns 1 in the debug build, 0 otherwise. */
#define BN_DEBUG_SPILL 1u
#define BN_DEBUG_INDEX 2u
uint32_t bn_debug_word(void);
int bn_debug_build(void);

#ifdef __cplusplus
}
#endif

#endif /* BN_GB300_H */
