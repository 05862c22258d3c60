// C ABI of the library (include/bn.h): plans, argument validation, the
// host-buffer path and the one-shot forms with their per-size plan cache.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>

#include "bn_internal.h"

struct bn_plan_s {
    bn_op op;
    uint32_t na, nb, nout;
    uint64_t batch;
    int device;
    bn::AddConfig add;
    bn::QuadConfig quad;
    bn::NttPlan *ntt = nullptr;
    bn::Ntt3Plan *ntt3 = nullptr;
    bn::QuadTcPlan *qtc = nullptr;
    // Device staging for bn_plan_execute_host (allocated on first use).
    uint32_t *d_a = nullptr, *d_b = nullptr, *d_c = nullptr;
    uint64_t staged_batch = 0;
};

namespace {

thread_local char g_last_error[256] = "";

void set_error(const char *what, cudaError_t e) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s)", what, cudaGetErrorName(e),
                  cudaGetErrorString(e));
}

void set_error_text(const char *what) { std::snprintf(g_last_error, sizeof g_last_error, "%s", what); }

bn_status cuda_status(const char *what, cudaError_t e) {
    if (e == cudaSuccess) return BN_OK;
    set_error(what, e);
    if (e == cudaErrorMemoryAllocation) return BN_ENOMEM;
    return BN_ECUDA;
}

bool overlaps(const void *p, uint64_t pbytes, const void *q, uint64_t qbytes) {
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return a < b + qbytes && b < a + pbytes;
}

uint32_t out_limbs(bn_op op, uint32_t na, uint32_t nb) {
    return op == BN_OP_ADD ? (na > nb ? na : nb) + 1 : na + nb;
}

bn_status configure(bn_plan_s *p, const bn_tuning *t) {
    switch (p->op) {
    case BN_OP_ADD: return bn::add_configure(p->add, p->na, p->nb, t);
    case BN_OP_MUL_QUAD: return bn::quad_configure(p->quad, p->na, p->nb, t);
    case BN_OP_MUL_NTT64:
    case BN_OP_MUL_NTT_CRT:
        return bn::ntt_create(&p->ntt, p->op == BN_OP_MUL_NTT_CRT, p->na, p->nb, t);
    case BN_OP_MUL_NTT3: return bn::ntt3_create(&p->ntt3, p->na, p->nb, t);
    case BN_OP_MUL_QUAD_TC:
        if (t && (t->limbs_per_thread || t->cta_threads)) return BN_EINVAL;  // fixed geometry
        return bn::quad_tc_create(&p->qtc, p->na, p->nb);
    default: break;
    }
    return BN_EINVAL;
}

bn_status check_args(bn_plan_s *p, const uint32_t *a, const uint32_t *b, const uint32_t *c,
                     uint64_t batch) {
    if (!a || !b || !c) {
        set_error_text("null operand or result pointer");
        return BN_EINVAL;
    }
    const uint64_t ab = batch * p->na * 4ull, bb = batch * p->nb * 4ull, cb = batch * p->nout * 4ull;
    if (overlaps(c, cb, a, ab) || overlaps(c, cb, b, bb)) {
        set_error_text("result overlaps an operand");
        return BN_EINVAL;
    }
    return BN_OK;
}

bn_status launch(bn_plan_s *p, const uint32_t *a, const uint32_t *b, uint32_t *c, uint64_t batch,
                 cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    switch (p->op) {
    case BN_OP_ADD: e = bn::add_launch(p->add, a, b, c, batch, st); break;
    case BN_OP_MUL_QUAD: e = bn::quad_launch(p->quad, a, b, c, batch, st); break;
    case BN_OP_MUL_NTT64:
    case BN_OP_MUL_NTT_CRT: e = bn::ntt_launch(p->ntt, a, b, c, batch, st); break;
    case BN_OP_MUL_NTT3: e = bn::ntt3_launch(p->ntt3, a, b, c, batch, st); break;
    case BN_OP_MUL_QUAD_TC: e = bn::quad_tc_launch(p->qtc, a, b, c, batch, st); break;
    default: e = cudaErrorInvalidValue; break;
    }
    return cuda_status("kernel launch", e);
}

bn_status execute(bn_plan_s *p, const uint32_t *a, const uint32_t *b, uint32_t *c, uint64_t batch,
                  void *stream) {
    if (batch == 0) return BN_OK;
    bn_status s = check_args(p, a, b, c, batch);
    if (s != BN_OK) return s;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status("cudaGetDevice", e);
    if (dev != p->device) {
        set_error_text("plan was created on another device");
        return BN_EINVAL;
    }
    return launch(p, a, b, c, batch, (cudaStream_t)stream);
}

struct CacheKey {
    int op, device;
    uint32_t na, nb;
    bool operator<(const CacheKey &o) const {
        return std::tie(op, device, na, nb) < std::tie(o.op, o.device, o.na, o.nb);
    }
};

std::mutex g_cache_mutex;
std::map<CacheKey, bn_plan> g_cache;

bn_status cached_plan(bn_op op, uint32_t na, uint32_t nb, bn_plan *out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status("cudaGetDevice", e);
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    const CacheKey key{(int)op, dev, na, nb};
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *out = it->second;
        return BN_OK;
    }
    bn_plan p = nullptr;
    bn_status s = bn_plan_create(&p, op, na, nb, 0, nullptr);
    if (s != BN_OK) return s;
    g_cache.emplace(key, p);
    *out = p;
    return BN_OK;
}

bn_status one_shot(bn_op op, const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t na,
                   uint32_t nb, uint64_t batch, void *stream) {
    if (na == 0 || nb == 0) {
        set_error_text("zero limb count");
        return BN_EINVAL;
    }
    if (batch == 0) return BN_OK;
    bn_plan p = nullptr;
    bn_status s = cached_plan(op, na, nb, &p);
    if (s != BN_OK) return s;
    return execute(p, a, b, c, batch, stream);
}

}  // namespace

namespace bn {

void record_error(const char *what) { set_error_text(what); }

cudaError_t allow_max_smem(const void *kernel) {
    static std::mutex m;
    static std::map<std::pair<const void *, int>, bool> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(m);
    auto key = std::make_pair(kernel, dev);
    if (done.count(key)) return cudaSuccess;
    int optin = 0;
    cudaFuncAttributes fa{};
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    // The cap covers dynamic memory only; static plus dynamic must fit the opt-in limit.
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done[key] = true;
    return e;
}

}  // namespace bn

extern "C" {

bn_status bn_plan_create(bn_plan *out, bn_op op, uint32_t na, uint32_t nb, uint64_t batch,
                         const bn_tuning *tuning) {
    if (!out) {
        set_error_text("null plan pointer");
        return BN_EINVAL;
    }
    *out = nullptr;
    if (op != BN_OP_ADD && op != BN_OP_MUL_QUAD && op != BN_OP_MUL_NTT64 && op != BN_OP_MUL_NTT_CRT &&
        op != BN_OP_MUL_NTT3 && op != BN_OP_MUL_AUTO && op != BN_OP_MUL_QUAD_TC) {
        set_error_text("unknown op");
        return BN_EINVAL;
    }
    if (na == 0 || nb == 0) {
        set_error_text("zero limb count");
        return BN_EINVAL;
    }
    if (op == BN_OP_MUL_AUTO) {
        // The cost model's fastest product for the sizes (same choice as a
        // batch item without autotuning).
        if (na > BN_MUL_MAX_LIMBS || nb > BN_MUL_MAX_LIMBS) {
            set_error_text("size not supported by this op");
            return BN_EUNSUPPORTED;
        }
        static const bn_op kinds[5] = {BN_OP_MUL_QUAD, BN_OP_MUL_QUAD, BN_OP_MUL_NTT64, BN_OP_MUL_NTT_CRT,
                                       BN_OP_MUL_NTT3};
        const uint32_t k = bn::choose_mul(na, nb).kind;
        op = kinds[k < 5 ? k : 1];
        if (tuning && op != BN_OP_MUL_QUAD) tuning = nullptr;  // schoolbook tuning only
    }
    bn_plan_s *p = new (std::nothrow) bn_plan_s();
    if (!p) return BN_ENOMEM;
    p->op = op;
    p->na = na;
    p->nb = nb;
    p->nout = out_limbs(op, na, nb);
    p->batch = batch;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_status("cudaGetDevice", e);
    }
    bn_status s = configure(p, tuning);
    if (s != BN_OK) {
        if (s == BN_EUNSUPPORTED) set_error_text("size not supported by this op");
        else if (s == BN_EINVAL) set_error_text("bad size or tuning");
        delete p;
        return s;
    }
    *out = p;
    return BN_OK;
}

bn_status bn_plan_execute(bn_plan plan, const uint32_t *a, const uint32_t *b, uint32_t *c,
                          void *stream) {
    if (!plan) {
        set_error_text("null plan");
        return BN_EINVAL;
    }
    return execute(plan, a, b, c, plan->batch, stream);
}

namespace {

bn_status execute_host(bn_plan plan, const uint32_t *a, const uint32_t *b, uint32_t *c, void *stream,
                       bool sync) {
    if (!plan) {
        set_error_text("null plan");
        return BN_EINVAL;
    }
    const uint64_t batch = plan->batch;
    if (batch == 0) return BN_OK;
    if (!a || !b || !c) {
        set_error_text("null host pointer");
        return BN_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ab = batch * plan->na * 4ull, bb = batch * plan->nb * 4ull,
                 cb = batch * plan->nout * 4ull;
    if (plan->staged_batch < batch) {
        cudaFree(plan->d_a);
        cudaFree(plan->d_b);
        cudaFree(plan->d_c);
        plan->d_a = plan->d_b = plan->d_c = nullptr;
        plan->staged_batch = 0;
        cudaError_t e = cudaMalloc(&plan->d_a, ab);
        if (e == cudaSuccess) e = cudaMalloc(&plan->d_b, bb);
        if (e == cudaSuccess) e = cudaMalloc(&plan->d_c, cb);
        if (e != cudaSuccess) return cuda_status("staging allocation", e);
        plan->staged_batch = batch;
    }
    cudaError_t e = cudaMemcpyAsync(plan->d_a, a, ab, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan->d_b, b, bb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status("host to device copy", e);
    bn_status s = execute(plan, plan->d_a, plan->d_b, plan->d_c, batch, stream);
    if (s != BN_OK) return s;
    e = cudaMemcpyAsync(c, plan->d_c, cb, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status("device to host copy", e);
    return sync ? cuda_status("stream synchronize", cudaStreamSynchronize(st)) : BN_OK;
}

}  // namespace

bn_status bn_plan_execute_host(bn_plan plan, const uint32_t *a, const uint32_t *b, uint32_t *c,
                               void *stream) {
    return execute_host(plan, a, b, c, stream, true);
}

bn_status bn_plan_execute_host_async(bn_plan plan, const uint32_t *a, const uint32_t *b, uint32_t *c,
                                     void *stream) {
    return execute_host(plan, a, b, c, stream, false);
}

bn_status bn_plan_destroy(bn_plan plan) {
    if (!plan) return BN_OK;
    {
        // A destroyed plan must not stay reachable from the one-shot cache.
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
            if (it->second == plan) {
                g_cache.erase(it);
                break;
            }
    }
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(plan->d_a);
    cudaFree(plan->d_b);
    cudaFree(plan->d_c);
    if (plan->ntt) bn::ntt_destroy(plan->ntt);
    if (plan->ntt3) bn::ntt3_destroy(plan->ntt3);
    if (plan->qtc) bn::quad_tc_destroy(plan->qtc);
    delete plan;
    return cuda_status("cudaDeviceSynchronize", e);
}

uint32_t bn_plan_out_limbs(bn_plan plan) { return plan ? plan->nout : 0; }

int bn_plan_op(bn_plan plan) { return plan ? (int)plan->op : -1; }

size_t bn_plan_scratch_bytes(bn_plan plan) {
    if (plan && plan->ntt3) return bn::ntt3_scratch_bytes(plan->ntt3);
    if (plan && plan->qtc) return bn::quad_tc_scratch_bytes(plan->qtc);
    return (plan && plan->ntt) ? bn::ntt_scratch_bytes(plan->ntt) : 0;
}

uint32_t bn_plan_transform_length(bn_plan plan) {
    if (plan && plan->ntt3) return bn::ntt3_length(plan->ntt3);
    return (plan && plan->ntt) ? bn::ntt_length(plan->ntt) : 0;
}

bn_status bn_add(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t na, uint32_t nb,
                 uint64_t batch, void *stream) {
    return one_shot(BN_OP_ADD, a, b, c, na, nb, batch, stream);
}

bn_status bn_mul_quad(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t na, uint32_t nb,
                      uint64_t batch, void *stream) {
    return one_shot(BN_OP_MUL_QUAD, a, b, c, na, nb, batch, stream);
}

bn_status bn_mul_ntt(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t na, uint32_t nb,
                     uint64_t batch, int crt, void *stream) {
    return one_shot(crt ? BN_OP_MUL_NTT_CRT : BN_OP_MUL_NTT64, a, b, c, na, nb, batch, stream);
}

bn_status bn_mul_ntt3(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t na, uint32_t nb,
                      uint64_t batch, void *stream) {
    return one_shot(BN_OP_MUL_NTT3, a, b, c, na, nb, batch, stream);
}

bn_status bn_mul_quad_tc(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t na, uint32_t nb,
                         uint64_t batch, void *stream) {
    return one_shot(BN_OP_MUL_QUAD_TC, a, b, c, na, nb, batch, stream);
}

bn_status bn_tc_check(void) {
    uint32_t flag = 0;
    cudaError_t e = bn::tc_fault_take(&flag);
    if (e != cudaSuccess) return cuda_status("tensor-core status", e);
    if (flag) {
        set_error_text("a tensor-core kernel gave up waiting for its MMAs");
        return BN_ETIMEOUT;
    }
    return BN_OK;
}

bn_status bn_tc_wait_selftest(uint32_t limit_us) {
    uint32_t flag = 0;
    cudaError_t e = bn::tc_fault_take(&flag);  // start from a clear flag
    if (e == cudaSuccess) e = bn::tc_wait_selftest(limit_us);
    if (e == cudaSuccess) e = bn::tc_fault_take(&flag);
    if (e != cudaSuccess) return cuda_status("tensor-core wait self-test", e);
    if (!flag) {
        set_error_text("the self-test's wait did not give up");
        return BN_OK;
    }
    return BN_ETIMEOUT;
}

bn_status bn_mul(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t na, uint32_t nb,
                 uint64_t batch, void *stream) {
    return one_shot(BN_OP_MUL_AUTO, a, b, c, na, nb, batch, stream);
}

const char *bn_status_str(bn_status s) {
    switch (s) {
    case BN_OK: return "ok";
    case BN_EINVAL: return "invalid argument";
    case BN_ENOMEM: return "out of memory";
    case BN_ECUDA: return "CUDA error";
    case BN_EUNSUPPORTED: return "unsupported size";
    case BN_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char *bn_last_error(void) { return g_last_error; }

int bn_version(void) { return 100; }

uint32_t bn_debug_word(void) {
    if (cudaDeviceSynchronize() != cudaSuccess) return ~0u;
    return bn::debug_word_quad() | bn::debug_word_quad_tc() | bn::debug_word_ntt() |
           bn::debug_word_ntt3_small() | bn::debug_word_ntt3_mid() | bn::debug_word_ntt3_large();
}

int bn_debug_build(void) {
#ifdef BN_DEBUG
    return 1;
#else
    return 0;
#endif
}

}  // extern "C"
