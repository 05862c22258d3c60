// Mixed-size batches (include/bn.h, bn_batch_*): many operations of different
// sizes and kinds run as one CUDA graph.
//
// Classes.  Items are grouped by kind and size: additions and schoolbook
// products by ceil(log2(longer operand)), transform products by their
// transform length N.  Each class is one persistent, descriptor-driven kernel
// (k_add_team_batch, k_mul_quad_batch, k_mul_ntt_batch) whose CTAs take items
// from a device work queue, largest items first.  The class kernels are
// captured once, spread over a few streams so small classes run beside large
// ones, and the graph is replayed on each execution with new buffer bindings.
//
// Cost model.  For BN_OP_MUL_AUTO items the batch estimates the time of the
// schoolbook product (word products / the class's word-product rate) and of
// both transform forms (per-item time at the item's N) and keeps the fastest.
// The built-in figures were measured on GB300 with the size-sweep batches;
// BN_BATCH_AUTOTUNE re-measures them for the classes present, on synthetic
// items at each class's largest size, and also picks each schoolbook class's
// window size Q and CTA size.
//
// Baselines.  BN_BATCH_PLAIN runs every item as its own ordinary launch.
// BN_BATCH_PLAIN_CLASSES runs the plain method the way a caller of the
// per-size entry points would: per class, the items' operands are gathered
// into contiguous rows zero-padded to the class's largest sizes (products
// take the longer operand first), one ordinary batched launch computes the
// class, and the low limbs of each padded result are scattered back.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <new>
#include <vector>

#include "bn_internal.h"

namespace {

enum Kind { K_ADD = 0, K_QUAD = 1, K_NTT64 = 2, K_CRT = 3, K_NTT3 = 4 };

uint32_t ceil_log2(uint32_t x) {
    uint32_t l = 0;
    while ((1u << l) < x) ++l;
    return l;
}

uint32_t transform_length(bool crt, uint32_t na, uint32_t nb) {
    const uint32_t d = crt ? na + nb : 2 * (na + nb);
    return 1u << ceil_log2(d < 2 ? 2 : d);
}

using bn::default_ntt_us;
using bn::default_quad_rate;

struct Class {
    Kind kind;
    uint32_t key;           // log2 size (add/quad) or log2 N (transforms)
    uint32_t first = 0, count = 0;  // range in the sorted item array
    double est_us = 0;      // estimated class time
    bn::AddClass ac;
    bn::QuadClass qc;
    bn::NttPlan *ntt = nullptr;
    bn::Ntt3Plan *ntt3 = nullptr;
};

// One item of a padded plain class: operand x (the longer one for products)
// and y, taken from the flat a or b array, and the result limbs to keep.
struct PlainItem {
    uint64_t off_x, off_y, off_c;
    uint32_t nx, ny, nout, x_from_b;
};

struct PlainClass {
    Kind kind;
    uint32_t first = 0, count = 0;     // range in the sorted item array
    uint32_t pad_x = 0, pad_y = 0, out = 0;
    uint32_t *X = nullptr, *Y = nullptr, *C = nullptr;  // count x pad_x / pad_y / out
    bn::AddConfig add;
    bn::QuadConfig quad;
    bn::NttPlan *ntt = nullptr;
    bn::Ntt3Plan *ntt3 = nullptr;
};

// Copies each item's operands into its zero-padded rows of X and Y.
__global__ void k_plain_gather(const PlainItem *items, uint32_t count, uint32_t pad_x, uint32_t pad_y,
                               const uint32_t *a, const uint32_t *b, uint32_t *X, uint32_t *Y) {
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
        const PlainItem it = items[i];
        const uint32_t *sx = it.x_from_b ? b + it.off_x : a + it.off_x;
        const uint32_t *sy = it.x_from_b ? a + it.off_y : b + it.off_y;
        uint32_t *dx = X + (size_t)i * pad_x, *dy = Y + (size_t)i * pad_y;
        for (uint32_t k = threadIdx.x; k < pad_x; k += blockDim.x) dx[k] = k < it.nx ? sx[k] : 0u;
        for (uint32_t k = threadIdx.x; k < pad_y; k += blockDim.x) dy[k] = k < it.ny ? sy[k] : 0u;
    }
}

// Copies the low nout limbs of each padded result row to the item's result.
__global__ void k_plain_scatter(const PlainItem *items, uint32_t count, uint32_t out,
                                const uint32_t *C, uint32_t *c) {
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
        const PlainItem it = items[i];
        const uint32_t *src = C + (size_t)i * out;
        for (uint32_t k = threadIdx.x; k < it.nout; k += blockDim.x) c[it.off_c + k] = src[k];
    }
}

}  // namespace

struct bn_batch_s {
    int device = 0;
    uint32_t flags = 0;
    std::vector<bn::BatchItem> items;  // sorted by class, then cost (host copy)
    std::vector<Kind> kinds;           // per sorted item (plain mode)
    std::vector<uint32_t> class_of;    // per sorted item: its class (plain mode)
    std::vector<Class> classes;
    bn::BatchItem *d_items = nullptr;
    uint32_t *d_queues = nullptr;
    bn::BatchBinding *d_bind = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bn_batch_info info{};
    std::map<uint32_t, bn::QuadConfig> plain_quad;  // (na << 16 | nb) -> config
    std::vector<PlainClass> plain;     // BN_BATCH_PLAIN_CLASSES
    PlainItem *d_plain_items = nullptr;
    uint32_t *d_plain_buf = nullptr;
};

namespace {

void release(bn_batch_s *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->events) cudaEventDestroy(e);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto &c : b->classes) {
        if (c.ntt) bn::ntt_destroy(c.ntt);
        if (c.ntt3) bn::ntt3_destroy(c.ntt3);
    }
    for (auto &c : b->plain) {
        if (c.ntt) bn::ntt_destroy(c.ntt);
        if (c.ntt3) bn::ntt3_destroy(c.ntt3);
    }
    cudaFree(b->d_plain_items);
    cudaFree(b->d_plain_buf);
    cudaFree(b->d_items);
    cudaFree(b->d_queues);
    cudaFree(b->d_bind);
    delete b;
}

bn_status fail(bn_batch_s *b, bn_status s, const char *what) {
    bn::record_error(what);
    release(b);
    return s;
}

// Launches one class's kernel.
cudaError_t launch_class(const Class &c, const bn::BatchItem *items, uint32_t *queue,
                         const bn::BatchBinding *bind, cudaStream_t st) {
    switch (c.kind) {
    case K_ADD: return bn::add_batch_launch(c.ac, items + c.first, c.count, bind, st);
    case K_QUAD: return bn::quad_batch_launch(c.qc, items + c.first, c.count, queue, bind, st);
    case K_NTT3: return bn::ntt3_batch_launch(c.ntt3, items + c.first, c.count, queue, bind, st);
    default: return bn::ntt_batch_launch(c.ntt, items + c.first, c.count, queue, bind, st);
    }
}

// Autotuning: time candidate configurations on synthetic items at the class's
// largest size, in scratch buffers filled with a fixed byte pattern.
struct Tuner {
    uint32_t *a = nullptr, *b = nullptr, *c = nullptr;
    bn::BatchItem *items = nullptr;
    uint32_t *queue = nullptr;
    bn::BatchBinding *bind = nullptr;
    size_t limbs = 0;
    uint32_t max_items = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;

    bool init(size_t limbs_cap, uint32_t items_cap) {
        limbs = limbs_cap;
        max_items = items_cap;
        if (cudaMalloc(&a, limbs * 4) || cudaMalloc(&b, limbs * 4) || cudaMalloc(&c, 2 * limbs * 4) ||
            cudaMalloc(&items, items_cap * sizeof(bn::BatchItem)) || cudaMalloc(&queue, 4) ||
            cudaMalloc(&bind, sizeof(bn::BatchBinding)))
            return false;
        cudaMemset(a, 0x5A, limbs * 4);
        cudaMemset(b, 0xA5, limbs * 4);
        const bn::BatchBinding hb{a, b, c};
        cudaMemcpy(bind, &hb, sizeof hb, cudaMemcpyHostToDevice);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        return cudaGetLastError() == cudaSuccess;
    }
    ~Tuner() {
        cudaFree(a); cudaFree(b); cudaFree(c); cudaFree(items); cudaFree(queue); cudaFree(bind);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
    // Microseconds per item for `n` synthetic items of na x nb limbs.
    double time_class(const Class &cls, uint32_t na, uint32_t nb, uint32_t n, uint32_t out) {
        n = std::min<uint32_t>(n, max_items);
        n = std::min<uint64_t>(n, limbs / std::max(na, nb));
        if (n == 0) return 1e30;
        std::vector<bn::BatchItem> h(n);
        for (uint32_t i = 0; i < n; ++i) h[i] = {0, 0, (uint64_t)i * out, na, nb};
        cudaMemcpy(items, h.data(), n * sizeof(bn::BatchItem), cudaMemcpyHostToDevice);
        Class c = cls;
        c.first = 0;
        c.count = n;
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaMemsetAsync(queue, 0, 4, 0);
            cudaEventRecord(e0, 0);
            if (launch_class(c, items, queue, bind, 0) != cudaSuccess) return 1e30;
            cudaEventRecord(e1, 0);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);
        }
        return best * 1000.0 / n;
    }
};

}  // namespace

extern "C" {

bn_status bn_batch_create(bn_batch *out, const bn_batch_item *items, uint64_t count, uint32_t flags) {
    using namespace bn;
    if (!out || (!items && count)) {
        record_error("null argument");
        return BN_EINVAL;
    }
    *out = nullptr;
    if (count > 0xffffffffull) {
        record_error("more than 2^32 - 1 items");
        return BN_EUNSUPPORTED;
    }
    bn_batch_s *b = new (std::nothrow) bn_batch_s();
    if (!b) return BN_ENOMEM;
    b->flags = flags;
    if (cudaGetDevice(&b->device) != cudaSuccess) return fail(b, BN_ECUDA, "cudaGetDevice failed");
    const auto t_start = std::chrono::steady_clock::now();

    // Validate and find the candidate classes of every item.
    for (uint64_t i = 0; i < count; ++i) {
        const bn_batch_item &it = items[i];
        const bool is_add = it.op == BN_OP_ADD;
        const uint32_t lim = is_add ? BN_ADD_MAX_LIMBS : BN_MUL_MAX_LIMBS;
        if (it.reserved || it.op > BN_OP_MUL_AUTO || it.na == 0 || it.nb == 0)
            return fail(b, BN_EINVAL, "bad batch item (op, zero size or reserved field)");
        if (it.na > lim || it.nb > lim) return fail(b, BN_EUNSUPPORTED, "batch item above the op's size limit");
    }

    // Schoolbook rates and transform times: built-in, or measured.
    std::map<uint32_t, double> quad_rate;          // key -> word products per us
    std::map<uint32_t, std::pair<uint32_t, uint32_t>> quad_cfg;  // key -> (Q, CTA target)
    std::map<uint32_t, double> t64, tcrt, t3;      // logN -> us per item
    auto quad_key = [](uint32_t na, uint32_t nb) { return ceil_log2(std::max(na, nb)); };
    for (uint64_t i = 0; i < count; ++i) {
        const bn_batch_item &it = items[i];
        if (it.op == BN_OP_ADD) continue;
        const uint32_t k = quad_key(it.na, it.nb);
        quad_rate[k] = default_quad_rate(k);
        quad_cfg[k] = {8u, 256u};
        if (it.op == BN_OP_MUL_AUTO || it.op == BN_OP_MUL_NTT64) {
            const uint32_t l = ceil_log2(transform_length(false, it.na, it.nb));
            t64[l] = default_ntt_us(false, l);
        }
        if (it.op == BN_OP_MUL_AUTO || it.op == BN_OP_MUL_NTT_CRT) {
            const uint32_t l = ceil_log2(transform_length(true, it.na, it.nb));
            tcrt[l] = default_ntt_us(true, l);
        }
        if (it.op == BN_OP_MUL_AUTO) {
            const uint32_t l = ceil_log2(transform_length(true, it.na, it.nb));
            t3[l] = default_ntt3_us(l);
        }
    }
    std::map<std::pair<int, uint32_t>, NttPlan *> ntt_plans;  // (crt, logN) -> plan
    auto get_plan = [&](bool crt, uint32_t logN) -> NttPlan * {
        auto key = std::make_pair((int)crt, logN);
        auto it = ntt_plans.find(key);
        if (it != ntt_plans.end()) return it->second;
        NttPlan *p = nullptr;
        if (ntt_batch_plan(&p, crt, 1u << logN) != BN_OK) p = nullptr;
        ntt_plans[key] = p;
        return p;
    };
    std::map<uint32_t, Ntt3Plan *> ntt3_plans;  // logN -> plan
    auto get_plan3 = [&](uint32_t logN) -> Ntt3Plan * {
        auto it = ntt3_plans.find(logN);
        if (it != ntt3_plans.end()) return it->second;
        Ntt3Plan *p = nullptr;
        if (ntt3_batch_plan(&p, 1u << logN) != BN_OK) p = nullptr;
        ntt3_plans[logN] = p;
        return p;
    };
    auto free_unused_plans = [&]() {
        for (auto &kv : ntt_plans)
            if (kv.second) ntt_destroy(kv.second);
        ntt_plans.clear();
        for (auto &kv : ntt3_plans)
            if (kv.second) ntt3_destroy(kv.second);
        ntt3_plans.clear();
    };

    if (flags & BN_BATCH_AUTOTUNE) {
        Tuner tu;
        if (!tu.init(64u << 20, 1u << 16)) {
            free_unused_plans();
            return fail(b, BN_ENOMEM, "autotune buffers");
        }
        for (auto &kv : quad_rate) {
            const uint32_t n = 1u << kv.first;
            double best = 0;
            for (uint32_t q : {4u, 8u})
                for (uint32_t cta : {256u, 512u}) {
                    Class c{K_QUAD, kv.first};
                    if (quad_batch_class(c.qc, q, std::min(n, BN_MUL_MAX_LIMBS), cta) != BN_OK) continue;
                    const uint32_t m = std::min(n, BN_MUL_MAX_LIMBS);
                    const double us = tu.time_class(c, m, m, 2 * c.qc.grid * c.qc.ipb, 2 * m);
                    const double rate = (double)m * m / us;
                    if (rate > best) {
                        best = rate;
                        quad_cfg[kv.first] = {q, cta};
                    }
                }
            if (best > 0) kv.second = best;
        }
        for (int crt = 0; crt < 2; ++crt)
            for (auto &kv : (crt ? tcrt : t64)) {
                NttPlan *p = get_plan(crt, kv.first);
                if (!p) continue;
                const uint32_t N = 1u << kv.first, side = crt ? N / 2 : N / 4;
                if (side > BN_MUL_MAX_LIMBS) continue;
                Class c{crt ? K_CRT : K_NTT64, kv.first};
                c.ntt = p;
                kv.second = tu.time_class(c, side, side, 2 * 152, 2 * side);
            }
        for (auto &kv : t3) {
            Ntt3Plan *p = get_plan3(kv.first);
            const uint32_t side = (1u << kv.first) / 2;
            if (!p || side > BN_MUL_MAX_LIMBS) continue;
            Class c{K_NTT3, kv.first};
            c.ntt3 = p;
            kv.second = tu.time_class(c, side, side, 4 * 152, 2 * side);
        }
        if (cudaGetLastError() != cudaSuccess) {
            free_unused_plans();
            return fail(b, BN_ECUDA, "autotuning failed");
        }
    }

    // Assign each item a kind and class key.
    struct Tmp {
        Kind kind;
        uint32_t key;
        double cost;
        bn::BatchItem item;
    };
    std::vector<Tmp> tmp;
    tmp.reserve(count);
    for (uint64_t i = 0; i < count; ++i) {
        const bn_batch_item &it = items[i];
        const bn::BatchItem bi{it.a_offset, it.b_offset, it.c_offset, it.na, it.nb};
        const uint32_t mx = std::max(it.na, it.nb);
        if (it.op == BN_OP_ADD) {
            tmp.push_back({K_ADD, ceil_log2(mx), (double)(it.na + it.nb), bi});
            continue;
        }
        const uint32_t qk = quad_key(it.na, it.nb);
        const double cq = (double)it.na * it.nb / quad_rate[qk];
        const uint32_t l64 = ceil_log2(transform_length(false, it.na, it.nb));
        const uint32_t lcrt = ceil_log2(transform_length(true, it.na, it.nb));
        Kind k = K_QUAD;
        double cost = cq;
        if (it.op == BN_OP_MUL_NTT64) k = K_NTT64;
        else if (it.op == BN_OP_MUL_NTT_CRT) k = K_CRT;
        else if (it.op == BN_OP_MUL_AUTO) {
            const double c64 = t64.count(l64) ? t64[l64] : 1e30, cc = tcrt.count(lcrt) ? tcrt[lcrt] : 1e30;
            const double c3 = t3.count(lcrt) ? t3[lcrt] : 1e30;
            if (c64 < cost) { k = K_NTT64; cost = c64; }
            if (cc < cost) { k = K_CRT; cost = cc; }
            if (c3 < cost) { k = K_NTT3; cost = c3; }
        }
        if (k == K_NTT64) cost = t64.count(l64) ? t64[l64] : default_ntt_us(false, l64);
        if (k == K_CRT) cost = tcrt.count(lcrt) ? tcrt[lcrt] : default_ntt_us(true, lcrt);
        const uint32_t key = k == K_QUAD ? qk : (k == K_NTT64 ? l64 : lcrt);  // K_NTT3: lcrt
        tmp.push_back({k, key, k == K_QUAD ? (double)it.na * it.nb : cost * 1e6 + it.na + it.nb, bi});
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const Tmp &x, const Tmp &y) {
        if (x.kind != y.kind) return x.kind < y.kind;
        if (x.key != y.key) return x.key < y.key;
        return x.cost > y.cost;  // largest first within a class
    });

    // Build the classes.
    b->items.reserve(tmp.size());
    b->kinds.reserve(tmp.size());
    for (size_t i = 0; i < tmp.size();) {
        size_t j = i;
        while (j < tmp.size() && tmp[j].kind == tmp[i].kind && tmp[j].key == tmp[i].key) ++j;
        Class c{tmp[i].kind, tmp[i].key};
        c.first = (uint32_t)i;
        c.count = (uint32_t)(j - i);
        bn_status st = BN_OK;
        if (c.kind == K_ADD) {
            st = add_batch_class(c.ac, std::min(1u << c.key, BN_ADD_MAX_LIMBS));
            for (size_t k = i; k < j; ++k) c.est_us += (tmp[k].item.na + tmp[k].item.nb) * 4e-6;
        } else if (c.kind == K_QUAD) {
            const auto cfg = quad_cfg.count(c.key) ? quad_cfg[c.key] : std::make_pair(8u, 256u);
            st = quad_batch_class(c.qc, cfg.first, std::min(1u << c.key, BN_MUL_MAX_LIMBS), cfg.second);
            for (size_t k = i; k < j; ++k)
                c.est_us += (double)tmp[k].item.na * tmp[k].item.nb / quad_rate[c.key];
        } else if (c.kind == K_NTT3) {
            c.ntt3 = get_plan3(c.key);
            if (!c.ntt3) st = BN_ENOMEM;
            ntt3_plans.erase(c.key);  // owned by the class now
            c.est_us = (t3.count(c.key) ? t3[c.key] : 1.0) * c.count;
        } else {
            c.ntt = get_plan(c.kind == K_CRT, c.key);
            if (!c.ntt) st = BN_ENOMEM;
            ntt_plans.erase(std::make_pair((int)(c.kind == K_CRT), c.key));  // owned by the class now
            const double per = c.kind == K_CRT ? (tcrt.count(c.key) ? tcrt[c.key] : 1.0)
                                               : (t64.count(c.key) ? t64[c.key] : 1.0);
            c.est_us = per * c.count;
        }
        if (st != BN_OK) {
            b->classes.push_back(c);  // released with the batch
            free_unused_plans();
            return fail(b, st, "could not set up a batch class");
        }
        b->classes.push_back(c);
        for (size_t k = i; k < j; ++k) {
            b->items.push_back(tmp[k].item);
            b->kinds.push_back(tmp[k].kind);
            b->class_of.push_back((uint32_t)(b->classes.size() - 1));
            switch (tmp[k].kind) {
            case K_ADD: ++b->info.items_add; break;
            case K_QUAD: ++b->info.items_quad; break;
            case K_NTT64: ++b->info.items_ntt64; break;
            case K_CRT: ++b->info.items_crt; break;
            case K_NTT3: ++b->info.items_ntt3; break;
            }
        }
        i = j;
    }
    free_unused_plans();
    b->info.classes = (uint32_t)b->classes.size();

    // Device copies of the items, queues and binding.
    const size_t nq = std::max<size_t>(b->classes.size(), 1);
    if (cudaMalloc(&b->d_items, std::max<size_t>(b->items.size(), 1) * sizeof(bn::BatchItem)) ||
        cudaMalloc(&b->d_queues, nq * 4) || cudaMalloc(&b->d_bind, sizeof(bn::BatchBinding)))
        return fail(b, BN_ENOMEM, "batch device allocation");
    if (!b->items.empty() &&
        cudaMemcpy(b->d_items, b->items.data(), b->items.size() * sizeof(bn::BatchItem),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(b, BN_ECUDA, "batch item upload");

    if ((flags & BN_BATCH_PLAIN) && (flags & BN_BATCH_PLAIN_CLASSES))
        return fail(b, BN_EINVAL, "BN_BATCH_PLAIN and BN_BATCH_PLAIN_CLASSES exclude each other");
    if (flags & BN_BATCH_PLAIN) {
        b->info.launches = (uint32_t)b->items.size();
    } else if (flags & BN_BATCH_PLAIN_CLASSES) {
        // Per class: padded sizes, a plain plan for them, and the rows.
        std::vector<PlainItem> pitems(b->items.size());
        size_t words = 0;
        for (const Class &c : b->classes) {
            PlainClass pc;
            pc.kind = c.kind;
            pc.first = c.first;
            pc.count = c.count;
            for (uint32_t i = c.first; i < c.first + c.count; ++i) {
                const bn::BatchItem &it = b->items[i];
                PlainItem &q = pitems[i];
                const bool swap = c.kind != K_ADD && it.nb > it.na;  // longer operand first
                q.off_x = swap ? it.off_b : it.off_a;
                q.off_y = swap ? it.off_a : it.off_b;
                q.off_c = it.off_c;
                q.nx = swap ? it.nb : it.na;
                q.ny = swap ? it.na : it.nb;
                q.x_from_b = swap;
                q.nout = c.kind == K_ADD ? std::max(it.na, it.nb) + 1 : it.na + it.nb;
                pc.pad_x = std::max(pc.pad_x, c.kind == K_ADD ? std::max(q.nx, q.ny) : q.nx);
                pc.pad_y = std::max(pc.pad_y, c.kind == K_ADD ? std::max(q.nx, q.ny) : q.ny);
            }
            pc.out = c.kind == K_ADD ? pc.pad_x + 1 : pc.pad_x + pc.pad_y;
            bn_status st = BN_OK;
            switch (c.kind) {
            case K_ADD: st = add_configure(pc.add, pc.pad_x, pc.pad_y, nullptr); break;
            case K_QUAD: st = quad_configure(pc.quad, pc.pad_x, pc.pad_y, nullptr); break;
            case K_NTT3: st = ntt3_create(&pc.ntt3, pc.pad_x, pc.pad_y, nullptr); break;
            default: st = ntt_create(&pc.ntt, c.kind == K_CRT, pc.pad_x, pc.pad_y, nullptr); break;
            }
            b->plain.push_back(pc);
            if (st != BN_OK) return fail(b, st, "could not set up a plain class");
            words += (size_t)c.count * (pc.pad_x + pc.pad_y + pc.out);
        }
        if (cudaMalloc(&b->d_plain_items, std::max<size_t>(pitems.size(), 1) * sizeof(PlainItem)) ||
            cudaMalloc(&b->d_plain_buf, std::max<size_t>(words, 1) * 4))
            return fail(b, BN_ENOMEM, "plain class buffers");
        if (!pitems.empty() && cudaMemcpy(b->d_plain_items, pitems.data(), pitems.size() * sizeof(PlainItem),
                                          cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(b, BN_ECUDA, "plain item upload");
        size_t off = 0;
        for (PlainClass &pc : b->plain) {
            pc.X = b->d_plain_buf + off;
            off += (size_t)pc.count * pc.pad_x;
            pc.Y = b->d_plain_buf + off;
            off += (size_t)pc.count * pc.pad_y;
            pc.C = b->d_plain_buf + off;
            off += (size_t)pc.count * pc.out;
        }
        b->info.launches = 3u * (uint32_t)b->plain.size();
    } else if (!b->classes.empty()) {
        // Capture: zero the queues, fork to the streams, one launch per class
        // (largest estimated classes first, round robin), join.
        const int S = (int)std::min<size_t>(4, b->classes.size());
        b->streams.resize(S);
        b->events.resize(S);
        for (int s = 0; s < S; ++s) {
            if (cudaStreamCreateWithFlags(&b->streams[s], cudaStreamNonBlocking) ||
                cudaEventCreateWithFlags(&b->events[s], cudaEventDisableTiming))
                return fail(b, BN_ECUDA, "batch streams");
        }
        std::vector<size_t> order(b->classes.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](size_t x, size_t y) { return b->classes[x].est_us > b->classes[y].est_us; });
        cudaStream_t s0 = b->streams[0];
        cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queues, 0, nq * 4, s0);
        if (e == cudaSuccess) e = cudaEventRecord(b->events[0], s0);
        for (int s = 1; s < S && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->streams[s], b->events[0], 0);
        for (size_t r = 0; r < order.size() && e == cudaSuccess; ++r) {
            const size_t ci = order[r];
            e = launch_class(b->classes[ci], b->d_items, b->d_queues + ci, b->d_bind,
                             b->streams[r % S]);
        }
        for (int s = 1; s < S && e == cudaSuccess; ++s) {
            e = cudaEventRecord(b->events[s], b->streams[s]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, b->events[s], 0);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(s0, &g);
        if (e == cudaSuccess) e = e2;
        b->graph = g;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) return fail(b, BN_ECUDA, "batch graph capture");
        b->info.launches = (uint32_t)b->classes.size();
    }
    b->info.tune_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    *out = b;
    return BN_OK;
}

bn_status bn_batch_execute(bn_batch b, const uint32_t *a, const uint32_t *bb, uint32_t *c, void *stream) {
    using namespace bn;
    if (!b) {
        record_error("null batch");
        return BN_EINVAL;
    }
    if (b->items.empty()) return BN_OK;
    if (!a || !bb || !c) {
        record_error("null operand or result array");
        return BN_EINVAL;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) {
        record_error("batch was created on another device");
        return BN_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (b->flags & BN_BATCH_PLAIN) {
        // One ordinary launch per item: the same kernels and choices as the
        // batch, without classes, queues or a graph.
        for (size_t i = 0; i < b->items.size(); ++i) {
            const bn::BatchItem &it = b->items[i];
            const uint32_t *pa = a + it.off_a, *pb = bb + it.off_b;
            uint32_t *pc = c + it.off_c;
            cudaError_t e = cudaSuccess;
            if (b->kinds[i] == K_ADD) {
                AddConfig cfg;
                add_configure(cfg, it.na, it.nb, nullptr);
                e = add_launch(cfg, pa, pb, pc, 1, st);
            } else if (b->kinds[i] == K_QUAD) {
                const uint32_t key = (it.na << 16) | it.nb;
                auto f = b->plain_quad.find(key);
                if (f == b->plain_quad.end()) {
                    QuadConfig cfg;
                    quad_configure(cfg, it.na, it.nb, nullptr);
                    f = b->plain_quad.emplace(key, cfg).first;
                }
                e = quad_launch(f->second, pa, pb, pc, 1, st);
            } else {
                const Class &cls = b->classes[b->class_of[i]];
                e = cls.ntt3 ? ntt3_launch_sized(cls.ntt3, it.na, it.nb, pa, pb, pc, st)
                             : ntt_launch_sized(cls.ntt, it.na, it.nb, pa, pb, pc, st);
            }
            if (e != cudaSuccess) {
                record_error("plain batch launch failed");
                return BN_ECUDA;
            }
        }
        return BN_OK;
    }
    if (b->flags & BN_BATCH_PLAIN_CLASSES) {
        // Per class, in order: gather into padded rows, one plain launch, scatter.
        for (const PlainClass &pc : b->plain) {
            const PlainItem *pi = b->d_plain_items + pc.first;
            const unsigned grid = std::min<uint32_t>(pc.count, 65535u);
            k_plain_gather<<<grid, 256, 0, st>>>(pi, pc.count, pc.pad_x, pc.pad_y, a, bb, pc.X, pc.Y);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) {
                switch (pc.kind) {
                case K_ADD: e = add_launch(pc.add, pc.X, pc.Y, pc.C, pc.count, st); break;
                case K_QUAD: e = quad_launch(pc.quad, pc.X, pc.Y, pc.C, pc.count, st); break;
                case K_NTT3: e = ntt3_launch(pc.ntt3, pc.X, pc.Y, pc.C, pc.count, st); break;
                default: e = ntt_launch(pc.ntt, pc.X, pc.Y, pc.C, pc.count, st); break;
                }
            }
            if (e == cudaSuccess) {
                k_plain_scatter<<<grid, 256, 0, st>>>(pi, pc.count, pc.out, pc.C, c);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) {
                record_error("plain class launch failed");
                return BN_ECUDA;
            }
        }
        return BN_OK;
    }
    const bn::BatchBinding h{a, bb, c};
    cudaError_t e = cudaMemcpyAsync(b->d_bind, &h, sizeof h, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) {
        record_error("batch graph launch failed");
        return BN_ECUDA;
    }
    return BN_OK;
}

bn_status bn_batch_get_info(bn_batch b, bn_batch_info *info) {
    if (!b || !info) return BN_EINVAL;
    *info = b->info;
    return BN_OK;
}

bn_status bn_batch_destroy(bn_batch b) {
    if (!b) return BN_OK;
    const cudaError_t e = cudaDeviceSynchronize();
    release(b);
    return e == cudaSuccess ? BN_OK : BN_ECUDA;
}

}  // extern "C"
