// Serving loop (include/bn.h, bn_server_*): continuous batching of requests
// whose operands are already in device memory.
//
// A scheduler thread owns `max_inflight` slots, each a stream, an event and
// its own descriptor buffers and transform plans.  Each turn it (1) retires
// slots whose event has completed, turning their requests into completions,
// and (2) fills every free slot with pending requests, oldest first, as long
// as each result fits in the device result pool; the admitted requests are
// grouped into size classes (the batch cost model) and the class kernels
// (the batched add / schoolbook / transform kernels) are launched on the
// slot's stream.  Requests arriving while slots are busy wait in the queue and
// go into the next free slot, so new work overlaps work already on the GPU.
// The pool is a first-fit free list with coalescing; results stay there until
// released, and admission stops while the oldest pending result does not fit.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bn_internal.h"
#include "pool_alloc.h"

namespace {

uint32_t clog2(uint32_t x) {
    uint32_t l = 0;
    while ((1u << l) < x) ++l;
    return l;
}

using bn::PoolAllocator;

struct Req {
    uint64_t ticket;
    uint32_t op, na, nb, nout;
    const uint32_t *a, *b;
    double arrival;
    uint64_t c_off = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Req> reqs;
    bn::BatchItem *h_items = nullptr;  // pinned staging
    bn::BatchItem *d_items = nullptr;
    uint32_t *d_queues = nullptr;
    bn::BatchBinding *d_bind = nullptr;
    std::map<std::pair<int, uint32_t>, bn::NttPlan *> plans;  // (crt, log2 N)
    std::map<uint32_t, bn::Ntt3Plan *> plans3;                 // three primes, log2 N
};

constexpr uint32_t kMaxClasses = 64;

}  // namespace

struct bn_server_s {
    int device = 0;
    bn_server_config cfg{};
    uint8_t *d_pool = nullptr;
    PoolAllocator *alloc = nullptr;
    std::mutex pool_mutex;
    std::unordered_map<uint64_t, std::pair<uint64_t, uint64_t>> results;  // ticket -> (off, bytes)
    std::mutex queue_mutex;
    std::condition_variable queue_cv;
    std::deque<Req> pending;
    std::mutex done_mutex;
    std::vector<bn_completion> completed;
    std::vector<Slot> slots;
    std::map<uint32_t, bn::QuadClass> quad_classes;
    std::map<uint32_t, bn::AddClass> add_classes;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::atomic<uint64_t> next_ticket{1}, submitted{0}, completed_count{0}, batches{0};
    std::atomic<uint32_t> inflight{0}, max_inflight_seen{0};
    std::atomic<bool> worker_error{false};
    std::chrono::steady_clock::time_point t0;

    double now_us() const {
        return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

bn::NttPlan *slot_plan(Slot &s, bool crt, uint32_t logn) {
    auto key = std::make_pair((int)crt, logn);
    auto it = s.plans.find(key);
    if (it != s.plans.end()) return it->second;
    bn::NttPlan *p = nullptr;
    if (bn::ntt_batch_plan(&p, crt, 1u << logn) != BN_OK) p = nullptr;
    s.plans[key] = p;
    return p;
}

bn::Ntt3Plan *slot_plan3(Slot &s, uint32_t logn) {
    auto it = s.plans3.find(logn);
    if (it != s.plans3.end()) return it->second;
    bn::Ntt3Plan *p = nullptr;
    if (bn::ntt3_batch_plan(&p, 1u << logn) != BN_OK) p = nullptr;
    s.plans3[logn] = p;
    return p;
}

struct Choice {
    uint32_t kind, key;  // 0 add, 1 schoolbook, 2 ntt64, 3 crt, 4 three primes; class key
    double cost;
};

Choice classify(const Req &r) {
    const uint32_t mx = std::max(r.na, r.nb);
    if (r.op == BN_OP_ADD) return {0, clog2(mx), (double)(r.na + r.nb)};
    const bn::MulChoice m = bn::choose_mul(r.na, r.nb);
    uint32_t kind = m.kind;
    if (r.op == BN_OP_MUL_QUAD) kind = 1;
    if (r.op == BN_OP_MUL_NTT64) kind = 2;
    if (r.op == BN_OP_MUL_NTT_CRT) kind = 3;
    const uint32_t key = kind == 1 ? m.quad_key : (kind == 2 ? m.log_n64 : m.log_ncrt);
    return {kind, key, kind == 1 ? (double)r.na * r.nb : (double)(r.na + r.nb)};
}

// Launches the slot's requests: grouped by class (batched mode) or one plain
// launch per request (sequential mode).
cudaError_t launch_slot(bn_server_s *sv, Slot &s) {
    const bool seq = sv->cfg.flags & BN_SERVER_SEQUENTIAL;
    cudaError_t e = cudaSuccess;
    if (seq) {
        for (const Req &r : s.reqs) {
            const Choice ch = classify(r);
            uint32_t *c = reinterpret_cast<uint32_t *>(sv->d_pool + r.c_off);
            if (ch.kind == 0) {
                bn::AddConfig cfg;
                bn::add_configure(cfg, r.na, r.nb, nullptr);
                e = bn::add_launch(cfg, r.a, r.b, c, 1, s.stream);
            } else if (ch.kind == 1) {
                bn::QuadConfig cfg;
                bn::quad_configure(cfg, r.na, r.nb, nullptr);
                e = bn::quad_launch(cfg, r.a, r.b, c, 1, s.stream);
            } else if (ch.kind == 4) {
                bn::Ntt3Plan *p = slot_plan3(s, ch.key);
                e = p ? bn::ntt3_launch_sized(p, r.na, r.nb, r.a, r.b, c, s.stream) : cudaErrorMemoryAllocation;
            } else {
                bn::NttPlan *p = slot_plan(s, ch.kind == 3, ch.key);
                e = p ? bn::ntt_launch_sized(p, r.na, r.nb, r.a, r.b, c, s.stream) : cudaErrorMemoryAllocation;
            }
            if (e != cudaSuccess) return e;
        }
        return cudaEventRecord(s.done, s.stream);
    }
    // Batched: sort by (kind, key, cost desc), descriptors into pinned staging.
    const size_t n = s.reqs.size();
    std::vector<std::pair<Choice, uint32_t>> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = {classify(s.reqs[i]), (uint32_t)i};
    std::sort(order.begin(), order.end(), [](const auto &x, const auto &y) {
        if (x.first.kind != y.first.kind) return x.first.kind < y.first.kind;
        if (x.first.key != y.first.key) return x.first.key < y.first.key;
        return x.first.cost > y.first.cost;
    });
    for (size_t i = 0; i < n; ++i) {
        const Req &r = s.reqs[order[i].second];
        s.h_items[i] = {(uint64_t)(uintptr_t)r.a / 4, (uint64_t)(uintptr_t)r.b / 4, r.c_off / 4, r.na, r.nb};
    }
    e = cudaMemcpyAsync(s.d_items, s.h_items, n * sizeof(bn::BatchItem), cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.d_queues, 0, kMaxClasses * 4, s.stream);
    uint32_t ci = 0;
    for (size_t i = 0; i < n && e == cudaSuccess;) {
        size_t j = i;
        while (j < n && order[j].first.kind == order[i].first.kind && order[j].first.key == order[i].first.key) ++j;
        const uint32_t kind = order[i].first.kind, key = order[i].first.key, cnt = (uint32_t)(j - i);
        uint32_t *queue = s.d_queues + (ci++ % kMaxClasses);
        if (kind == 0) {
            e = bn::add_batch_launch(sv->add_classes.at(key), s.d_items + i, cnt, s.d_bind, s.stream);
        } else if (kind == 1) {
            e = bn::quad_batch_launch(sv->quad_classes.at(key), s.d_items + i, cnt, queue, s.d_bind, s.stream);
        } else if (kind == 4) {
            bn::Ntt3Plan *p = slot_plan3(s, key);
            e = p ? bn::ntt3_batch_launch(p, s.d_items + i, cnt, queue, s.d_bind, s.stream)
                  : cudaErrorMemoryAllocation;
        } else {
            bn::NttPlan *p = slot_plan(s, kind == 3, key);
            e = p ? bn::ntt_batch_launch(p, s.d_items + i, cnt, queue, s.d_bind, s.stream)
                  : cudaErrorMemoryAllocation;
        }
        if (ci > kMaxClasses) {  // queues would be reused within one micro-batch
            e = cudaErrorInvalidConfiguration;
        }
        i = j;
    }
    if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
    return e;
}

void worker_main(bn_server_s *sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        bool progressed = false;
        // (1) retire finished micro-batches
        for (Slot &s : sv->slots) {
            if (!s.busy || cudaEventQuery(s.done) != cudaSuccess) continue;
            const double t = sv->now_us();
            {
                std::lock_guard<std::mutex> lk(sv->done_mutex);
                for (const Req &r : s.reqs)
                    sv->completed.push_back({r.ticket, reinterpret_cast<uint32_t *>(sv->d_pool + r.c_off),
                                             r.nout, 0, r.arrival, t});
            }
            sv->completed_count += s.reqs.size();
            s.reqs.clear();
            s.busy = false;
            --sv->inflight;
            progressed = true;
        }
        // (2) admit pending requests into free slots
        for (Slot &s : sv->slots) {
            if (s.busy) continue;
            {
                std::lock_guard<std::mutex> lk(sv->queue_mutex);
                while (!sv->pending.empty() && s.reqs.size() < sv->cfg.max_batch) {
                    Req &r = sv->pending.front();
                    const uint64_t bytes = ((uint64_t)r.nout * 4 + 15) & ~15ull;
                    uint64_t off;
                    {
                        std::lock_guard<std::mutex> pl(sv->pool_mutex);
                        if (!sv->alloc->alloc(bytes, &off)) break;  // wait for releases
                        sv->results[r.ticket] = {off, bytes};
                    }
                    r.c_off = off;
                    s.reqs.push_back(r);
                    sv->pending.pop_front();
                }
            }
            if (s.reqs.empty()) break;
            if (launch_slot(sv, s) != cudaSuccess) sv->worker_error = true;
            s.busy = true;
            const uint32_t now_inflight = ++sv->inflight;
            uint32_t seen = sv->max_inflight_seen.load();
            while (now_inflight > seen && !sv->max_inflight_seen.compare_exchange_weak(seen, now_inflight)) {}
            ++sv->batches;
            progressed = true;
        }
        if (sv->stop && sv->inflight == 0) {
            // Stop once nothing is queued, or nothing more can be admitted
            // (results that were never released fill the pool).
            std::lock_guard<std::mutex> lk(sv->queue_mutex);
            if (sv->pending.empty() || !progressed) break;
        }
        if (!progressed) {
            if (sv->inflight > 0) {
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            } else {
                std::unique_lock<std::mutex> lk(sv->queue_mutex);
                sv->queue_cv.wait_for(lk, std::chrono::microseconds(200),
                                      [&] { return !sv->pending.empty() || sv->stop.load(); });
            }
        }
    }
}

void destroy_server(bn_server_s *sv) {
    for (Slot &s : sv->slots) {
        for (auto &kv : s.plans)
            if (kv.second) bn::ntt_destroy(kv.second);
        for (auto &kv : s.plans3)
            if (kv.second) bn::ntt3_destroy(kv.second);
        if (s.h_items) cudaFreeHost(s.h_items);
        cudaFree(s.d_items);
        cudaFree(s.d_queues);
        cudaFree(s.d_bind);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    cudaFree(sv->d_pool);
    delete sv->alloc;
    delete sv;
}

}  // namespace

extern "C" {

bn_status bn_server_create(bn_server *out, const bn_server_config *cfg_in) {
    using namespace bn;
    if (!out) return BN_EINVAL;
    *out = nullptr;
    bn_server_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    if (cfg.reserved || (cfg.flags & ~BN_SERVER_SEQUENTIAL)) {
        record_error("bad server config");
        return BN_EINVAL;
    }
    if (cfg.pool_bytes == 0) cfg.pool_bytes = 1ull << 30;
    if (cfg.pool_bytes > BN_SERVER_MAX_POOL) {
        record_error("pool above BN_SERVER_MAX_POOL");
        return BN_EUNSUPPORTED;
    }
    if (cfg.max_inflight == 0) cfg.max_inflight = 4;
    if (cfg.max_batch == 0) cfg.max_batch = 4096;
    if (cfg.flags & BN_SERVER_SEQUENTIAL) {
        cfg.max_inflight = 1;
        cfg.max_batch = 1;
    }
    if (cfg.max_inflight > 64) {
        record_error("at most 64 slots");
        return BN_EINVAL;
    }
    bn_server_s *sv = new (std::nothrow) bn_server_s();
    if (!sv) return BN_ENOMEM;
    sv->cfg = cfg;
    sv->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&sv->device) != cudaSuccess || cudaMalloc(&sv->d_pool, cfg.pool_bytes) != cudaSuccess) {
        destroy_server(sv);
        record_error("server pool allocation");
        return BN_ENOMEM;
    }
    sv->alloc = new PoolAllocator(cfg.pool_bytes);
    // Size classes the cost model can pick, and per-slot transform plans.
    for (uint32_t key = 0; (1u << key) <= BN_MUL_MAX_LIMBS * 2 && key < 15; ++key) {
        const uint32_t n = std::min(1u << key, BN_ADD_MAX_LIMBS);
        AddClass ac;
        if (add_batch_class(ac, n) == BN_OK) sv->add_classes[key] = ac;
        if ((1u << key) <= BN_MUL_MAX_LIMBS) {
            QuadClass qc;
            if (quad_batch_class(qc, 8, n, 256) == BN_OK) sv->quad_classes[key] = qc;
        }
    }
    sv->slots.resize(cfg.max_inflight);
    for (Slot &s : sv->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&s.h_items, cfg.max_batch * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaMalloc(&s.d_items, cfg.max_batch * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaMalloc(&s.d_queues, kMaxClasses * 4);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_bind, sizeof(BatchBinding));
        const BatchBinding hb{nullptr, nullptr, reinterpret_cast<uint32_t *>(sv->d_pool)};
        if (e == cudaSuccess) e = cudaMemcpy(s.d_bind, &hb, sizeof hb, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            destroy_server(sv);
            record_error("server slot set-up");
            return BN_ECUDA;
        }
        for (uint32_t l = 11; l <= 15; ++l) slot_plan(s, false, l);  // transforms the
        for (uint32_t l = 10; l <= 14; ++l) slot_plan(s, true, l);   // cost model can pick
        for (uint32_t l = 9; l <= 14; ++l) slot_plan3(s, l);
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return BN_OK;
}

bn_status bn_server_submit(bn_server sv, const bn_request *reqs, uint32_t count, uint64_t *tickets) {
    using namespace bn;
    if (!sv || (count && (!reqs || !tickets))) return BN_EINVAL;
    for (uint32_t i = 0; i < count; ++i) {
        const bn_request &r = reqs[i];
        const uint32_t lim = r.op == BN_OP_ADD ? BN_ADD_MAX_LIMBS : BN_MUL_MAX_LIMBS;
        if (r.reserved || r.op > BN_OP_MUL_AUTO || !r.na || !r.nb || !r.a || !r.b ||
            ((uintptr_t)r.a % 4) || ((uintptr_t)r.b % 4) || r.na > lim || r.nb > lim) {
            record_error("bad request (op, size, or null/unaligned operand)");
            return BN_EINVAL;
        }
    }
    const double now = sv->now_us();
    {
        std::lock_guard<std::mutex> lk(sv->queue_mutex);
        for (uint32_t i = 0; i < count; ++i) {
            const bn_request &r = reqs[i];
            const uint64_t t = sv->next_ticket++;
            tickets[i] = t;
            const uint32_t nout = r.op == BN_OP_ADD ? std::max(r.na, r.nb) + 1 : r.na + r.nb;
            sv->pending.push_back({t, r.op, r.na, r.nb, nout, r.a, r.b, r.arrival_us < 0 ? now : r.arrival_us});
        }
    }
    sv->submitted += count;
    sv->queue_cv.notify_one();
    return BN_OK;
}

bn_status bn_server_poll(bn_server sv, bn_completion *out, uint32_t max, uint32_t *n) {
    if (!sv || !n || (max && !out)) return BN_EINVAL;
    if (sv->worker_error) {
        bn::record_error("a server launch failed");
        return BN_ECUDA;
    }
    std::lock_guard<std::mutex> lk(sv->done_mutex);
    const uint32_t k = (uint32_t)std::min<size_t>(max, sv->completed.size());
    std::copy(sv->completed.begin(), sv->completed.begin() + k, out);
    sv->completed.erase(sv->completed.begin(), sv->completed.begin() + k);
    *n = k;
    return BN_OK;
}

bn_status bn_server_release(bn_server sv, const uint64_t *tickets, uint32_t count) {
    if (!sv || (count && !tickets)) return BN_EINVAL;
    std::lock_guard<std::mutex> pl(sv->pool_mutex);
    bn_status st = BN_OK;
    for (uint32_t i = 0; i < count; ++i) {
        auto it = sv->results.find(tickets[i]);
        if (it == sv->results.end()) {
            bn::record_error("unknown or already released ticket");
            st = BN_EINVAL;
            continue;
        }
        sv->alloc->release(it->second.first, it->second.second);
        sv->results.erase(it);
    }
    return st;
}

bn_status bn_server_drain(bn_server sv, double timeout_s) {
    if (!sv) return BN_EINVAL;
    const auto end = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        bool empty;
        {
            std::lock_guard<std::mutex> lk(sv->queue_mutex);
            empty = sv->pending.empty();
        }
        if (empty && sv->inflight == 0) return sv->worker_error ? BN_ECUDA : BN_OK;
        if (std::chrono::steady_clock::now() > end) {
            bn::record_error("drain timed out (results may be waiting for pool memory)");
            return BN_ETIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

double bn_server_now_us(bn_server sv) { return sv ? sv->now_us() : 0.0; }

bn_status bn_server_get_stats(bn_server sv, bn_server_stats *out) {
    if (!sv || !out) return BN_EINVAL;
    *out = {};
    out->submitted = sv->submitted;
    out->completed = sv->completed_count;
    out->batches = sv->batches;
    {
        std::lock_guard<std::mutex> pl(sv->pool_mutex);
        out->pool_high_water = sv->alloc->high_water();
    }
    out->max_inflight_seen = sv->max_inflight_seen;
    return BN_OK;
}

bn_status bn_server_destroy(bn_server sv) {
    if (!sv) return BN_OK;
    sv->stop = true;
    sv->queue_cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    const cudaError_t e = cudaDeviceSynchronize();
    destroy_server(sv);
    return e == cudaSuccess ? BN_OK : BN_ECUDA;
}

}  // extern "C"
