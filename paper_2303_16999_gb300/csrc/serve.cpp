// Serving loop: resident sparse weights, HBM-budget admission, continuous
// batching of column-block requests into persistent tensor-core launches on
// several in-flight streams, completion tracking and latency statistics.
// (The paper benchmarks single products; this is the deployment form the
// library adds around them.)
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/spmm_serve.h"
#include "spmm_internal.h"

using namespace spmm;

namespace {

double now_us() {
    return std::chrono::duration<double, std::micro>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// The batcher spins (yielding) this long after its last launch before it
// blocks on its condition variable.
constexpr double kSpinUs = 200.0;

// First-fit allocator over the staging pool, in 256-byte units.
struct Pool {
    std::map<int64_t, int64_t> free_;  // offset -> length (bytes)
    void init(int64_t size) { free_ = {{0, size}}; }
    bool alloc(int64_t bytes, int64_t *off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const int64_t rest = it->second - bytes;
                const int64_t noff = it->first + bytes;
                free_.erase(it);
                if (rest > 0) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(int64_t off, int64_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum ReqState { kQueued, kLaunched, kDone };

struct Req {
    int32_t w = 0;
    const void *hX = nullptr;
    void *hY = nullptr;
    int64_t n = 0, ldx = 0;
    double t_arr = 0, t_done = 0;
    ReqState state = kQueued;
    spmm_status st = SPMM_OK;
    int64_t xoff = -1, yoff = -1, xbytes = 0, ybytes = 0;
};

struct Launch {
    int slot = 0;
    std::vector<uint64_t> reqs;
    std::vector<int32_t> busy_weights;
};

size_t es_of(const spmm_plan *p) { return dtype_size(p->xdt); }

bool batchable(const spmm_plan *p) {
    return p->kernel == SPMM_KERNEL_TC && (p->xdt == SPMM_F16 || p->xdt == SPMM_BF16);
}

}  // namespace

struct serve_server {
    serve_config cfg{};
    int dev = 0;
    char *pool_base = nullptr;
    Pool pool;
    std::vector<spmm_plan *> weights;
    std::vector<int> weight_busy;
    std::mutex mu;
    std::condition_variable cv_batcher, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Req> reqs;
    uint64_t next_id = 1;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<bool> slot_busy;
    std::vector<Launch> inflight;
    std::thread batcher, completer;
    bool stop = false;
    // statistics
    std::vector<double> lat;
    int64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, failed = 0, launches = 0;
    double sum_reqs = 0, sum_cols = 0, first_arr = -1, last_done = -1, flops_done = 0;

    void fail_locked(uint64_t id, spmm_status st) {
        Req &r = reqs[id];
        r.state = kDone;
        r.st = st;
        ++failed;
    }

    void batcher_loop();
    void completer_loop();
};

void serve_server::batcher_loop() {
    cudaSetDevice(dev);
    std::unique_lock<std::mutex> lk(mu);
    double last_active = now_us();
    while (!stop) {
        int slot = -1;
        for (int i = 0; i < cfg.max_inflight; ++i)
            if (!slot_busy[i]) {
                slot = i;
                break;
            }
        if (queue.empty() || slot < 0) {
            // wait for a request or a free slot: spin (yielding) for a while
            // after the last activity, then block; a blocked thread's wake-up
            // would add its latency to the next request's
            if (now_us() - last_active < kSpinUs) {
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                cv_batcher.wait(lk);
            }
            continue;
        }
        last_active = now_us();
        // admit from the head of the queue while the launch and the budget allow
        Launch L;
        L.slot = slot;
        int64_t cols = 0;
        bool tc = false;
        while (!queue.empty()) {
            const uint64_t id = queue.front();
            Req &r = reqs[id];
            spmm_plan *p = weights[r.w];
            const bool b = batchable(p);
            if (!L.reqs.empty() && (!b || !tc)) break;
            if ((int)L.reqs.size() >= cfg.max_batch || cols + r.n > cfg.max_batch_n) break;
            // a weight with split rows (shared workspace) or a non-batched
            // weight runs in one launch at a time, once per launch
            const bool exclusive = !b || p->n_red > 0;
            if (exclusive) {
                if (weight_busy[r.w]) break;
                bool dup = false;
                for (uint64_t o : L.reqs) dup |= reqs[o].w == r.w;
                if (dup) break;
            }
            if (cfg.inject_alloc_fail) {
                queue.pop_front();
                fail_locked(id, SPMM_ERR_OOM);
                cv_done.notify_all();
                continue;
            }
            int64_t xo, yo;
            if (!pool.alloc(r.xbytes, &xo)) break;
            if (!pool.alloc(r.ybytes, &yo)) {
                pool.release(xo, r.xbytes);
                break;
            }
            r.xoff = xo;
            r.yoff = yo;
            queue.pop_front();
            L.reqs.push_back(id);
            cols += r.n;
            tc = b;
            ++admitted;
            if (exclusive) {
                L.busy_weights.push_back(r.w);
                weight_busy[r.w] = 1;
            }
            if (!b) break;  // non-batched weights: one request per launch
        }
        if (L.reqs.empty()) {
            // budget full: wait for a completion to free staging
            cv_batcher.wait(lk);
            continue;
        }
        slot_busy[slot] = true;
        // snapshot what the launch needs, then enqueue without the lock
        const int cnt = (int)L.reqs.size();
        std::vector<spmm_plan *> plans(cnt);
        std::vector<const void *> xs(cnt);
        std::vector<void *> ys(cnt);
        std::vector<int64_t> ns(cnt), lxs(cnt), lys(cnt);
        std::vector<const void *> hx(cnt);
        std::vector<void *> hy(cnt);
        for (int i = 0; i < cnt; ++i) {
            Req &r = reqs[L.reqs[i]];
            r.state = kLaunched;
            plans[i] = weights[r.w];
            xs[i] = pool_base + r.xoff;
            ys[i] = pool_base + r.yoff;
            ns[i] = r.n;
            lxs[i] = r.ldx;
            lys[i] = r.n;
            hx[i] = r.hX;
            hy[i] = r.hY;
        }
        lk.unlock();
        if (cfg.inject_delay_us > 0)
            std::this_thread::sleep_for(std::chrono::microseconds(cfg.inject_delay_us));
        cudaStream_t s = streams[slot];
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < cnt && e == cudaSuccess; ++i) {
            // X arrives dense (ld = n) but the tensor map needs 16-byte rows:
            // one contiguous copy, then (n not a multiple of 8) a re-stride
            // on the device out of the Y staging, which is free until the
            // product and at least as large when m >= k; a strided copy of
            // k short rows is the fallback
            const size_t es = es_of(plans[i]);
            const int64_t k = plans[i]->k, m = plans[i]->m;
            if (lxs[i] == ns[i]) {
                e = cudaMemcpyAsync((void *)xs[i], hx[i], k * ns[i] * es, cudaMemcpyHostToDevice, s);
            } else if (m >= k) {
                e = cudaMemcpyAsync(ys[i], hx[i], k * ns[i] * es, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess)
                    e = launch_restride(ys[i], (void *)xs[i], k, ns[i], lxs[i], es, s);
            } else {
                e = cudaMemcpy2DAsync((void *)xs[i], lxs[i] * es, hx[i], ns[i] * es, ns[i] * es, k,
                                      cudaMemcpyHostToDevice, s);
            }
        }
        if (e == cudaSuccess) {
            if (tc) {
                e = launch_tc_batch(cnt, plans.data(), xs.data(), ns.data(), lxs.data(), ys.data(),
                                    lys.data(), s, false);
                for (int i = 0; i < cnt && e == cudaSuccess; ++i)
                    if (plans[i]->n_red > 0) e = launch_reduce(plans[i], ns[i], ys[i], lys[i], s);
            } else {
                spmm_status st = spmm_run(plans[0], nullptr, nullptr, nullptr, xs[0], ns[0],
                                          lxs[0], ys[0], lys[0], s);
                if (st != SPMM_OK) e = cudaErrorUnknown;
            }
        }
        for (int i = 0; i < cnt && e == cudaSuccess; ++i) {
            const size_t es = es_of(plans[i]);
            e = cudaMemcpyAsync(hy[i], ys[i], plans[i]->m * ns[i] * es, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaEventRecord(events[slot], s);
        lk.lock();
        ++launches;
        sum_reqs += cnt;
        sum_cols += cols;
        if (e != cudaSuccess) {
            // nothing of this launch will complete normally: finish it here
            cudaStreamSynchronize(s);
            for (uint64_t id : L.reqs) {
                Req &r = reqs[id];
                pool.release(r.xoff, r.xbytes);
                pool.release(r.yoff, r.ybytes);
                fail_locked(id, SPMM_ERR_CUDA);
            }
            for (int32_t w : L.busy_weights) weight_busy[w] = 0;
            slot_busy[slot] = false;
            cv_done.notify_all();
            continue;
        }
        inflight.push_back(std::move(L));
        cv_done.notify_all();
    }
}

void serve_server::completer_loop() {
    cudaSetDevice(dev);
    // While launches are in flight their events are polled back to back
    // (yielding between rounds): a timed sleep here lasted about 55 us (a
    // Linux thread's default timer slack is 50 us), which every request's
    // latency paid.
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        if (inflight.empty()) {
            if (stop) break;
            cv_done.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        bool any = false;
        for (size_t i = 0; i < inflight.size();) {
            Launch &L = inflight[i];
            if (cudaEventQuery(events[L.slot]) == cudaErrorNotReady) {
                ++i;
                continue;
            }
            const double t = now_us();
            for (uint64_t id : L.reqs) {
                Req &r = reqs[id];
                const spmm_plan *p = weights[r.w];
                r.state = kDone;
                r.t_done = t;
                pool.release(r.xoff, r.xbytes);
                pool.release(r.yoff, r.ybytes);
                lat.push_back(t - r.t_arr);
                ++completed;
                flops_done += 2.0 * (double)p->nnzb * p->b * p->b * (double)r.n;
                last_done = std::max(last_done, t);
            }
            for (int32_t w : L.busy_weights) weight_busy[w] = 0;
            slot_busy[L.slot] = false;
            inflight.erase(inflight.begin() + i);
            any = true;
        }
        if (any) {
            cv_done.notify_all();
            cv_batcher.notify_all();
        } else {
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        }
    }
}

extern "C" {

spmm_status serve_create(const serve_config *cfg, serve_server **out) {
    if (!cfg || !out || cfg->hbm_budget_bytes <= 0 || cfg->max_inflight < 1 ||
        cfg->max_inflight > 8 || cfg->max_batch < 1 || cfg->max_batch > kMaxBatchProblems ||
        cfg->max_batch_n < 1 || cfg->inject_delay_us < 0) {
        set_error("serve_create: budget > 0, 1 <= max_inflight <= 8, 1 <= max_batch <= %d, "
                  "max_batch_n >= 1", kMaxBatchProblems);
        return SPMM_ERR_ARG;
    }
    *out = nullptr;
    serve_server *s = new (std::nothrow) serve_server();
    if (!s) return SPMM_ERR_OOM;
    s->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&s->dev);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->pool_base, cfg->hbm_budget_bytes);
    if (e != cudaSuccess) {
        delete s;
        set_error("serve_create: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SPMM_ERR_OOM : SPMM_ERR_CUDA;
    }
    s->pool.init(cfg->hbm_budget_bytes);
    s->streams.resize(cfg->max_inflight);
    s->events.resize(cfg->max_inflight);
    s->slot_busy.assign(cfg->max_inflight, false);
    for (int i = 0; i < cfg->max_inflight && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaFree(s->pool_base);
        delete s;
        set_error("serve_create: %s", cudaGetErrorString(e));
        return SPMM_ERR_CUDA;
    }
    s->batcher = std::thread([s] { s->batcher_loop(); });
    s->completer = std::thread([s] { s->completer_loop(); });
    *out = s;
    return SPMM_OK;
}

spmm_status serve_register_weight(serve_server *s, spmm_plan *p, int32_t *weight_id) {
    if (!s || !p || !weight_id || p->host_only || p->mode != SPMM_STATIC || !p->packed) {
        set_error("serve_register_weight: a device static plan with packed values is required");
        return SPMM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    *weight_id = (int32_t)s->weights.size();
    s->weights.push_back(p);
    s->weight_busy.push_back(0);
    return SPMM_OK;
}

spmm_status serve_submit(serve_server *s, int32_t w, const void *h_X, int64_t n, void *h_Y,
                         uint64_t *ticket) {
    if (!s || !h_X || !h_Y || !ticket) {
        set_error("serve_submit: server, X, Y and ticket required");
        return SPMM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (w < 0 || w >= (int32_t)s->weights.size()) {
        set_error("serve_submit: unknown weight %d", w);
        return SPMM_ERR_ARG;
    }
    const spmm_plan *p = s->weights[w];
    if (n < 1 || n > p->n_max || n > s->cfg.max_batch_n) {
        set_error("serve_submit: n=%lld outside [1, min(n_max, max_batch_n)]", (long long)n);
        return SPMM_ERR_SHAPE;
    }
    Req r;
    r.w = w;
    r.hX = h_X;
    r.hY = h_Y;
    r.n = n;
    r.ldx = (n + 7) / 8 * 8;  // 16-byte rows for the tensor map
    const size_t es = es_of(p);
    r.xbytes = p->k * r.ldx * (int64_t)es;
    r.ybytes = p->m * n * (int64_t)es;
    if ((r.xbytes + 255) / 256 * 256 + (r.ybytes + 255) / 256 * 256 > s->cfg.hbm_budget_bytes) {
        ++s->rejected;
        set_error("serve_submit: request needs %lld staging bytes, budget is %lld",
                  (long long)(r.xbytes + r.ybytes), (long long)s->cfg.hbm_budget_bytes);
        return SPMM_ERR_CAPACITY;
    }
    r.t_arr = now_us();
    if (s->first_arr < 0) s->first_arr = r.t_arr;
    const uint64_t id = s->next_id++;
    s->reqs.emplace(id, r);
    s->queue.push_back(id);
    ++s->submitted;
    *ticket = id;
    s->cv_batcher.notify_one();
    return SPMM_OK;
}

spmm_status serve_wait(serve_server *s, uint64_t ticket, int64_t timeout_ms) {
    if (!s) return SPMM_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("serve_wait: unknown ticket %llu", (unsigned long long)ticket);
        return SPMM_ERR_ARG;
    }
    auto done = [&] { return s->reqs[ticket].state == kDone; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        set_error("serve_wait: request %llu not done after %lld ms", (unsigned long long)ticket,
                  (long long)timeout_ms);
        return SPMM_ERR_TIMEOUT;
    }
    const spmm_status st = s->reqs[ticket].st;
    s->reqs.erase(ticket);
    return st;
}

static double pct(std::vector<double> v, double q) {
    if (v.empty()) return 0;
    const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
}

spmm_status serve_stats(serve_server *s, serve_stats_t *o) {
    if (!s || !o) return SPMM_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    serve_stats_t r{};
    r.submitted = s->submitted;
    r.admitted = s->admitted;
    r.completed = s->completed;
    r.rejected = s->rejected;
    r.failed = s->failed;
    r.queued = (int64_t)s->queue.size();
    for (const Launch &L : s->inflight) r.in_flight += (int64_t)L.reqs.size();
    r.launches = s->launches;
    r.mean_requests_per_launch = s->launches ? s->sum_reqs / s->launches : 0;
    r.mean_cols_per_launch = s->launches ? s->sum_cols / s->launches : 0;
    r.p50_us = pct(s->lat, 0.50);
    r.p99_us = pct(s->lat, 0.99);
    double sum = 0, mx = 0;
    for (double v : s->lat) {
        sum += v;
        mx = std::max(mx, v);
    }
    r.mean_us = s->lat.empty() ? 0 : sum / (double)s->lat.size();
    r.max_us = mx;
    r.span_s = (s->first_arr >= 0 && s->last_done >= 0) ? (s->last_done - s->first_arr) * 1e-6 : 0;
    r.throughput_rps = r.span_s > 0 ? (double)s->completed / r.span_s : 0;
    r.tflops_nz = r.span_s > 0 ? s->flops_done / r.span_s / 1e12 : 0;
    *o = r;
    return SPMM_OK;
}

spmm_status serve_reset_stats(serve_server *s) {
    if (!s) return SPMM_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat.clear();
    s->submitted = s->admitted = s->completed = s->rejected = s->failed = s->launches = 0;
    s->sum_reqs = s->sum_cols = s->flops_done = 0;
    s->first_arr = s->last_done = -1;
    return SPMM_OK;
}

spmm_status serve_replay(serve_server *s, int64_t count, const double *t_arr, const int32_t *w,
                         const int64_t *n, const void *const *hX, void *const *hY,
                         serve_stats_t *out) {
    if (!s || count < 0 || (count > 0 && (!t_arr || !w || !n || !hX || !hY)) || !out) {
        set_error("serve_replay: server, arrays and out required");
        return SPMM_ERR_ARG;
    }
    spmm_status st = serve_reset_stats(s);
    if (st != SPMM_OK) return st;
    std::vector<uint64_t> tickets;
    tickets.reserve(count);
    spmm_status first = SPMM_OK;
    const double t0 = now_us();
    for (int64_t i = 0; i < count; ++i) {
        const double due = t0 + t_arr[i] * 1e6;
        while (now_us() < due) {
        }
        uint64_t t = 0;
        st = serve_submit(s, w[i], hX[i], n[i], hY[i], &t);
        if (st != SPMM_OK) {
            if (first == SPMM_OK) first = st;
            continue;
        }
        tickets.push_back(t);
    }
    for (uint64_t t : tickets) {
        st = serve_wait(s, t, -1);
        if (st != SPMM_OK && first == SPMM_OK) first = st;
    }
    st = serve_stats(s, out);
    return first != SPMM_OK ? first : st;
}

void serve_destroy(serve_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (uint64_t id : s->queue) s->fail_locked(id, SPMM_ERR_ARG);
        s->queue.clear();
    }
    s->cv_batcher.notify_all();
    s->cv_done.notify_all();
    if (s->batcher.joinable()) s->batcher.join();
    if (s->completer.joinable()) s->completer.join();
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
    cudaFree(s->pool_base);
    delete s;
}

}  // extern "C"
