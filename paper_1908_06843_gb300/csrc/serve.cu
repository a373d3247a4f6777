// serve.cu -- encoding service with continuous batching ("Model.inference",
// paper Sec. 3, run as a service).
//
// A host scheduler thread owns n_slots device slots.  Each slot has its own
// CUDA stream, device input/output buffers, pinned host staging and per-slot
// scratch; the dictionary constants (Gram matrix, norms, BF16 operand image,
// GSC subset table) are computed once at start and shared read-only.  Whenever
// a slot is free and requests are waiting, the scheduler packs waiting
// requests in arrival order into that slot (up to slot_points points), copies
// them in, launches the encode kernels on the slot's stream and queues the
// copy back; it then looks for the next free slot without waiting, so several
// batches are on the GPU at once and a request that arrives while others run
// is admitted as soon as a slot frees.  Completion is detected with
// cudaEventQuery (no device-side spin).  Per-point results do not depend on the
// batch or slot a point lands in (every kernel treats points independently).
#include "internal.cuh"

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <time.h>
#include <unordered_map>
#include <vector>

namespace prosper {

static int64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

struct Request {
    uint64_t ticket;
    int n;
    std::vector<float> y;
    int64_t t_submit;
};

struct Result {
    bool done = false;
    int status = PROSPER_OK;
    int n = 0;
    std::vector<int16_t> sel, map;
    std::vector<float> smean, mapp, logz;
    int64_t t_submit = 0, t_done = 0;
};

struct Slot {
    prosper_ctx sub;              // copy of the context with this slot's scratch
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    float *d_y = nullptr, *h_y = nullptr;
    int16_t *d_sel = nullptr, *d_map = nullptr, *h_sel = nullptr, *h_map = nullptr;
    float *d_smean = nullptr, *d_mapp = nullptr, *d_logz = nullptr;
    float *h_smean = nullptr, *h_mapp = nullptr, *h_logz = nullptr;
    bool busy = false;
    std::vector<std::pair<uint64_t, int>> members;   // (ticket, n) in packing order
    int launch_rc = PROSPER_OK;
};

struct ServeState {
    prosper_ctx *ctx = nullptr;
    prosper_params params{};
    int n_slots = 0, slot_points = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    std::atomic<bool> stop{false};
    std::thread worker;
};

static void free_slot(Slot &s) {
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.done) cudaEventDestroy(s.done);
    cudaFree(s.d_y); cudaFree(s.d_sel); cudaFree(s.d_map); cudaFree(s.d_smean);
    cudaFree(s.d_mapp); cudaFree(s.d_logz);
    cudaFree(s.sub.sel); cudaFree(s.sub.selp); cudaFree(s.sub.yy); cudaFree(s.sub.d_status);
    if (s.h_y) cudaFreeHost(s.h_y);
    if (s.h_sel) cudaFreeHost(s.h_sel);
    if (s.h_map) cudaFreeHost(s.h_map);
    if (s.h_smean) cudaFreeHost(s.h_smean);
    if (s.h_mapp) cudaFreeHost(s.h_mapp);
    if (s.h_logz) cudaFreeHost(s.h_logz);
}

// encode one packed batch of n points on the slot's stream (no constants rebuild)
static int launch_slot(ServeState *S, Slot &s, int n) {
    prosper_ctx *c = &s.sub;
    const prosper_params *p = &S->params;
    cudaStream_t st = s.stream;
    const int D = c->D, Hp = c->Hp, g = c->gamma;
    PROSPER_CUDA_TRY(cudaMemcpyAsync(s.d_y, s.h_y, sizeof(float) * (size_t)n * D,
                                     cudaMemcpyHostToDevice, st));
    int rc;
    if (linear_model(c->model)) {
        rc = launch_linear_proj(c, s.d_y, p->W, n, st);
        if (!rc)
            rc = launch_linear_states(c, p->theta, n, 0, nullptr, s.d_sel, s.d_smean,
                                      g > 0 ? s.d_map : nullptr, nullptr, s.d_mapp, s.d_logz, st);
    } else if (max_model(c->model)) {
        rc = launch_mca_estep(c, p->W, p->theta, s.d_y, n, nullptr, s.d_sel, s.d_smean,
                              g > 0 ? s.d_map : nullptr, s.d_mapp, s.d_logz, st);
    } else {
        rc = launch_gsc_estep(c, p, s.d_y, n, nullptr, s.d_sel, s.d_smean, g > 0 ? s.d_map : nullptr,
                              s.d_mapp, s.d_logz, st);
    }
    if (rc) return rc;
    PROSPER_CUDA_TRY(cudaMemcpyAsync(s.h_sel, s.d_sel, sizeof(int16_t) * (size_t)n * Hp, cudaMemcpyDeviceToHost, st));
    PROSPER_CUDA_TRY(cudaMemcpyAsync(s.h_smean, s.d_smean, sizeof(float) * (size_t)n * Hp, cudaMemcpyDeviceToHost, st));
    if (g > 0)
        PROSPER_CUDA_TRY(cudaMemcpyAsync(s.h_map, s.d_map, sizeof(int16_t) * (size_t)n * g, cudaMemcpyDeviceToHost, st));
    PROSPER_CUDA_TRY(cudaMemcpyAsync(s.h_mapp, s.d_mapp, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    PROSPER_CUDA_TRY(cudaMemcpyAsync(s.h_logz, s.d_logz, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    PROSPER_CUDA_TRY(cudaEventRecord(s.done, st));
    return PROSPER_OK;
}

static void scheduler(ServeState *S) {
    cudaSetDevice(S->ctx->device);
    const int D = S->ctx->D, Hp = S->ctx->Hp, g = S->ctx->gamma;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progressed = false;
        // 1. retire finished slots
        for (auto &s : S->slots) {
            if (!s.busy) continue;
            lk.unlock();
            const cudaError_t q = s.launch_rc ? cudaSuccess : cudaEventQuery(s.done);
            lk.lock();
            if (q == cudaErrorNotReady) continue;
            const int64_t t = now_ns();
            int off = 0;
            for (auto &mem : s.members) {
                Result &r = S->results[mem.first];
                const int n = mem.second;
                if (s.launch_rc || q != cudaSuccess) {
                    r.status = s.launch_rc ? s.launch_rc : PROSPER_ECUDA;
                } else {
                    r.sel.assign(s.h_sel + (size_t)off * Hp, s.h_sel + (size_t)(off + n) * Hp);
                    r.smean.assign(s.h_smean + (size_t)off * Hp, s.h_smean + (size_t)(off + n) * Hp);
                    if (g > 0) r.map.assign(s.h_map + (size_t)off * g, s.h_map + (size_t)(off + n) * g);
                    r.mapp.assign(s.h_mapp + off, s.h_mapp + off + n);
                    r.logz.assign(s.h_logz + off, s.h_logz + off + n);
                }
                r.done = true;
                r.t_done = t;
                off += n;
            }
            s.members.clear();
            s.busy = false;
            progressed = true;
            S->cv_done.notify_all();
        }
        // 2. pack waiting requests into free slots
        for (auto &s : S->slots) {
            if (s.busy || S->queue.empty()) continue;
            int n = 0;
            while (!S->queue.empty() && n + S->queue.front().n <= S->slot_points) {
                Request &rq = S->queue.front();
                std::memcpy(s.h_y + (size_t)n * D, rq.y.data(), sizeof(float) * (size_t)rq.n * D);
                s.members.emplace_back(rq.ticket, rq.n);
                n += rq.n;
                S->queue.pop_front();
            }
            s.busy = true;
            lk.unlock();
            s.launch_rc = launch_slot(S, s, n);
            lk.lock();
            progressed = true;
        }
        if (S->stop.load() && S->queue.empty()) {
            bool any = false;
            for (auto &s : S->slots) any |= s.busy;
            if (!any) break;
        }
        if (!progressed) {
            bool any_busy = false;
            for (auto &s : S->slots) any_busy |= s.busy;
            if (any_busy) {
                // GPU work in flight: poll again shortly
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
}

}  // namespace prosper

using namespace prosper;

extern "C" {

int prosper_serve_start(prosper_ctx *c, const prosper_params *p, int n_slots, int slot_points) {
    if (!c || !p || !p->W || !p->theta) { set_error("serve_start: bad arguments"); return PROSPER_EINVAL; }
    if (c->serve) { set_error("serve_start: already running"); return PROSPER_ESTATE; }
    if (n_slots < 1 || n_slots > 64 || slot_points < 1 || slot_points > (1 << 22)) {
        set_error("serve_start: n_slots in [1, 64], slot_points in [1, 2^22]");
        return PROSPER_EINVAL;
    }
    if (c->model == PROSPER_GSC && (!p->mu || !p->psi)) { set_error("serve_start: GSC needs mu, psi"); return PROSPER_EINVAL; }
    ServeState *S = new ServeState();
    S->ctx = c;
    S->params = *p;
    S->n_slots = n_slots;
    S->slot_points = slot_points;
    S->slots.resize(n_slots);
    // resident constants, computed once on the default stream
    int rc = PROSPER_OK;
    if (linear_model(c->model)) rc = launch_bsc_prep(c, p->W, nullptr);
    else if (c->model == PROSPER_GSC) rc = launch_gsc_prep(c, p, nullptr);
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) { set_error("serve_start: constants failed"); rc = PROSPER_ECUDA; }
    const size_t sp = (size_t)slot_points, D = c->D, Hp = c->Hp, g = c->gamma > 0 ? c->gamma : 1;
    for (auto &s : S->slots) {
        if (rc) break;
        s.sub = *c;
        s.sub.serve = nullptr;
        s.sub.trace = nullptr;
        s.sub.sel = nullptr; s.sub.selp = nullptr; s.sub.yy = nullptr; s.sub.es = nullptr;
        s.sub.d_status = nullptr;
        s.sub.chunk = slot_points;
        bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMalloc(&s.d_y, sizeof(float) * sp * D) == cudaSuccess &&
                  cudaMalloc(&s.d_sel, sizeof(int16_t) * sp * Hp) == cudaSuccess &&
                  cudaMalloc(&s.d_map, sizeof(int16_t) * sp * g) == cudaSuccess &&
                  cudaMalloc(&s.d_smean, sizeof(float) * sp * Hp) == cudaSuccess &&
                  cudaMalloc(&s.d_mapp, sizeof(float) * sp) == cudaSuccess &&
                  cudaMalloc(&s.d_logz, sizeof(float) * sp) == cudaSuccess &&
                  cudaMalloc(&s.sub.d_status, sizeof(unsigned)) == cudaSuccess &&
                  cudaMallocHost(&s.h_y, sizeof(float) * sp * D) == cudaSuccess &&
                  cudaMallocHost(&s.h_sel, sizeof(int16_t) * sp * Hp) == cudaSuccess &&
                  cudaMallocHost(&s.h_map, sizeof(int16_t) * sp * g) == cudaSuccess &&
                  cudaMallocHost(&s.h_smean, sizeof(float) * sp * Hp) == cudaSuccess &&
                  cudaMallocHost(&s.h_mapp, sizeof(float) * sp) == cudaSuccess &&
                  cudaMallocHost(&s.h_logz, sizeof(float) * sp) == cudaSuccess;
        if (ok && linear_model(c->model))
            ok = cudaMalloc(&s.sub.sel, sizeof(int32_t) * sp * SEL_STRIDE) == cudaSuccess &&
                 cudaMalloc(&s.sub.selp, sizeof(float) * sp * SEL_STRIDE) == cudaSuccess &&
                 cudaMalloc(&s.sub.yy, sizeof(float) * sp * 2) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            set_error("serve_start: slot allocation failed");
            rc = PROSPER_ENOMEM;
        } else if (cudaMemset(s.sub.d_status, 0, sizeof(unsigned)) != cudaSuccess) {
            rc = PROSPER_ECUDA;
        }
    }
    if (rc) {
        for (auto &s : S->slots) free_slot(s);
        delete S;
        return rc;
    }
    c->serve = S;
    S->worker = std::thread(scheduler, S);
    return PROSPER_OK;
}

int prosper_serve_submit(prosper_ctx *c, const float *Y_host, int n, uint64_t *ticket) {
    if (!c || !c->serve) { set_error("serve_submit: service not started"); return PROSPER_ESTATE; }
    ServeState *S = c->serve;
    if (n < 1 || !Y_host || !ticket) { set_error("serve_submit: bad arguments"); return PROSPER_EINVAL; }
    if (n > S->slot_points) {
        set_error("serve_submit: request of %d points exceeds the slot size %d", n, S->slot_points);
        return PROSPER_EBUSY;
    }
    Request rq;
    rq.n = n;
    rq.y.assign(Y_host, Y_host + (size_t)n * c->D);
    rq.t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop.load()) { set_error("serve_submit: stopping"); return PROSPER_ESTATE; }
        rq.ticket = S->next_ticket++;
        Result &r = S->results[rq.ticket];
        r.n = n;
        r.t_submit = rq.t_submit;
        *ticket = rq.ticket;
        S->queue.push_back(std::move(rq));
    }
    S->cv_work.notify_one();
    return PROSPER_OK;
}

int prosper_serve_wait(prosper_ctx *c, uint64_t ticket, int timeout_ms, int16_t *sel_host,
                       float *s_mean_host, int16_t *map_idx_host, float *map_p_host,
                       float *logZ_host, int64_t *t_submit_ns, int64_t *t_done_ns) {
    if (!c || !c->serve) { set_error("serve_wait: service not started"); return PROSPER_ESTATE; }
    ServeState *S = c->serve;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) { set_error("serve_wait: unknown ticket"); return PROSPER_EINVAL; }
    auto ready = [&] { return S->results[ticket].done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        set_error("serve_wait: ticket %llu not finished within %d ms", (unsigned long long)ticket, timeout_ms);
        return PROSPER_ETIMEOUT;
    }
    Result r = std::move(S->results[ticket]);
    S->results.erase(ticket);
    lk.unlock();
    if (r.status) { set_error("serve_wait: batch failed"); return r.status; }
    const int Hp = c->Hp, g = c->gamma;
    if (sel_host) std::memcpy(sel_host, r.sel.data(), sizeof(int16_t) * r.sel.size());
    if (s_mean_host) std::memcpy(s_mean_host, r.smean.data(), sizeof(float) * r.smean.size());
    if (map_idx_host && g > 0) std::memcpy(map_idx_host, r.map.data(), sizeof(int16_t) * r.map.size());
    if (map_p_host) std::memcpy(map_p_host, r.mapp.data(), sizeof(float) * r.mapp.size());
    if (logZ_host) std::memcpy(logZ_host, r.logz.data(), sizeof(float) * r.logz.size());
    (void)Hp;
    if (t_submit_ns) *t_submit_ns = r.t_submit;
    if (t_done_ns) *t_done_ns = r.t_done;
    return PROSPER_OK;
}

int prosper_serve_loadgen(prosper_ctx *c, const float *Y_pool_host, int64_t pool_points, int n_req,
                          const int32_t *sizes, const int64_t *offsets, const int64_t *arrival_ns,
                          int64_t *t_submit_ns, int64_t *t_observed_ns, int64_t *t_done_ns) {
    if (!c || !c->serve) { set_error("serve_loadgen: service not started"); return PROSPER_ESTATE; }
    if (!Y_pool_host || n_req < 0 || !sizes || !offsets || !arrival_ns || !t_submit_ns || !t_observed_ns) {
        set_error("serve_loadgen: bad arguments");
        return PROSPER_EINVAL;
    }
    for (int i = 0; i < n_req; ++i)
        if (sizes[i] < 1 || sizes[i] > c->serve->slot_points || offsets[i] < 0 ||
            offsets[i] + sizes[i] > pool_points) {
            set_error("serve_loadgen: request %d (%d points at %lld) outside the pool or the slot size", i,
                      sizes[i], (long long)offsets[i]);
            return PROSPER_EINVAL;
        }
    const int D = c->D, Hp = c->Hp, g = c->gamma > 0 ? c->gamma : 1;
    std::vector<uint64_t> tickets(n_req, 0);
    std::vector<std::atomic<int>> state(n_req);   // 0 pending, 1 submitted, -1 submit failed
    for (auto &x : state) x.store(0);
    std::atomic<int> submit_rc{PROSPER_OK};
    const int64_t t0 = now_ns() + 2000000;        // start 2 ms from now
    // open-loop submitter: request i is submitted at t0 + arrival_ns[i] whatever
    // the state of earlier requests (sleep until ~50 us before, then spin)
    std::thread submitter([&] {
        for (int i = 0; i < n_req; ++i) {
            const int64_t due = t0 + arrival_ns[i];
            for (;;) {
                const int64_t left = due - now_ns();
                if (left <= 0) break;
                if (left > 60000) std::this_thread::sleep_for(std::chrono::nanoseconds(left - 50000));
            }
            t_submit_ns[i] = now_ns();
            const int rc = prosper_serve_submit(c, Y_pool_host + offsets[i] * D, sizes[i], &tickets[i]);
            if (rc) { submit_rc.store(rc); state[i].store(-1); break; }
            state[i].store(1, std::memory_order_release);
        }
    });
    // observer: polls every outstanding ticket without blocking and copies each
    // finished request's results to host memory, as a client would
    std::vector<int16_t> o_sel((size_t)c->serve->slot_points * Hp), o_map((size_t)c->serve->slot_points * g);
    std::vector<float> o_sm((size_t)c->serve->slot_points * Hp), o_p(c->serve->slot_points), o_z(c->serve->slot_points);
    int rc = PROSPER_OK, next = 0, remaining = n_req;
    std::vector<int> open;
    while (remaining > 0 && !rc) {
        while (next < n_req && state[next].load(std::memory_order_acquire) != 0) {
            if (state[next].load() < 0) { rc = submit_rc.load(); break; }
            open.push_back(next++);
        }
        if (rc) break;
        bool any = false;
        for (size_t k = 0; k < open.size();) {
            const int i = open[k];
            int64_t td = 0;
            const int w = prosper_serve_wait(c, tickets[i], 0, o_sel.data(), o_sm.data(), o_map.data(),
                                             o_p.data(), o_z.data(), nullptr, &td);
            if (w == PROSPER_ETIMEOUT) { ++k; continue; }
            if (w) { rc = w; break; }
            t_observed_ns[i] = now_ns();
            if (t_done_ns) t_done_ns[i] = td;
            open[k] = open.back();
            open.pop_back();
            --remaining;
            any = true;
        }
        if (!any) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    submitter.join();
    if (rc) return rc;
    set_error("%s", "");
    return PROSPER_OK;
}

int prosper_serve_stop(prosper_ctx *c) {
    if (!c || !c->serve) return PROSPER_OK;
    ServeState *S = c->serve;
    S->stop.store(true);
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &s : S->slots) free_slot(s);
    delete S;
    c->serve = nullptr;
    return PROSPER_OK;
}

}  // extern "C"
