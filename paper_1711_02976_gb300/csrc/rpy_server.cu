// Serving loop for many resident bead systems (continuous batching).
//
// Every registered system owns, once admitted, a tree handle and device
// buffers for positions, forces and velocities, which stay on the device
// between requests.  A pool of worker threads, one CUDA stream each, takes
// requests from one queue: a request is started as soon as a worker is free,
// its system is not busy with an earlier request, and its system is resident
// or fits the memory budget (idle resident systems are evicted, least
// recently used first).  Requests of different systems therefore run at the
// same time on the device; requests of one system keep their order.
//
// Host data lives in page-locked (pinned) buffers from a pool owned by the
// server: a submit copies the caller's positions and forces into pinned
// buffers, so the worker's host-to-device copies run at full bus speed and the
// caller may reuse its arrays at once; a system's last good positions (needed
// to rebuild it after an eviction or a failed request) stay in a pinned buffer.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "rpy_internal.h"

namespace rpy {

using clk = std::chrono::steady_clock;

// Page-locked host buffers, reused by size.
struct PinnedPool {
    std::mutex mu;
    std::multimap<size_t, double *> free_;
    std::vector<double *> all;
    double *get(size_t count) {
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = free_.find(count);
            if (it != free_.end()) {
                double *p = it->second;
                free_.erase(it);
                return p;
            }
        }
        void *p = nullptr;
        if (cudaHostAlloc(&p, sizeof(double) * count, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        std::lock_guard<std::mutex> lk(mu);
        all.push_back(static_cast<double *>(p));
        return static_cast<double *>(p);
    }
    void put(double *p, size_t count) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        free_.emplace(count, p);
    }
    ~PinnedPool() {
        for (double *p : all) cudaFreeHost(p);
    }
};

struct SrvSystem {
    int64_t n = 0;
    double a = 0;
    rpy_build_params params{};
    double *pos = nullptr;             // last good positions (pinned host, 3 n)
    rpy_tree tree = nullptr;           // resident when non-null
    double *d_buf = nullptr;           // positions, forces, velocities: 9 n doubles
    int64_t bytes = 0;                 // device bytes held (estimate until built)
    bool busy = false;
    bool needs_build = true;           // device positions stale or tree absent
    uint64_t last_use = 0;
    int64_t est = 0;                   // admission estimate
};

struct SrvRequest {
    int64_t id = 0;
    int sys = 0;
    double *pos = nullptr;             // pinned copy of new positions, or null: keep the system's
    double *f = nullptr;               // pinned copy of the forces
    double s = 0;
    double *u_host = nullptr;
    clk::time_point t_submit, t_start, t_done;
    rpy_request_times times{};
    enum { QUEUED, RUNNING, DONE } state = QUEUED;
    int status = RPY_OK;
};

struct Server {
    rpy_server_params prm{};
    PinnedPool pinned;                 // destroyed last: requests and systems return into it
    int device = 0;
    int64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<SrvSystem> systems;
    std::deque<std::shared_ptr<SrvRequest>> queue;
    std::unordered_map<int64_t, std::shared_ptr<SrvRequest>> reqs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;   // one per worker, destroyed after the systems
    bool stop = false;
    int64_t next_id = 1;
    uint64_t tick = 0;
    int running = 0;
    int64_t resident = 0, peak = 0;
    rpy_server_stats st{};
    std::vector<double> lat;
    clk::time_point first_submit, last_done;
    bool any_submit = false;
};

// Return a finished request's pinned buffers (its positions only when not kept by the system).
static void release_buffers(Server &S, SrvRequest &r, int64_t n) {
    S.pinned.put(r.f, 3 * size_t(n));
    r.f = nullptr;
    S.pinned.put(r.pos, 3 * size_t(n));
    r.pos = nullptr;
}

// Free a resident system's device state (caller holds no lock; the system is not busy).
static void drop_device_state(SrvSystem &sy) {
    if (sy.tree) rpy_tree_free(sy.tree);
    if (sy.d_buf) cudaFree(sy.d_buf);
    sy.tree = nullptr;
    sy.d_buf = nullptr;
    sy.needs_build = true;
}

// Choose the next startable request (mu held).  Victims to evict are moved to `evict`.
static std::shared_ptr<SrvRequest> pick(Server &S, std::vector<SrvSystem *> &evict) {
    std::vector<char> blocked(S.systems.size(), 0);
    for (auto it = S.queue.begin(); it != S.queue.end(); ++it) {
        auto r = *it;
        SrvSystem &sy = S.systems[r->sys];
        if (blocked[r->sys] || sy.busy) {
            blocked[r->sys] = 1;   // keep per-system order
            continue;
        }
        if (!sy.tree && sy.bytes == 0) {
            int64_t need = sy.est;
            if (S.resident + need > S.budget) {
                // evict idle resident systems, least recently used first
                std::vector<int> cand;
                for (size_t k = 0; k < S.systems.size(); ++k)
                    if (int(k) != r->sys && S.systems[k].tree && !S.systems[k].busy) cand.push_back(int(k));
                std::sort(cand.begin(), cand.end(),
                          [&](int x, int y) { return S.systems[x].last_use < S.systems[y].last_use; });
                int64_t freed = 0;
                size_t take = 0;
                while (take < cand.size() && S.resident - freed + need > S.budget) freed += S.systems[cand[take++]].bytes;
                if (S.resident - freed + need > S.budget) {
                    blocked[r->sys] = 1;
                    continue;
                }
                for (size_t k = 0; k < take; ++k) {
                    SrvSystem &v = S.systems[cand[k]];
                    S.resident -= v.bytes;
                    v.bytes = 0;
                    v.busy = true;   // until its device state is freed by the picking worker
                    evict.push_back(&v);
                    S.st.evictions++;
                }
            }
            sy.bytes = need;          // reservation, replaced by the real size after the build
            S.resident += need;
            S.peak = std::max(S.peak, S.resident);
        }
        sy.busy = true;
        r->state = SrvRequest::RUNNING;
        r->t_start = clk::now();
        S.queue.erase(it);
        return r;
    }
    return nullptr;
}

// Events of one worker between the phases of a request (device time of each phase).
struct PhaseEvents {
    cudaEvent_t e[6] = {};
    bool ok = true;
    PhaseEvents() {
        for (auto &x : e) ok = ok && cudaEventCreate(&x) == cudaSuccess;
    }
    ~PhaseEvents() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
    double ms(int a, int b) const {
        float v = 0.f;
        return ok && cudaEventElapsedTime(&v, e[a], e[b]) == cudaSuccess ? double(v) : 0.0;
    }
};

static int run_request(Server &S, SrvSystem &sy, SrvRequest &r, cudaStream_t st, PhaseEvents &ev) {
    int64_t n = sy.n;
    bool fresh = false;
    if (!sy.d_buf) {
        RPY_CHECK(cudaMalloc(&sy.d_buf, sizeof(double) * 9 * size_t(n)));
        fresh = true;
    }
    double *dp = sy.d_buf, *df = sy.d_buf + 3 * n, *du = sy.d_buf + 6 * n;
    const double *pos = r.pos ? r.pos : sy.pos;
    const bool build = r.pos || fresh || sy.needs_build;
    if (ev.ok) RPY_CHECK(cudaEventRecord(ev.e[0], st));
    if (build) RPY_CHECK(cudaMemcpyAsync(dp, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    if (ev.ok) RPY_CHECK(cudaEventRecord(ev.e[1], st));
    if (build) {
        if (sy.tree) {
            RPY_TRY(rpy_tree_update_positions(sy.tree, dp, st));
            S.st.rebuilds++;
        } else {
            int64_t off[2] = {0, n};
            RPY_TRY(rpy_forest_build(dp, off, 1, &sy.a, &sy.params, st, &sy.tree));
        }
        sy.needs_build = false;
    }
    if (ev.ok) RPY_CHECK(cudaEventRecord(ev.e[2], st));
    RPY_CHECK(cudaMemcpyAsync(df, r.f, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    if (ev.ok) RPY_CHECK(cudaEventRecord(ev.e[3], st));
    RPY_TRY(rpy_matvec(sy.tree, df, r.s, du, st));
    if (ev.ok) RPY_CHECK(cudaEventRecord(ev.e[4], st));
    RPY_CHECK(cudaMemcpyAsync(r.u_host, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    if (ev.ok) RPY_CHECK(cudaEventRecord(ev.e[5], st));
    RPY_CHECK(cudaStreamSynchronize(st));
    if (ev.ok) {
        r.times.h2d_ms = ev.ms(0, 1) + ev.ms(2, 3);
        r.times.build_ms = build ? ev.ms(1, 2) : 0.0;
        r.times.matvec_ms = ev.ms(3, 4);
        r.times.d2h_ms = ev.ms(4, 5);
    }
    return RPY_OK;
}

static void worker(Server *S, cudaStream_t st) {
    cudaSetDevice(S->device);
    PhaseEvents ev;
    for (;;) {
        std::shared_ptr<SrvRequest> r;
        std::vector<SrvSystem *> evict;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop) break;
                r = pick(*S, evict);
                if (r) break;
                S->cv_work.wait(lk);
            }
            if (!r && S->stop) break;
            S->running++;
        }
        for (SrvSystem *v : evict) {
            drop_device_state(*v);
            std::lock_guard<std::mutex> lk(S->mu);
            v->busy = false;
        }
        SrvSystem &sy = S->systems[r->sys];
        int status = run_request(*S, sy, *r, st, ev);
        int64_t real = 0;
        if (sy.tree) {
            rpy_stats s{};
            if (rpy_tree_stats(sy.tree, &s) == RPY_OK) real = s.device_bytes + int64_t(sizeof(double)) * 9 * sy.n;
        }
        if (status != RPY_OK) {
            // a failed request leaves its system rebuildable from scratch
            drop_device_state(sy);
            real = 0;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->resident += real - sy.bytes;
            sy.bytes = real;
            S->peak = std::max(S->peak, S->resident);
            if (status == RPY_OK && r->pos) std::swap(sy.pos, r->pos);   // the new last good positions
            sy.busy = false;
            sy.last_use = ++S->tick;
            r->status = status;
            r->t_done = clk::now();
            r->times.queue_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
            r->times.run_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_start).count();
            r->state = SrvRequest::DONE;
            S->running--;
            if (status == RPY_OK) {
                S->st.completed++;
                S->st.beads_done += sy.n;
                S->lat.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
            } else {
                S->st.failed++;
            }
            S->last_done = r->t_done;
        }
        release_buffers(*S, *r, sy.n);
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace rpy

struct rpy_server_s {
    rpy::Server S;
};

using namespace rpy;

extern "C" {

int rpy_server_create(const rpy_server_params *params, rpy_server *out) {
    if (!out) return RPY_ERR_INVALID;
    *out = nullptr;
    rpy_server_params p{};
    if (params) p = *params;
    if (p.slots < 0 || p.slots > 64 || p.device_budget_bytes < 0) return RPY_ERR_INVALID;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return RPY_ERR_NODEVICE;
    }
    auto *h = new rpy_server_s();
    Server &S = h->S;
    S.prm = p;
    if (p.device >= 0) S.device = p.device;
    else cudaGetDevice(&S.device);
    if (S.device >= n) {
        delete h;
        return RPY_ERR_INVALID;
    }
    cudaSetDevice(S.device);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        delete h;
        return check_cuda("cudaMemGetInfo", cudaGetLastError());
    }
    S.budget = p.device_budget_bytes > 0 ? p.device_budget_bytes : int64_t(0.85 * double(fr));
    int slots = p.slots > 0 ? p.slots : 4;
    for (int k = 0; k < slots; ++k) {
        cudaStream_t st = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t q : S.streams) cudaStreamDestroy(q);
            delete h;
            return check_cuda("cudaStreamCreate", e);
        }
        S.streams.push_back(st);
    }
    for (int k = 0; k < slots; ++k) S.workers.emplace_back(worker, &S, S.streams[k]);
    *out = h;
    return RPY_OK;
}

int rpy_server_add_system(rpy_server h, const double *pos_host, int64_t n, double a, const rpy_build_params *params,
                          int *system_id) {
    if (!h || !pos_host || n < 1 || !(a > 0) || !params || !system_id) return RPY_ERR_INVALID;
    if (params->digits != 3 && params->digits != 6 && params->digits != 9) return RPY_ERR_DIGITS;
    Server &S = h->S;
    SrvSystem sy;
    sy.n = n;
    sy.a = a;
    sy.params = *params;
    int64_t fp = 0;
    RPY_TRY(rpy_tree_footprint(n, params->digits, params->precision, params->leaf_cap, &fp));
    sy.est = fp + int64_t(sizeof(double)) * 9 * n;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (sy.est > S.budget) return RPY_ERR_OOM;
    }
    cudaSetDevice(S.device);
    sy.pos = S.pinned.get(3 * size_t(n));
    if (!sy.pos) return RPY_ERR_OOM;
    std::memcpy(sy.pos, pos_host, sizeof(double) * 3 * size_t(n));
    std::lock_guard<std::mutex> lk(S.mu);
    S.systems.push_back(std::move(sy));
    *system_id = int(S.systems.size()) - 1;
    return RPY_OK;
}

int rpy_server_submit(rpy_server h, int system_id, const double *pos_host, const double *f_host, double kT_over_eta,
                      double *u_host, int64_t *request_id) {
    if (!h || !f_host || !u_host || !request_id || !std::isfinite(kT_over_eta)) return RPY_ERR_INVALID;
    Server &S = h->S;
    auto r = std::make_shared<SrvRequest>();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (S.stop) return RPY_ERR_STATE;
        if (system_id < 0 || system_id >= int(S.systems.size())) return RPY_ERR_INVALID;
    }
    int64_t n = S.systems[system_id].n;
    r->sys = system_id;
    cudaSetDevice(S.device);
    r->f = S.pinned.get(3 * size_t(n));
    if (pos_host) r->pos = S.pinned.get(3 * size_t(n));
    if (!r->f || (pos_host && !r->pos)) {
        release_buffers(S, *r, n);
        return RPY_ERR_OOM;
    }
    std::memcpy(r->f, f_host, sizeof(double) * 3 * size_t(n));
    if (pos_host) std::memcpy(r->pos, pos_host, sizeof(double) * 3 * size_t(n));
    r->s = kT_over_eta;
    r->u_host = u_host;
    r->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        r->id = S.next_id++;
        S.reqs[r->id] = r;
        S.queue.push_back(r);
        S.st.submitted++;
        if (!S.any_submit) {
            S.first_submit = r->t_submit;
            S.any_submit = true;
        }
        *request_id = r->id;
    }
    S.cv_work.notify_one();
    return RPY_OK;
}

int rpy_server_wait_times(rpy_server h, int64_t request_id, int timeout_ms, double *latency_ms,
                          rpy_request_times *times) {
    if (!h) return RPY_ERR_INVALID;
    Server &S = h->S;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.reqs.find(request_id);
    if (it == S.reqs.end()) return RPY_ERR_INVALID;
    auto r = it->second;
    auto done = [&] { return r->state == SrvRequest::DONE; };
    if (timeout_ms < 0) S.cv_done.wait(lk, done);
    else if (!S.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return RPY_ERR_TIMEOUT;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (times) *times = r->times;
    int status = r->status;
    S.reqs.erase(request_id);
    return status;
}

int rpy_server_wait(rpy_server h, int64_t request_id, int timeout_ms, double *latency_ms) {
    return rpy_server_wait_times(h, request_id, timeout_ms, latency_ms, nullptr);
}

int rpy_server_cancel(rpy_server h, int64_t request_id) {
    if (!h) return RPY_ERR_INVALID;
    Server &S = h->S;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        auto it = S.reqs.find(request_id);
        if (it == S.reqs.end()) return RPY_ERR_INVALID;
        auto r = it->second;
        if (r->state != SrvRequest::QUEUED) return RPY_ERR_STATE;
        S.queue.erase(std::remove(S.queue.begin(), S.queue.end(), r), S.queue.end());
        r->state = SrvRequest::DONE;
        r->status = RPY_ERR_STATE;
        r->t_done = clk::now();
        S.st.cancelled++;
        release_buffers(S, *r, S.systems[r->sys].n);
    }
    S.cv_done.notify_all();
    S.cv_work.notify_all();
    return RPY_OK;
}

int rpy_server_drain(rpy_server h) {
    if (!h) return RPY_ERR_INVALID;
    Server &S = h->S;
    std::unique_lock<std::mutex> lk(S.mu);
    S.cv_done.wait(lk, [&] { return S.queue.empty() && S.running == 0; });
    return RPY_OK;
}

int rpy_server_stats_get(rpy_server h, rpy_server_stats *out) {
    if (!h || !out) return RPY_ERR_INVALID;
    Server &S = h->S;
    std::lock_guard<std::mutex> lk(S.mu);
    *out = S.st;
    out->resident_bytes = S.resident;
    out->peak_resident_bytes = S.peak;
    int rs = 0;
    for (auto &sy : S.systems) rs += sy.tree ? 1 : 0;
    out->resident_systems = rs;
    out->queued = int(S.queue.size());
    out->running = S.running;
    if (!S.lat.empty()) {
        std::vector<double> v = S.lat;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, size_t(f * double(v.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / double(v.size());
    }
    if (S.any_submit) out->busy_s = std::chrono::duration<double>(S.last_done - S.first_submit).count();
    return RPY_OK;
}

void rpy_server_destroy(rpy_server h) {
    if (!h) return;
    Server &S = h->S;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        for (auto &r : S.queue) {
            r->state = SrvRequest::DONE;
            r->status = RPY_ERR_STATE;
            S.st.cancelled++;
            release_buffers(S, *r, S.systems[r->sys].n);
        }
        S.queue.clear();
        S.stop = true;
    }
    S.cv_work.notify_all();
    S.cv_done.notify_all();
    for (auto &w : S.workers) w.join();
    cudaSetDevice(S.device);
    for (auto &sy : S.systems) drop_device_state(sy);
    for (cudaStream_t q : S.streams) cudaStreamDestroy(q);
    delete h;   // the pinned pool (every system's positions and the requests' buffers) goes last
}

}  // extern "C"
