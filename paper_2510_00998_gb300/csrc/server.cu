// Solve server: continuous batching of independent solves on one GPU (each
// solved as dgmg_solve; serving has no counterpart in the paper).
//
// Requests (mesh, degree, kappa, device b and x) are queued by dgmg_submit and
// admitted by a scheduler thread as soon as an execution slot is free and the
// request's hierarchy fits the HBM budget. Hierarchies stay resident after a
// solve (a cache keyed by mesh, degree and kappa; least recently used idle
// entries are evicted when an admission needs room), so a repeated problem
// skips set-up. Every admitted request runs on its own CUDA stream as a
// non-blocking solve state machine (solver.cu); the scheduler advances all of
// them in turn, so requests that arrive while others are on the GPU join at
// the next CG iteration and their kernels overlap on the device.
#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "ctx.h"

namespace {

using Clock = std::chrono::steady_clock;

uint64_t hash_kappa(const std::vector<double> &k) {
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the bytes
    const unsigned char *p = reinterpret_cast<const unsigned char *>(k.data());
    for (size_t i = 0; i < k.size() * sizeof(double); ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct CacheEntry {
    dgmg_mesh mesh{};
    int p = 0;
    bool has_kappa = false;
    uint64_t khash = 0;
    std::vector<double> kappa;
    dgmg_ctx *ctx = nullptr;
    size_t bytes = 0;
    bool busy = false;
    uint64_t last_use = 0;
};

struct Request {
    uint64_t id = 0;
    dgmg_mesh mesh{};
    int p = 0;
    bool has_kappa = false;
    uint64_t khash = 0;
    std::vector<double> kappa;
    const double *b = nullptr;
    double *x = nullptr;
    int status = DGMG_PENDING;
    int rc = DGMG_OK;
    std::string error;
    dgmg_stats stats{};
    Clock::time_point t_submit, t_admit;
    CacheEntry *entry = nullptr;
    int slot = -1;
    SolveRun run;
};

bool same_problem(const CacheEntry &e, const Request &r) {
    if (e.p != r.p || e.mesh.dim != r.mesh.dim || e.has_kappa != r.has_kappa || e.khash != r.khash) return false;
    for (int a = 0; a < r.mesh.dim; ++a)
        if (e.mesh.n[a] != r.mesh.n[a]) return false;
    return !r.has_kappa || e.kappa == r.kappa;
}

}  // namespace

struct dgmg_server {
    size_t budget = 0;
    int max_active = 1;
    dgmg_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> pending;
    std::vector<Request *> active;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> requests;
    std::list<CacheEntry> cache;
    size_t bytes = 0;
    uint64_t next_id = 1, tick = 0;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    std::deque<std::pair<Request *, size_t>> to_setup;   // admitted, hierarchy not built yet (bytes reserved)
    int setting_up = 0;
    bool stop = false;
    long long n_done = 0, n_failed = 0, hits = 0, misses = 0, admitted = 0, evictions = 0;
    std::thread worker;
    std::vector<std::thread> setup_workers;

    int take_slot() {
        int slot = 0;
        while (slot_busy[slot]) ++slot;
        slot_busy[slot] = true;
        return slot;
    }

    void activate(Request *r, CacheEntry *e) {
        e->busy = true;
        r->entry = e;
        r->t_admit = Clock::now();
        r->status = DGMG_RUNNING;
        r->run.start(e->ctx, r->b, r->x, streams[r->slot]);
        active.push_back(r);
        ++admitted;
    }

    // Builds hierarchies for admitted requests off the scheduler thread, so
    // running solves keep being advanced meanwhile.
    void setup_loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv.wait(lk, [&] { return stop_setup || !to_setup.empty(); });
            if (to_setup.empty()) {
                if (stop_setup) return;
                continue;
            }
            Request *r = to_setup.front().first;
            const size_t reserved = to_setup.front().second;
            to_setup.pop_front();
            const double *kp = r->has_kappa ? r->kappa.data() : nullptr;
            lk.unlock();
            dgmg_ctx *ctx = nullptr;
            const int rc = create_ctx(&r->mesh, r->p, kp, &opts, CREATE_SHARED_GPU, &ctx);
            const std::string err = rc == DGMG_OK ? "" : dgmg_last_error();
            size_t actual = 0;
            if (rc == DGMG_OK) {
                dgmg_info_t inf;
                dgmg_info(ctx, &inf);
                actual = inf.device_bytes;
            }
            lk.lock();
            --setting_up;
            bytes -= reserved;
            if (rc != DGMG_OK) {
                slot_busy[r->slot] = false;
                finish(r, DGMG_FAILED, rc, err);
            } else {
                cache.emplace_back();
                CacheEntry *e = &cache.back();
                e->mesh = r->mesh;
                e->p = r->p;
                e->has_kappa = r->has_kappa;
                e->khash = r->khash;
                e->kappa = r->kappa;
                e->ctx = ctx;
                e->bytes = actual;
                bytes += actual;
                r->kappa.clear();
                r->kappa.shrink_to_fit();
                activate(r, e);
            }
            cv.notify_all();
        }
    }
    bool stop_setup = false;

    void finish(Request *r, int status, int rc, const std::string &err) {
        r->status = status;
        r->rc = rc;
        r->error = err;
        r->kappa.clear();
        r->kappa.shrink_to_fit();
        if (status == DGMG_DONE)
            ++n_done;
        else
            ++n_failed;
    }

    // Admit queued requests while slots and memory allow (scheduler thread only).
    // A resident hierarchy of the same problem is reused at once; otherwise the
    // bytes are reserved (evicting least recently used idle hierarchies as
    // needed) and the build is handed to the set-up workers.
    void admit() {
        while (!pending.empty() && (int)active.size() + setting_up < max_active) {
            Request *r = pending.front();
            CacheEntry *e = nullptr;
            for (auto &c : cache)
                if (!c.busy && same_problem(c, *r)) {
                    e = &c;
                    break;
                }
            if (e) {
                ++hits;
                pending.pop_front();
                r->slot = take_slot();
                r->kappa.clear();
                r->kappa.shrink_to_fit();
                activate(r, e);
                continue;
            }
            size_t est = 0;
            if (dgmg_estimate_bytes(&r->mesh, r->p, &opts, &est) != DGMG_OK) {
                pending.pop_front();
                finish(r, DGMG_FAILED, DGMG_EINVAL, dgmg_last_error());
                continue;
            }
            if (est > budget) {
                pending.pop_front();
                finish(r, DGMG_FAILED, DGMG_EBUDGET,
                       "request needs " + std::to_string(est) + " bytes, budget " + std::to_string(budget));
                continue;
            }
            while (bytes + est > budget) {   // evict least recently used idle hierarchies
                auto victim = cache.end();
                for (auto it = cache.begin(); it != cache.end(); ++it)
                    if (!it->busy && (victim == cache.end() || it->last_use < victim->last_use)) victim = it;
                if (victim == cache.end()) break;
                bytes -= victim->bytes;
                destroy_idle(victim->ctx);
                cache.erase(victim);
                ++evictions;
            }
            if (bytes + est > budget) return;   // wait for running solves to release memory
            ++misses;
            pending.pop_front();
            bytes += est;
            r->slot = take_slot();
            ++setting_up;
            to_setup.emplace_back(r, est);
            cv.notify_all();
        }
    }

    // An idle hierarchy: its last solve has completed (the run's final event),
    // so it is freed without a device-wide synchronisation.
    static void destroy_idle(dgmg_ctx *ctx) { delete ctx; }

    void loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            if (stop && active.empty() && pending.empty() && setting_up == 0) break;
            admit();
            std::vector<Request *> work = active;
            lk.unlock();
            std::vector<Request *> finished;
            for (Request *r : work)
                if (r->run.advance(false)) finished.push_back(r);
            lk.lock();
            for (Request *r : finished) {
                r->stats = r->run.stats;
                r->stats.seconds = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
                r->stats.queue_seconds = std::chrono::duration<double>(r->t_admit - r->t_submit).count();
                r->entry->busy = false;
                r->entry->last_use = ++tick;
                slot_busy[r->slot] = false;
                active.erase(std::find(active.begin(), active.end(), r));
                const int st = r->run.status == DGMG_OK ? DGMG_DONE : DGMG_FAILED;
                finish(r, st, r->run.status, r->run.status == DGMG_OK ? "" : dgmg_last_error());
            }
            if (!finished.empty()) cv.notify_all();
            if (finished.empty())   // nothing completed: let the GPU work, wake on new requests
                cv.wait_for(lk, std::chrono::microseconds(active.empty() ? 2000 : 20));
        }
    }
};

extern "C" {

int dgmg_server_create(size_t hbm_budget_bytes, int max_active, const dgmg_opts *opts, dgmg_server **out) {
    if (!out) return fail(DGMG_EINVAL, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes == 0) return fail(DGMG_EINVAL, "hbm_budget_bytes must be > 0");
    if (max_active < 1 || max_active > 1024) return fail(DGMG_EINVAL, "max_active must be in 1..1024");
    std::unique_ptr<dgmg_server> S(new dgmg_server());
    S->budget = hbm_budget_bytes;
    S->max_active = max_active;
    dgmg_default_opts(&S->opts);
    if (opts) S->opts = *opts;
    if (S->opts.outer == DGMG_OUTER_RELIABLE && S->opts.precision != DGMG_MIXED_FP32)
        return fail(DGMG_EINVAL, "DGMG_OUTER_RELIABLE needs DGMG_MIXED_FP32");
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    S->streams.resize(max_active);
    S->slot_busy.assign(max_active, false);
    for (int i = 0; i < max_active; ++i) {
        e = cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaStreamDestroy(S->streams[k]);
            return cuda_fail(e, "cudaStreamCreate");
        }
    }
    dgmg_server *raw = S.get();
    S->worker = std::thread([raw]() { raw->loop(); });
    for (int i = 0; i < 6; ++i) S->setup_workers.emplace_back([raw]() { raw->setup_loop(); });
    *out = S.release();
    return DGMG_OK;
}

int dgmg_submit(dgmg_server *S, const dgmg_mesh *mesh, int p, const double *kappa_host, const double *b_dev,
                double *x_dev, uint64_t *ticket) {
    if (!S || !mesh || !b_dev || !x_dev || !ticket) return fail(DGMG_EINVAL, "NULL argument");
    if (b_dev == x_dev) return fail(DGMG_EINVAL, "b and x must not overlap");
    size_t est = 0;
    RC(dgmg_estimate_bytes(mesh, p, &S->opts, &est));   // validates mesh and p
    std::unique_ptr<Request> r(new Request());
    r->mesh = *mesh;
    r->p = p;
    const int64_t ncell = (int64_t)mesh->n[0] * mesh->n[1] * (mesh->dim == 3 ? mesh->n[2] : 1);
    if (kappa_host) {
        r->has_kappa = true;
        r->kappa.assign(kappa_host, kappa_host + ncell);
        for (int64_t i = 0; i < ncell; ++i)
            if (!(r->kappa[i] > 0.0) || !std::isfinite(r->kappa[i]))
                return fail(DGMG_EINVAL, "kappa must be positive and finite");
        r->khash = hash_kappa(r->kappa);
    }
    r->b = b_dev;
    r->x = x_dev;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(DGMG_EINVAL, "server is shutting down");
    r->id = S->next_id++;
    *ticket = r->id;
    S->pending.push_back(r.get());
    S->requests[r->id] = std::move(r);
    S->cv.notify_all();
    return DGMG_OK;
}

int dgmg_poll(dgmg_server *S, uint64_t ticket, int *status, dgmg_stats *stats) {
    if (!S || !status) return fail(DGMG_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->requests.find(ticket);
    if (it == S->requests.end()) return fail(DGMG_EINVAL, "unknown ticket");
    Request *r = it->second.get();
    *status = r->status;
    if (r->status != DGMG_DONE && r->status != DGMG_FAILED) return DGMG_OK;
    // the result is handed over once: the scheduler no longer touches a finished
    // request, so its record is released here and the table stays bounded
    if (stats) *stats = r->stats;
    const int rc = r->rc;
    const bool failed = r->status == DGMG_FAILED;
    const std::string err = r->error;
    S->requests.erase(it);
    return failed ? fail(rc, err) : DGMG_OK;
}

int dgmg_server_info(dgmg_server *S, dgmg_server_info_t *info) {
    if (!S || !info) return fail(DGMG_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(info, 0, sizeof(*info));
    info->pending = (int)S->pending.size();
    info->active = (int)S->active.size();
    info->done = S->n_done;
    info->failed = S->n_failed;
    info->admitted = S->admitted;
    info->cache_entries = (int)S->cache.size();
    info->cache_hits = S->hits;
    info->cache_misses = S->misses;
    info->evictions = S->evictions;
    info->bytes_in_use = S->bytes;
    info->budget = S->budget;
    return DGMG_OK;
}

int dgmg_server_destroy(dgmg_server *S) {
    if (!S) return DGMG_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (Request *r : S->pending) S->finish(r, DGMG_FAILED, DGMG_EINVAL, "server destroyed before admission");
        S->pending.clear();
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop_setup = true;
        S->cv.notify_all();
    }
    for (auto &w : S->setup_workers) w.join();
    for (auto &c : S->cache) dgmg_server::destroy_idle(c.ctx);
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    delete S;
    return DGMG_OK;
}

}  // extern "C"
