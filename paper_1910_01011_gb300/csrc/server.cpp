// server.cpp -- request loop for planning solves (the serving layer above
// the solver): scenes (mesh, materials, transducer) are registered once and
// their device state -- geometry, near-field corrections, preconditioner,
// assembled operators -- stays resident between requests; requests (a set of
// piston excitations for one scene) arrive at any time, wait in a FIFO queue
// and are admitted to one of `slots` worker threads as soon as a worker and
// enough of the device-memory budget are free.  Requests for the same scene
// that are queued when a worker picks that scene are merged into one solve
// of up to max_batch_rhs excitations (by default block GMRES over blocks of
// at most 16 excitations, one GEMM per operator application); requests for different scenes run on different
// workers, each scene on its own CUDA stream, so their kernels overlap on the
// GPU.  The budget is a hard limit: every device allocation of every scene
// draws on one shared counter and fails (BEM_ERR_OUT_OF_BUDGET) past it;
// admission reserves each solve's estimated growth first and evicts idle
// scenes (least recently used first) to make room.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bem.h"
#include "ctx.h"

namespace gbem {
void release_device_memory(bem_ctx* ctx);
int64_t estimate_solve_bytes(const bem_ctx* ctx, int64_t n_exc, const bem_solve_opts& o);
int64_t solve_batch_width(const bem_solve_opts& o, int64_t n_exc);
int copy_solution(bem_ctx* ctx, int64_t rhs0, int64_t n, double2* host);
}  // namespace gbem

using namespace gbem;
using Clock = std::chrono::steady_clock;

namespace {

struct Scene {
    bem_ctx* ctx = nullptr;
    int64_t n_elem = 0;
    int64_t n_dofs = 0;
    bool busy = false;
    int64_t peak = 0;        // largest device footprint seen (bytes)
    Clock::time_point last;  // last use, for eviction
};

struct Request {
    int64_t handle = 0;
    int32_t scene = 0;
    int64_t n_exc = 0;
    std::vector<double> w;   // [n_exc][n_elem] complex
    int state = BEM_REQ_QUEUED;
    int rc = BEM_OK;
    std::string err;
    std::vector<double2> u;  // [n_exc][n_dofs]
    bem_solve_report rep{};
    int64_t batch_exc = 0;   // excitations solved together with this request
    bool retried = false;
    Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct bem_server {
    int device = 0;
    bem_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::unique_ptr<Scene>> scenes;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::deque<int64_t> queue;
    std::atomic<int64_t> pool{0};  // device bytes held by all scenes
    int64_t reserved = 0;          // admitted growth not yet allocated
    int64_t next_handle = 1;
    int running = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    // statistics
    std::vector<double> lat_ms, wait_ms;
    int64_t done_req = 0, done_exc = 0, failed = 0, batches = 0, batch_exc_sum = 0, evictions = 0, joined = 0;
    int64_t peak_pool = 0;
    Clock::time_point t_first, t_last;
    bool any = false;

    void worker();
    bool pick(std::vector<Request*>& group, Scene*& sc, int64_t& extra);
    // joining running solves: mixed precision only (its refinement boundaries)
    bool joins() const { return opts.join && opts.solve.precision == BEM_PREC_FP32 && opts.solve.batch_rhs > 1; }
    int64_t join_cap() const { return solve_batch_width(opts.solve, opts.solve.batch_rhs); }
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

// Under the lock: choose the next group to run (oldest admissible request,
// plus later queued requests of the same scene up to max_batch_rhs
// excitations) and reserve its memory.  Returns false if nothing can start.
bool bem_server::pick(std::vector<Request*>& group, Scene*& sc, int64_t& extra) {
    for (size_t qi = 0; qi < queue.size(); qi++) {
        Request* r0 = reqs[queue[qi]].get();
        Scene* s = scenes[r0->scene].get();
        if (s->busy) continue;
        const int64_t budget = opts.hbm_budget_bytes;
        // the group: r0, then later requests of the same scene while the
        // merged solve stays within max_batch_rhs and its estimate within the budget
        std::vector<size_t> idx{qi};
        int64_t n = r0->n_exc;
        for (size_t qj = qi + 1; qj < queue.size(); qj++) {
            Request* r = reqs[queue[qj]].get();
            if (r->scene != r0->scene || r->retried) continue;
            if (n + r->n_exc > std::max<int64_t>(opts.max_batch_rhs, r0->n_exc)) continue;
            if (budget > 0 && estimate_solve_bytes(s->ctx, n + r->n_exc, opts.solve) > budget) continue;
            idx.push_back(qj);
            n += r->n_exc;
        }
        // memory: estimated footprint of this solve minus what the scene holds
        int64_t need = std::max(s->peak, estimate_solve_bytes(s->ctx, n, opts.solve));
        // a retry (the estimate fell short) asks for more, at most the whole budget
        if (r0->retried) {
            need = std::max(need, s->peak + s->peak / 4);
            if (opts.hbm_budget_bytes > 0) need = std::min<int64_t>(need, opts.hbm_budget_bytes);
        }
        int64_t grow = std::max<int64_t>(0, need - (int64_t)s->ctx->used_bytes);
        if (budget > 0 && need > budget) {
            // r0 alone can never fit (the group holds only r0 then)
            r0->state = BEM_REQ_FAILED;
            r0->rc = BEM_ERR_OUT_OF_BUDGET;
            r0->err = "solve needs more device memory than the whole budget";
            r0->t_done = Clock::now();
            failed++;
            queue.erase(queue.begin() + qi);
            cv_done.notify_all();
            return pick(group, sc, extra);
        }
        while (budget > 0 && pool.load() + reserved + grow > budget) {
            // evict the least recently used idle scene that holds memory
            Scene* victim = nullptr;
            for (auto& o : scenes)
                if (o.get() != s && !o->busy && o->ctx->used_bytes > 0 && (!victim || o->last < victim->last))
                    victim = o.get();
            if (!victim) break;
            release_device_memory(victim->ctx);
            evictions++;
        }
        if (budget > 0 && pool.load() + reserved + grow > budget) {
            if (running == 0 && s->ctx->used_bytes > 0) {
                // nothing else holds memory: start over from an empty scene
                release_device_memory(s->ctx);
                grow = need;
                if (pool.load() + reserved + grow > budget) return false;
            } else {
                return false;  // wait for a running solve to finish (keeps FIFO order)
            }
        }
        // admit
        group.clear();
        for (size_t k : idx) group.push_back(reqs[queue[k]].get());
        for (size_t k = idx.size(); k-- > 0;) queue.erase(queue.begin() + idx[k]);
        s->busy = true;
        sc = s;
        extra = grow;
        reserved += grow;
        return true;
    }
    return false;
}

void bem_server::worker() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        std::vector<Request*> group;
        Scene* s = nullptr;
        int64_t extra = 0;
        while (!stop && !pick(group, s, extra)) cv_work.wait(lk);
        if (stop) return;
        running++;
        const auto t0 = Clock::now();
        int64_t n = 0;
        for (Request* r : group) {
            r->state = BEM_REQ_RUNNING;
            r->t_start = t0;
            n += r->n_exc;
        }
        // the batch's excitation matrix
        std::vector<double> W;
        W.reserve(2 * n * s->n_elem);
        for (Request* r : group) W.insert(W.end(), r->w.begin(), r->w.end());
        lk.unlock();

        bem_ctx* ctx = s->ctx;
        bem_solve_report rep{};
        if (joins()) {
            // later requests for this scene join at a refinement boundary (FIFO order, while they fit)
            const int32_t scene_id = group.front()->scene;
            ctx->join_hook = [this, scene_id, ctx, &group, &extra, n_cur = n](int64_t room,
                                                                              std::vector<double>& w) mutable -> int64_t {
                std::lock_guard<std::mutex> g(mu);
                int64_t k = 0;
                for (size_t qi = 0; qi < queue.size();) {
                    Request* r = reqs[queue[qi]].get();
                    if (r->scene != scene_id || r->retried || r->n_exc > room - k) {
                        qi++;
                        continue;
                    }
                    // the solve's estimate grows with the joined excitations: reserve the growth
                    const int64_t add = std::max<int64_t>(
                        0, estimate_solve_bytes(ctx, n_cur + k + r->n_exc, opts.solve) -
                               estimate_solve_bytes(ctx, n_cur + k, opts.solve));
                    if (opts.hbm_budget_bytes > 0 && pool.load() + reserved + add > opts.hbm_budget_bytes) {
                        qi++;
                        continue;
                    }
                    reserved += add;
                    extra += add;
                    r->state = BEM_REQ_RUNNING;
                    r->t_start = Clock::now();
                    w.insert(w.end(), r->w.begin(), r->w.end());
                    k += r->n_exc;
                    group.push_back(r);
                    queue.erase(queue.begin() + qi);
                    joined++;
                }
                n_cur += k;
                return k;
            };
        }
        int rc = bem_set_excitations(ctx, (const bem_z*)W.data(), n);
        if (!rc) rc = bem_solve(ctx, &opts.solve, &rep);
        ctx->join_hook = nullptr;
        n = 0;
        for (Request* r : group) n += r->n_exc;  // joined requests included
        const bool converged_fail = rc == BEM_ERR_NOT_CONVERGED;
        std::string err = rc ? bem_last_error(ctx) : std::string();
        std::vector<double2> U;
        if (!rc || converged_fail) {
            // the solutions (kept also when the tolerance was not met, if the solve finished)
            U.resize((size_t)n * s->n_dofs);
            if (copy_solution(ctx, 0, n, U.data())) U.clear();
        }
        const auto t1 = Clock::now();

        lk.lock();
        running--;
        reserved -= extra;
        s->busy = false;
        s->last = t1;
        s->peak = std::max<int64_t>(s->peak, (int64_t)ctx->peak_bytes);
        peak_pool = std::max(peak_pool, pool.load());
        batches++;
        batch_exc_sum += n;
        int64_t off = 0;
        for (Request* r : group) {
            r->batch_exc = n;
            if (rc == BEM_ERR_OUT_OF_BUDGET && !r->retried) {
                // the estimate was short: queue again at the front, once
                r->retried = true;
                r->state = BEM_REQ_QUEUED;
                queue.push_front(r->handle);
                continue;
            }
            r->rc = rc;
            r->err = err;
            r->rep = rep;
            if (!U.empty())
                r->u.assign(U.begin() + off * s->n_dofs, U.begin() + (off + r->n_exc) * s->n_dofs);
            off += r->n_exc;
            r->t_done = t1;
            r->state = (rc == BEM_OK) ? BEM_REQ_DONE : BEM_REQ_FAILED;
            if (rc == BEM_OK) {
                done_req++;
                done_exc += r->n_exc;
                lat_ms.push_back(ms_between(r->t_submit, t1));
                wait_ms.push_back(ms_between(r->t_submit, r->t_start));
                if (!any || t1 > t_last) t_last = t1;
            } else {
                failed++;
            }
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

extern "C" {

int bem_server_default_opts(bem_server_opts* o) {
    if (!o) return BEM_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof *o);
    o->slots = 2;
    o->max_batch_rhs = 64;
    o->hbm_budget_bytes = (int64_t)150 << 30;
    bem_default_solve_opts(&o->solve);
    o->solve.precision = BEM_PREC_FP32;
    o->solve.batch_rhs = 64;
    o->solve.block_gmres = 1;
    o->solve.operator_mode = 2;
    o->solve.recycle = 256;
    o->join = 1;
    return BEM_OK;
}

int bem_server_create(bem_server** out, int device, const bem_server_opts* opts) {
    if (!out) return BEM_ERR_INVALID_ARG;
    *out = nullptr;
    bem_server_opts o;
    bem_server_default_opts(&o);
    if (opts) o = *opts;
    if (o.slots < 1 || o.slots > 64 || o.max_batch_rhs < 1 || o.hbm_budget_bytes < 0 || o.join < 0 || o.join > 1)
        return BEM_ERR_INVALID_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return BEM_ERR_CUDA;
    bem_server* s = new (std::nothrow) bem_server();
    if (!s) return BEM_ERR_OUT_OF_BUDGET;
    s->device = device;
    s->opts = o;
    s->opts.solve.batch_rhs = std::max(s->opts.solve.batch_rhs, o.max_batch_rhs);
    for (int i = 0; i < o.slots; i++) s->workers.emplace_back(&bem_server::worker, s);
    *out = s;
    return BEM_OK;
}

int bem_server_destroy(bem_server* s) {
    if (!s) return BEM_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& sc : s->scenes) {
        sc->ctx->pool = nullptr;
        bem_destroy(sc->ctx);
    }
    delete s;
    return BEM_OK;
}

int bem_server_add_scene(bem_server* s, bem_ctx* ctx, int32_t* scene_id) {
    if (!s || !ctx || !scene_id) return BEM_ERR_INVALID_ARG;
    if (ctx->field_kind != 2) return ctx->fail(BEM_ERR_STATE, "a served scene needs a transducer (bem_set_transducer)");
    if (ctx->doms.empty()) return ctx->fail(BEM_ERR_STATE, "a served scene needs at least one domain");
    if (ctx->device != s->device) return ctx->fail(BEM_ERR_INVALID_ARG, "scene context is on another device");
    std::lock_guard<std::mutex> g(s->mu);
    // the scene's memory counts against the server budget from now on
    if (ctx->pool) return ctx->fail(BEM_ERR_STATE, "context already belongs to a server");
    s->pool += (int64_t)ctx->used_bytes;
    ctx->pool = &s->pool;
    ctx->pool_limit = s->opts.hbm_budget_bytes;
    if (!ctx->stream) {
        // a stream of its own, so that this scene's kernels overlap with the
        // other scenes' (the legacy default stream would serialise them)
        cudaSetDevice(s->device);
        cudaDeviceSynchronize();
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
            ctx->stream = st;
            ctx->own_stream = true;
        }
    }
    auto sc = std::make_unique<Scene>();
    sc->ctx = ctx;
    sc->n_elem = (int64_t)ctx->tr_r.size();
    int64_t nd = 0;
    bem_num_dofs(ctx, &nd);
    sc->n_dofs = nd;
    sc->last = Clock::now();
    s->scenes.push_back(std::move(sc));
    *scene_id = (int32_t)s->scenes.size() - 1;
    return BEM_OK;
}

int bem_server_scene_info(bem_server* s, int32_t scene_id, int64_t* n_dofs, int64_t* n_elem, int64_t* device_bytes) {
    if (!s) return BEM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (scene_id < 0 || scene_id >= (int32_t)s->scenes.size()) return BEM_ERR_INVALID_ARG;
    const Scene& sc = *s->scenes[scene_id];
    if (n_dofs) *n_dofs = sc.n_dofs;
    if (n_elem) *n_elem = sc.n_elem;
    if (device_bytes) *device_bytes = (int64_t)sc.ctx->used_bytes;
    return BEM_OK;
}

int bem_server_estimate(bem_server* s, int32_t scene_id, int64_t n_exc, int64_t* bytes) {
    if (!s || !bytes || n_exc < 1) return BEM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (scene_id < 0 || scene_id >= (int32_t)s->scenes.size()) return BEM_ERR_INVALID_ARG;
    const Scene& sc = *s->scenes[scene_id];
    *bytes = std::max(sc.peak, estimate_solve_bytes(sc.ctx, n_exc, s->opts.solve));
    return BEM_OK;
}

int bem_server_submit(bem_server* s, int32_t scene_id, const bem_z* weights, int64_t n_exc, int64_t* handle) {
    if (!s || !weights || n_exc < 1 || !handle) return BEM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (scene_id < 0 || scene_id >= (int32_t)s->scenes.size()) return BEM_ERR_INVALID_ARG;
    const Scene& sc = *s->scenes[scene_id];
    auto r = std::make_unique<Request>();
    r->handle = s->next_handle++;
    r->scene = scene_id;
    r->n_exc = n_exc;
    r->w.assign((const double*)weights, (const double*)weights + 2 * n_exc * sc.n_elem);
    r->t_submit = Clock::now();
    if (!s->any) {
        s->t_first = r->t_submit;
        s->any = true;
    }
    *handle = r->handle;
    s->queue.push_back(r->handle);
    s->reqs[r->handle] = std::move(r);
    s->cv_work.notify_all();
    return BEM_OK;
}

int bem_server_poll(bem_server* s, int64_t handle, int32_t* state) {
    if (!s || !state) return BEM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(handle);
    if (it == s->reqs.end()) return BEM_ERR_INVALID_ARG;
    *state = it->second->state;
    return BEM_OK;
}

int bem_server_wait(bem_server* s, int64_t handle, double timeout_s, int32_t* state) {
    if (!s) return BEM_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(handle);
    if (it == s->reqs.end()) return BEM_ERR_INVALID_ARG;
    Request* r = it->second.get();
    auto done = [r] { return r->state == BEM_REQ_DONE || r->state == BEM_REQ_FAILED; };
    if (timeout_s < 0) s->cv_done.wait(lk, done);
    else s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
    if (state) *state = r->state;
    return done() ? BEM_OK : BEM_ERR_TIMEOUT;
}

int bem_server_result(bem_server* s, int64_t handle, bem_z* u, bem_solve_report* report, double* latency_ms,
                      int64_t* batch_exc, int release) {
    if (!s) return BEM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(handle);
    if (it == s->reqs.end()) return BEM_ERR_INVALID_ARG;
    Request* r = it->second.get();
    if (r->state != BEM_REQ_DONE && r->state != BEM_REQ_FAILED) return BEM_ERR_STATE;
    if (u && !r->u.empty()) std::memcpy(u, r->u.data(), r->u.size() * sizeof(double2));
    if (report) *report = r->rep;
    if (latency_ms) *latency_ms = ms_between(r->t_submit, r->t_done);
    if (batch_exc) *batch_exc = r->batch_exc;
    const int rc = r->rc;
    if (release) s->reqs.erase(it);
    return rc;
}

const char* bem_server_error(bem_server* s, int64_t handle) {
    if (!s) return "null server";
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(handle);
    if (it == s->reqs.end()) return "unknown request";
    return it->second->err.c_str();
}

int bem_server_get_stats(bem_server* s, bem_server_stats* st) {
    if (!s || !st) return BEM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    std::memset(st, 0, sizeof *st);
    st->completed = s->done_req;
    st->excitations = s->done_exc;
    st->failed = s->failed;
    st->queued = (int64_t)s->queue.size();
    st->running = s->running;
    st->batches = s->batches;
    st->mean_batch_exc = s->batches ? (double)s->batch_exc_sum / s->batches : 0.0;
    st->p50_ms = percentile(s->lat_ms, 0.50);
    st->p99_ms = percentile(s->lat_ms, 0.99);
    st->max_ms = s->lat_ms.empty() ? 0.0 : *std::max_element(s->lat_ms.begin(), s->lat_ms.end());
    st->p50_wait_ms = percentile(s->wait_ms, 0.50);
    const double span = s->any && s->done_req ? ms_between(s->t_first, s->t_last) / 1e3 : 0.0;
    st->requests_per_s = span > 0 ? s->done_req / span : 0.0;
    st->excitations_per_s = span > 0 ? s->done_exc / span : 0.0;
    st->device_bytes = s->pool.load();
    st->peak_device_bytes = std::max(s->peak_pool, s->pool.load());
    st->evictions = s->evictions;
    st->joined = s->joined;
    return BEM_OK;
}

}  // extern "C"
