// server.cu -- a continuous-batching request runtime over sse_state.
//
// Requests (a mesh, parameters, an initial state, a scheme and a horizon of
// n_steps large steps) are queued in arrival order.  One worker thread admits
// them while their device footprint (sse_state_footprint) fits the HBM budget
// and the active-slot limit, gives each admitted request its own non-blocking
// stream and a resident state, and then keeps every active request's stream
// fed with `steps_per_launch` large steps at a time, so the work of all
// active requests overlaps on the device.  Requests that arrive while others
// run are admitted as soon as a slot and memory free up.  A finished request
// reads its (u, h, tracers) back into the caller's buffers, frees its state
// (stream-ordered, no device-wide synchronisation) and releases its memory.
// Each request's arithmetic is that of sse_step on its own state: results
// do not depend on what else runs.
#include <stdint.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <algorithm>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sse.h"

namespace {

struct Req {
    int64_t id = 0;
    const sse_mesh *mesh = nullptr;
    sse_params prm{};
    int order = 3, M = 1, n_steps = 0;
    double dt = 0.0;
    int nE = 0, nC = 0, L = 0;
    std::vector<double> u, h, tr, wind;  // host copies of the inputs
    double *u_out = nullptr, *h_out = nullptr, *tr_out = nullptr;
    size_t footprint = 0;
    sse_tuning tun{};
    int steps_done = 0, inflight = 0, inflight_alone = 0;
    sse_state *st = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = SSE_REQ_PENDING;
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

// a packed group: the active requests of one precision and order advanced
// together by sse_step_batch (3-D kernels of all of them in one launch)
struct PackGroup {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<Req *> members;   // the members of the round in flight
    int k = 0;                    // steps of the round in flight (0: idle)
};

struct sse_server {
    int device = 0;
    size_t budget = 0, used = 0, peak = 0;
    int max_active = 1, chunk = 1, tune = -1, flags = 0;
    std::unordered_map<int, PackGroup> groups;    // by precision * 4 + order
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::vector<Req *> active;                    // owned by the worker
    std::unordered_map<int64_t, Req *> reqs;
    int64_t next_id = 1;
    int n_active = 0, max_seen_active = 0;
    bool stop = false;
    std::thread worker;
    std::vector<cudaStream_t> streams;            // recycled streams and events
    std::vector<cudaEvent_t> events;
};

namespace {

void fail(sse_server *S, Req *r, int code) {
    if (r->st) sse_state_destroy(r->st);
    r->st = nullptr;
    if (r->s) S->streams.push_back(r->s);
    if (r->ev) S->events.push_back(r->ev);
    r->s = nullptr;
    r->ev = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= r->footprint;
    S->n_active--;
    r->status = code;
    r->t_done = now_s(S->t0);
    S->cv_done.notify_all();
}

int start(sse_server *S, Req *r) {
    if (!S->streams.empty()) {
        r->s = S->streams.back();
        S->streams.pop_back();
    } else if (cudaStreamCreateWithFlags(&r->s, cudaStreamNonBlocking) != cudaSuccess) {
        return SSE_ERR_CUDA;
    }
    if (!S->events.empty()) {
        r->ev = S->events.back();
        S->events.pop_back();
    } else if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
        return SSE_ERR_CUDA;
    }
    int rc = sse_state_create_ex(r->mesh, &r->prm, &r->tun, r->s, &r->st);
    if (rc) return rc;
    rc = sse_state_set(r->st, SSE_FIELD_U, r->u.data());
    if (!rc) rc = sse_state_set(r->st, SSE_FIELD_H, r->h.data());
    for (int t = 0; !rc && t < r->prm.nTracers; t++)
        rc = sse_state_set(r->st, SSE_FIELD_TRACER0 + t, r->tr.data() + (size_t)t * r->nC * r->L);
    if (!rc && !r->wind.empty()) rc = sse_state_set(r->st, SSE_FIELD_WIND, r->wind.data());
    // the inputs are on the device now
    std::vector<double>().swap(r->u);
    std::vector<double>().swap(r->h);
    std::vector<double>().swap(r->tr);
    std::vector<double>().swap(r->wind);
    return rc;
}

int finish(Req *r) {
    int rc = sse_state_get(r->st, SSE_FIELD_U, r->u_out);
    if (!rc) rc = sse_state_get(r->st, SSE_FIELD_H, r->h_out);
    for (int t = 0; !rc && t < r->prm.nTracers; t++)
        rc = sse_state_get(r->st, SSE_FIELD_TRACER0 + t, r->tr_out + (size_t)t * r->nC * r->L);
    sse_state_destroy(r->st);
    r->st = nullptr;
    return rc;
}

// release a finished or failed request's slot
void retire(sse_server *S, Req *r, int rc) {
    if (r->st) {
        sse_state_destroy(r->st);
        r->st = nullptr;
    }
    S->streams.push_back(r->s);
    S->events.push_back(r->ev);
    r->s = nullptr;
    r->ev = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= r->footprint;
    S->n_active--;
    r->status = rc ? rc : SSE_REQ_DONE;
    r->t_done = now_s(S->t0);
    S->cv_done.notify_all();
}

// Packed mode: the active requests of each (precision, order) advance in
// rounds of k steps, all of them in one sse_step_batch call on the group's
// stream; between rounds finished requests retire and new ones join.
// Requests whose states cannot be packed step alone, as in the default mode.
bool packed_round(sse_server *S) {
    bool progressed = false;
    // rounds in flight: account for the finished ones
    for (auto &kv : S->groups) {
        PackGroup &g = kv.second;
        if (!g.k) continue;
        const cudaError_t q = cudaEventQuery(g.ev);
        if (q == cudaErrorNotReady) continue;
        for (Req *r : g.members) { r->steps_done += g.k; r->inflight = 0; }
        g.members.clear();
        g.k = 0;
        progressed = true;
    }
    // requests stepping alone (not packable) in flight
    for (Req *r : S->active) {
        if (r->inflight && r->inflight_alone && cudaEventQuery(r->ev) != cudaErrorNotReady) {
            r->steps_done += r->inflight;
            r->inflight = 0;
            r->inflight_alone = 0;
            progressed = true;
        }
    }
    // retire the finished
    for (size_t i = 0; i < S->active.size();) {
        Req *r = S->active[i];
        if (r->inflight || r->steps_done < r->n_steps) { i++; continue; }
        const int rc = finish(r);
        S->active.erase(S->active.begin() + i);
        retire(S, r, rc);
        progressed = true;
    }
    // start the next round of every idle group
    std::unordered_map<int, std::vector<Req *>> ready;
    for (Req *r : S->active)
        if (!r->inflight) ready[r->prm.precision * 4 + r->order].push_back(r);
    for (auto &kv : ready) {
        PackGroup &g = S->groups[kv.first];
        if (g.k) continue;   // still running; these requests wait for it
        if (!g.s && (cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming) != cudaSuccess))
            continue;
        std::vector<Req *> &rs = kv.second;
        int k = S->chunk;
        for (Req *r : rs) k = std::min(k, r->n_steps - r->steps_done);
        std::vector<sse_state *> sts;
        std::vector<double> dts;
        std::vector<int32_t> Ms;
        for (Req *r : rs) { sts.push_back(r->st); dts.push_back(r->dt); Ms.push_back(r->M); }
        int rc = sse_step_batch(sts.data(), (int)sts.size(), rs[0]->order, dts.data(), Ms.data(),
                                k, g.s);
        if (rc == SSE_OK && cudaEventRecord(g.ev, g.s) == cudaSuccess) {
            g.members = rs;
            g.k = k;
            for (Req *r : rs) r->inflight = k;
            progressed = true;
            continue;
        }
        // not packable: each steps alone on its own stream
        for (Req *r : rs) {
            const int kk = std::min(S->chunk, r->n_steps - r->steps_done);
            int rr = sse_step(r->st, r->order, r->dt, r->M, kk);
            if (!rr && cudaEventRecord(r->ev, r->s) != cudaSuccess) rr = SSE_ERR_CUDA;
            if (rr) {
                S->active.erase(std::find(S->active.begin(), S->active.end(), r));
                retire(S, r, rr);
            } else {
                r->inflight = kk;
                r->inflight_alone = 1;
            }
            progressed = true;
        }
    }
    return progressed;
}

void worker_loop(sse_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Req *> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop && S->active.empty()) break;
            // admission in arrival order: the head waits until it fits
            while (!S->stop && !S->pending.empty() &&
                   S->n_active + (int)admit.size() < S->max_active) {
                Req *r = S->pending.front();
                if (S->used + r->footprint > S->budget) break;
                S->pending.pop_front();
                S->used += r->footprint;
                S->peak = std::max(S->peak, S->used);
                r->status = SSE_REQ_ACTIVE;
                r->t_admit = now_s(S->t0);
                admit.push_back(r);
            }
            S->n_active += (int)admit.size();
            S->max_seen_active = std::max(S->max_seen_active, S->n_active);
        }
        for (Req *r : admit) {
            const int rc = start(S, r);
            if (rc) {
                fail(S, r, rc);
                continue;
            }
            S->active.push_back(r);
        }
        bool progressed = !admit.empty();
        if (S->flags & SSE_SERVER_PACKED) {
            progressed = packed_round(S) || progressed;
            if (!progressed) {
                std::unique_lock<std::mutex> lk(S->mu);
                S->cv_work.wait_for(lk, std::chrono::microseconds(50));
            }
            continue;
        }
        for (size_t i = 0; i < S->active.size();) {
            Req *r = S->active[i];
            if (r->inflight) {
                const cudaError_t q = cudaEventQuery(r->ev);
                if (q == cudaErrorNotReady) { i++; continue; }
                r->steps_done += r->inflight;
                r->inflight = 0;
                progressed = true;
            }
            int rc = SSE_OK;
            if (r->steps_done < r->n_steps) {
                const int k = std::min(S->chunk, r->n_steps - r->steps_done);
                rc = sse_step(r->st, r->order, r->dt, r->M, k);
                if (!rc && cudaEventRecord(r->ev, r->s) != cudaSuccess) rc = SSE_ERR_CUDA;
                if (!rc) {
                    r->inflight = k;
                    progressed = true;
                    i++;
                    continue;
                }
            } else {
                rc = finish(r);
            }
            // finished or failed: release the slot
            if (r->st) {
                sse_state_destroy(r->st);
                r->st = nullptr;
            }
            S->streams.push_back(r->s);
            S->events.push_back(r->ev);
            r->s = nullptr;
            r->ev = nullptr;
            S->active.erase(S->active.begin() + i);
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->used -= r->footprint;
                S->n_active--;
                r->status = rc ? rc : SSE_REQ_DONE;
                r->t_done = now_s(S->t0);
                S->cv_done.notify_all();
            }
            progressed = true;
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : S->events) cudaEventDestroy(e);
    for (auto &kv : S->groups) {
        if (kv.second.s) cudaStreamDestroy(kv.second.s);
        if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    }
    S->streams.clear();
    S->events.clear();
    S->groups.clear();
}

}  // namespace

extern "C" int sse_server_create(int device, size_t hbm_budget_bytes, int max_active,
                                 int steps_per_launch, int tune_objective, sse_server **out) {
    return sse_server_create_ex(device, hbm_budget_bytes, max_active, steps_per_launch,
                                tune_objective, 0, out);
}

extern "C" int sse_server_create_ex(int device, size_t hbm_budget_bytes, int max_active,
                                    int steps_per_launch, int tune_objective, int flags,
                                    sse_server **out) {
    if (!out || max_active < 1 || steps_per_launch < 1 || hbm_budget_bytes == 0 ||
        tune_objective < -1 || tune_objective > SSE_TUNE_THROUGHPUT ||
        (flags & ~SSE_SERVER_PACKED))
        return SSE_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return SSE_ERR_INVALID_ARG;
    sse_server *S = new (std::nothrow) sse_server();
    if (!S) return SSE_ERR_OOM;
    S->device = device;
    S->budget = hbm_budget_bytes;
    S->max_active = max_active;
    S->chunk = steps_per_launch;
    S->tune = tune_objective;
    S->flags = flags;
    S->t0 = std::chrono::steady_clock::now();
    // keep freed state memory in the device's pool for the next request
    cudaMemPool_t pool;
    if (cudaSetDevice(device) == cudaSuccess &&
        cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = hbm_budget_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    try {
        S->worker = std::thread(worker_loop, S);
    } catch (...) {
        delete S;
        return SSE_ERR_OOM;
    }
    *out = S;
    return SSE_OK;
}

extern "C" int sse_server_submit(sse_server *S, const sse_mesh *mesh, const sse_params *params,
                                 const double *u, const double *h, const double *tracers,
                                 const double *wind_stress, int order, double dt, int n_substeps,
                                 int n_steps, double *u_out, double *h_out, double *tracers_out,
                                 int64_t *id_out) {
    if (!S || !mesh || !params || !u || !h || !tracers || !u_out || !h_out || !tracers_out ||
        !id_out || n_steps < 0 || (order != 2 && order != 3) || !(dt > 0.0) || n_substeps < 1 ||
        params->nTracers < 1 || params->nTracers > 2)
        return SSE_ERR_INVALID_ARG;
    int32_t dims[4];
    int rc = sse_mesh_dims(mesh, dims);
    if (rc) return rc;
    const int nCells = dims[0], nEdges = dims[1], nLayers = dims[3];
    sse_tuning tun{};
    if (S->tune >= 0) {
        rc = sse_tune(mesh, params, S->tune, &tun);
        if (rc) return rc;
    }
    size_t fp = 0;
    rc = sse_state_footprint_ex(mesh, params, &tun, &fp);
    if (rc) return rc;
    if (fp > S->budget) return SSE_ERR_OOM;
    Req *r = new (std::nothrow) Req();
    if (!r) return SSE_ERR_OOM;
    r->mesh = mesh;
    r->prm = *params;
    r->order = order;
    r->dt = dt;
    r->M = n_substeps;
    r->n_steps = n_steps;
    r->nE = nEdges;
    r->nC = nCells;
    r->L = nLayers;
    r->footprint = fp;
    r->tun = tun;
    const size_t EL = (size_t)nEdges * nLayers, CL = (size_t)nCells * nLayers;
    try {
        r->u.assign(u, u + EL);
        r->h.assign(h, h + CL);
        r->tr.assign(tracers, tracers + CL * params->nTracers);
        if (wind_stress) r->wind.assign(wind_stress, wind_stress + nEdges);
    } catch (...) {
        delete r;
        return SSE_ERR_OOM;
    }
    r->u_out = u_out;
    r->h_out = h_out;
    r->tr_out = tracers_out;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return SSE_ERR_INVALID_ARG;
        }
        // registered in both containers or in neither: a failed insertion
        // leaves no request that the worker would never see
        const int64_t id = S->next_id;
        r->id = id;
        r->t_submit = now_s(S->t0);
        try {
            S->reqs[id] = r;
            S->pending.push_back(r);
        } catch (...) {
            S->reqs.erase(id);
            delete r;
            return SSE_ERR_OOM;
        }
        S->next_id++;
        *id_out = id;
    }
    S->cv_work.notify_one();
    return SSE_OK;
}

static void fill_info(const Req *r, sse_request_info *info) {
    info->id = r->id;
    info->status = r->status;
    info->steps_done = r->steps_done;
    info->t_submit = r->t_submit;
    info->t_admit = r->t_admit;
    info->t_done = r->t_done;
    info->footprint = r->footprint;
}

extern "C" int sse_server_query(sse_server *S, int64_t id, sse_request_info *info) {
    if (!S || !info) return SSE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return SSE_ERR_INVALID_ARG;
    fill_info(it->second, info);
    return SSE_OK;
}

extern "C" int sse_server_wait(sse_server *S, int64_t id, double timeout_s,
                               sse_request_info *info) {
    if (!S || !info) return SSE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return SSE_ERR_INVALID_ARG;
    Req *r = it->second;
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                           std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
    S->cv_done.wait_until(lk, until, [&] {
        return r->status != SSE_REQ_PENDING && r->status != SSE_REQ_ACTIVE;
    });
    fill_info(r, info);
    return (r->status == SSE_REQ_PENDING || r->status == SSE_REQ_ACTIVE) ? SSE_ERR_TIMEOUT
                                                                            : SSE_OK;
}

extern "C" int sse_server_release(sse_server *S, int64_t id) {
    if (!S) return SSE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return SSE_ERR_INVALID_ARG;
    Req *r = it->second;
    if (r->status == SSE_REQ_PENDING || r->status == SSE_REQ_ACTIVE) return SSE_ERR_INVALID_ARG;
    S->reqs.erase(it);
    delete r;
    return SSE_OK;
}

extern "C" int sse_server_stats(sse_server *S, sse_server_info *info) {
    if (!S || !info) return SSE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    info->pending = (int32_t)S->pending.size();
    info->active = S->n_active;
    info->max_active_seen = S->max_seen_active;
    info->used_bytes = S->used;
    info->peak_bytes = S->peak;
    info->budget_bytes = S->budget;
    return SSE_OK;
}

extern "C" void sse_server_destroy(sse_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // requests not yet admitted are cancelled; admitted ones run to the end
        for (Req *r : S->pending) r->status = SSE_ERR_CANCELLED;
        S->pending.clear();
        S->cv_done.notify_all();
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
}
