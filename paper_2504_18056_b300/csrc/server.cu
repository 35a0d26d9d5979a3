// server.cu -- continuous batching of frame updates from many filter sessions.
//
// Each session is a full filter context (particles, keyframe poses, tables and
// scratch resident in HBM). Frames arrive with their scan and odometry; a tick
// takes, for up to kMaxSlots sessions that have a pending frame and no frame on
// the GPU, the oldest pending frame each, writes the argument records of every
// kernel of those frames into a descriptor block, and replays a CUDA graph that
// copies the block to the device and runs the whole frame for all of them with
// one persistent launch per kernel family (the same kernel bodies as the
// single-session path, walking a work list of session blocks). Two descriptor
// blocks, each with its own graph and stream, let a second tick start on other
// sessions while the first is still on the GPU, so frames that arrive
// mid-tick do not wait for it. A host node at the end of each graph stamps the
// completion time; latency = completion - arrival.
//
// Admission is by device memory: a session opens only if its context and
// table estimate fit the remaining budget; closing a session returns its share.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/gmcs.h"
#include "context.h"
#include "kernels.h"

using namespace gmcs;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct TickDesc {
    BatchList<ScanPackArgs> pack;
    BatchList<KnnCovArgs> knn;       // GICP: scan normals
    BatchList<PredictArgs> pred;
    BatchList<SelectArgs> sel;
    BatchList<PassArgs> pgrad;
    BatchList<FinishArgs> fgrad;
    BatchList<PassArgs> pval;
    BatchList<FinishArgs> fval;
    BatchList<WeighArgs> weigh;
    BatchList<ScanArgs> scan;
    BatchList<TotalsArgs> tot;
    BatchList<SearchArgs> search;
    BatchList<GatherArgs> gather;
    BatchList<PruneArgs> prune;      // pruning policy: mark (scan blocks),
    BatchList<PruneArgs> ptot;       // totals (2 CTAs per session),
    BatchList<PruneArgs> pslot;      // spawn and reweigh (slot blocks)
};

template <typename A>
void list_clear(BatchList<A>& L) {
    L.count = 0;
    L.total = 0;
}

template <typename A>
void list_add(BatchList<A>& L, const A& a, int vgrid) {
    const int k = L.count++;
    L.args[k] = a;
    L.vgrid[k] = vgrid;
    L.offset[k] = L.total;
    L.total += vgrid;
}

struct Frame {
    uint64_t ticket = 0;
    int sid = 0;
    int ring_slot = 0;
    int N = 0;
    double dT[12];
    double cov[36];
    double t_arrive = 0.0;
};

struct Session {
    int id = 0;
    gmcs_ctx* ctx = nullptr;
    size_t bytes = 0;
    int Nmax = 0;
    bool ready = false;
    bool inflight = false;
    std::deque<Frame> pending;
    float* ring = nullptr;            // pinned scans, ring_slots x Nmax x 3
    std::vector<int> free_slots;
};

struct TickSet {
    cudaStream_t stream = nullptr;
    TickDesc* h_desc = nullptr;       // pinned
    TickDesc* d_desc = nullptr;
    WeighResult* d_res = nullptr;
    WeighResult* h_res = nullptr;     // pinned
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Frame> frames;
    std::vector<double> evals;
    std::atomic<double> t_start{0.0};
    std::atomic<double> t_done{0.0};
};

struct Result {
    gmcs_step_out out;
    double latency;
    int status;
};

void CUDART_CB stamp_start(void* p) { static_cast<TickSet*>(p)->t_start.store(now_s()); }
void CUDART_CB stamp_done(void* p) { static_cast<TickSet*>(p)->t_done.store(now_s()); }

constexpr int kRingSlots = 64;

}  // namespace

struct gmcs_server {
    gmcs_config cfg;
    int device = 0;
    size_t budget = 0, used = 0;
    int max_sessions = 0;
    cudaStream_t setup_stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::map<int, Session*> sessions;
    int next_sid = 1;
    uint64_t next_ticket = 1;
    std::map<uint64_t, Result> results;
    TickSet sets[2];
    std::vector<double> latencies;
    std::vector<std::pair<double, double>> busy;   // [start, done] of every tick, host clock
    uint64_t frames_done = 0, ticks = 0, slots_used = 0;
    double evals = 0.0, t_first = 0.0, t_last = 0.0;
    int max_inflight = 2;            // ticks on the GPU at once (1: strictly one after another)
    double tick_work = 4e8;          // evals (P x N x steps) a tick gathers beyond its oldest frame; 0: no cap
    std::thread worker;
    std::atomic<bool> running{false};
};

namespace {

int capture_graph(gmcs_server* s, TickSet& t) {
    cudaStream_t st = t.stream;
    TickDesc* d = t.d_desc;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GMCS_E_CUDA;
    cudaLaunchHostFunc(st, stamp_start, &t);
    cudaMemcpyAsync(d, t.h_desc, sizeof(TickDesc), cudaMemcpyHostToDevice, st);
    const bool gicp = s->cfg.model == GMCS_MODEL_GICP;
    launch_scan_pack_b(&d->pack, st);
    if (gicp) launch_knn_cov_b(&d->knn, s->cfg.knn, st);
    launch_predict_b(&d->pred, st);
    launch_select_b(&d->sel, st);
    for (int k = 0; k < s->cfg.steps; ++k) {
        if (gicp) launch_gicp_b(&d->pgrad, true, st);
        else launch_pass3_b(&d->pgrad, s->cfg.table_dtype, true, s->cfg.table_layout == GMCS_LAYOUT_COLUMNS, st);
        launch_finish_b(&d->fgrad, true, gicp, st);
    }
    if (gicp) launch_gicp_b(&d->pval, false, st);
    else launch_pass3_b(&d->pval, s->cfg.table_dtype, false, s->cfg.table_layout == GMCS_LAYOUT_COLUMNS, st);
    launch_finish_b(&d->fval, false, gicp, st);
    launch_weigh_b(&d->weigh, st);
    if (s->cfg.resample == GMCS_RESAMPLE_PRUNE) {
        launch_prune_mark_b(&d->prune, st);
        launch_prune_totals_b(&d->ptot, st);
        launch_prune_spawn_b(&d->pslot, st);
        launch_prune_reweigh_b(&d->pslot, st);
    } else {
        launch_resample_scan_b(&d->scan, st);
        launch_scan_totals_b(&d->tot, st);
        launch_resample_search_b(&d->search, st);
        launch_gather_b(&d->gather, st);
    }
    cudaMemcpyAsync(t.h_res, t.d_res, sizeof(WeighResult) * kMaxSlots, cudaMemcpyDeviceToHost, st);
    cudaLaunchHostFunc(st, stamp_done, &t);
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(st, &g) != cudaSuccess || !g) {
        cudaGetLastError();
        return GMCS_E_CUDA;
    }
    const cudaError_t e = cudaGraphInstantiate(&t.exec, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? GMCS_OK : GMCS_E_CUDA;
}

// Completed ticks -> results (caller holds the lock).
void collect(gmcs_server* s) {
    for (TickSet& t : s->sets) {
        if (!t.busy) continue;
        const cudaError_t q = cudaEventQuery(t.done);
        if (q == cudaErrorNotReady) {
            cudaGetLastError();
            continue;
        }
        const double t_done = t.t_done.load();
        for (size_t k = 0; k < t.frames.size(); ++k) {
            const Frame& f = t.frames[k];
            Result r;
            std::memset(&r, 0, sizeof(r));
            auto it = s->sessions.find(f.sid);
            const uint32_t frame = it != s->sessions.end() ? it->second->ctx->frame - 1 : 0;
            fill_out(t.h_res[k], frame, &r.out);
            r.status = (q == cudaSuccess) ? r.out.status : GMCS_E_CUDA;
            r.latency = t_done - f.t_arrive;
            s->results[f.ticket] = r;
            s->latencies.push_back(r.latency);
            s->evals += t.evals[k];
            if (it != s->sessions.end()) {
                it->second->inflight = false;
                it->second->free_slots.push_back(f.ring_slot);
            }
        }
        s->frames_done += t.frames.size();
        s->t_last = std::max(s->t_last, t_done);
        s->busy.emplace_back(t.t_start.load(), t_done);
        t.frames.clear();
        t.evals.clear();
        t.busy = false;
    }
}

// Launch one tick on a free descriptor block, if any session has a frame ready
// (caller holds the lock). Returns the number of sessions in the tick.
int launch_tick(gmcs_server* s) {
    TickSet* t = nullptr;
    int busy = 0;
    for (TickSet& c : s->sets) busy += c.busy ? 1 : 0;
    if (busy >= s->max_inflight) return 0;
    for (TickSet& c : s->sets)
        if (!c.busy) { t = &c; break; }
    if (!t) return 0;
    std::vector<Session*> cand;
    for (auto& kv : s->sessions) {
        Session* ss = kv.second;
        if (ss->ready && !ss->inflight && !ss->pending.empty()) cand.push_back(ss);
    }
    if (cand.empty()) return 0;
    std::sort(cand.begin(), cand.end(),
              [](Session* a, Session* b) { return a->pending.front().t_arrive < b->pending.front().t_arrive; });
    if ((int)cand.size() > kMaxSlots) cand.resize(kMaxSlots);
    // a tick's persistent launches end when its largest frame is done, so every
    // session in it waits for that frame: after the oldest frame, add frames (oldest
    // first) only while the tick's work stays under the cap. The frames left out go
    // to the next tick, which runs beside this one on the other stream.
    if (s->tick_work > 0.0) {
        std::vector<Session*> keep;
        double work = 0.0;
        for (Session* ss : cand) {
            const double wk = (double)ss->ctx->P * ss->pending.front().N * std::max(s->cfg.steps, 1);
            if (!keep.empty() && work + wk > s->tick_work) continue;
            keep.push_back(ss);
            work += wk;
        }
        cand.swap(keep);
    }
    TickDesc& D = *t->h_desc;
    list_clear(D.pack); list_clear(D.knn); list_clear(D.pred); list_clear(D.sel); list_clear(D.pgrad); list_clear(D.fgrad);
    list_clear(D.pval); list_clear(D.fval); list_clear(D.weigh); list_clear(D.scan); list_clear(D.tot);
    list_clear(D.search); list_clear(D.gather); list_clear(D.prune); list_clear(D.ptot); list_clear(D.pslot);
    for (size_t k = 0; k < cand.size(); ++k) {
        Session* ss = cand[k];
        gmcs_ctx* c = ss->ctx;
        Frame f = ss->pending.front();
        ss->pending.pop_front();
        if (f.N > 0)
            cudaMemcpyAsync(c->stage, ss->ring + (size_t)f.ring_slot * ss->Nmax * 3, sizeof(float) * 3 * (size_t)f.N,
                            cudaMemcpyHostToDevice, t->stream);
        const uint32_t frame = c->frame;
        c->path_now += std::sqrt(f.dT[3] * f.dT[3] + f.dT[7] * f.dT[7] + f.dT[11] * f.dT[11]);
        list_add(D.pack, ScanPackArgs{c->stage, f.N, c->scan}, grid_scan_pack(f.N));
        if (s->cfg.model == GMCS_MODEL_GICP) {
            KnnCovArgs ka;
            ka.pts = c->scan;
            ka.n = f.N;
            ka.k = s->cfg.knn;
            ka.eps = (double)s->cfg.cov_eps;
            ka.cov64 = nullptr;
            ka.nrm32 = c->scov;
            list_add(D.knn, ka, grid_knn_cov(f.N));
        }
        list_add(D.pred, predict_args(c, f.dT, f.cov, nullptr, frame), grid_per_particle(c->P));
        list_add(D.sel, select_args(c, nullptr), grid_per_particle(c->P));
        PassArgs pa;
        FinishArgs fa;
        pass_args(c, f.N, true, true, nullptr, nullptr, nullptr, nullptr, nullptr, &pa, &fa);
        list_add(D.pgrad, pa, grid_pass(pa));
        list_add(D.fgrad, fa, grid_per_particle(c->P));
        pass_args(c, f.N, false, false, c->ll, nullptr, nullptr, c->logw, nullptr, &pa, &fa);
        list_add(D.pval, pa, grid_pass(pa));
        list_add(D.fval, fa, grid_per_particle(c->P));
        WeighResult* res = t->d_res + k;
        list_add(D.weigh, weigh_args(c, nullptr, res), weigh_blocks(c->P));
        if (s->cfg.resample == GMCS_RESAMPLE_PRUNE) {
            // dead slots are refilled in place: the state buffer stays current
            const PruneArgs pa = prune_args(c, c->P, res, nullptr, c->ll, 0.0, 1, frame, true);
            list_add(D.prune, pa, pa.nblocks);
            list_add(D.ptot, pa, 2);
            list_add(D.pslot, pa, grid_prune_slots(c->P));
        } else {
            ScanArgs sa;
            TotalsArgs ta;
            SearchArgs se;
            resample_args(c, c->P, nullptr, res, c->w, 0.0, 1, frame, c->anc, &sa, &ta, &se);
            list_add(D.scan, sa, grid_resample_scan(c->P));
            list_add(D.tot, ta, 1);
            list_add(D.search, se, grid_resample_search(c->P));
            const GatherArgs g = gather_args(c, res);
            list_add(D.gather, g, grid_gather(g));
            // the gather writes the other buffer of the pair: it is current from the next frame on
            c->cur = 1 - c->cur;
        }
        c->frame = frame + 1;
        c->frames++;
        c->version++;
        c->last_valid = true;
        ss->inflight = true;
        t->frames.push_back(f);
        t->evals.push_back((double)c->P * f.N * s->cfg.steps);
    }
    if (cudaGraphLaunch(t->exec, t->stream) != cudaSuccess || cudaEventRecord(t->done, t->stream) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    t->busy = true;
    s->ticks++;
    s->slots_used += cand.size();
    return (int)cand.size();
}

void pump_locked(gmcs_server* s) {
    collect(s);
    while (launch_tick(s) > 0) {
    }
}

void worker_loop(gmcs_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (s->running.load()) {
        pump_locked(s);
        s->cv.notify_all();
        s->cv.wait_for(lock, std::chrono::microseconds(100));
    }
}

}  // namespace

extern "C" {

int gmcs_server_create(const gmcs_config* cfg, uint64_t budget_bytes, int max_sessions, gmcs_server** out) {
    if (!out) return GMCS_E_INVALID;
    *out = nullptr;
    if (!cfg || budget_bytes == 0 || max_sessions <= 0 || cfg->k_nb != 3 || cfg->steps < 0 || cfg->steps > 64)
        return GMCS_E_INVALID;
    gmcs_server* s = new (std::nothrow) gmcs_server();
    if (!s) return GMCS_E_OOM;
    s->cfg = *cfg;
    s->budget = budget_bytes;
    s->max_sessions = max_sessions;
    cudaGetDevice(&s->device);
    prepare_filter_batched();
    prepare_weights_batched();
    prepare_gicp_batched();
    int rc = GMCS_OK;
    if (cudaStreamCreateWithFlags(&s->setup_stream, cudaStreamNonBlocking) != cudaSuccess) rc = GMCS_E_CUDA;
    for (TickSet& t : s->sets) {
        if (rc) break;
        if (cudaStreamCreateWithFlags(&t.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess) {
            rc = GMCS_E_CUDA;
            break;
        }
        if (cudaMallocHost((void**)&t.h_desc, sizeof(TickDesc)) != cudaSuccess ||
            cudaMallocHost((void**)&t.h_res, sizeof(WeighResult) * kMaxSlots) != cudaSuccess ||
            cudaMalloc((void**)&t.d_desc, sizeof(TickDesc)) != cudaSuccess ||
            cudaMalloc((void**)&t.d_res, sizeof(WeighResult) * kMaxSlots) != cudaSuccess) {
            cudaGetLastError();
            rc = GMCS_E_OOM;
            break;
        }
        std::memset(t.h_desc, 0, sizeof(TickDesc));
        rc = capture_graph(s, t);
    }
    if (rc) {
        gmcs_server_destroy(s);
        return rc;
    }
    *out = s;
    return GMCS_OK;
}

int gmcs_server_set_inflight(gmcs_server* s, int ticks) {
    if (!s || ticks < 1 || ticks > 2) return GMCS_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    s->max_inflight = ticks;
    return GMCS_OK;
}

int gmcs_server_set_tick_work(gmcs_server* s, double max_evals) {
    if (!s || !(max_evals >= 0.0)) return GMCS_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    s->tick_work = max_evals;
    return GMCS_OK;
}

int gmcs_server_start(gmcs_server* s) {
    if (!s) return GMCS_E_INVALID;
    if (s->running.exchange(true)) return GMCS_OK;
    s->worker = std::thread(worker_loop, s);
    return GMCS_OK;
}

int gmcs_server_stop(gmcs_server* s) {
    if (!s) return GMCS_E_INVALID;
    if (s->running.exchange(false) && s->worker.joinable()) {
        s->cv.notify_all();
        s->worker.join();
    }
    return GMCS_OK;
}

int gmcs_server_pump(gmcs_server* s) {
    if (!s) return GMCS_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    pump_locked(s);
    return GMCS_OK;
}

int gmcs_server_open(gmcs_server* s, int max_particles, int max_keyframes, int max_points, uint64_t table_bytes,
                     uint64_t seed, int* sid) {
    if (!s || !sid || max_particles <= 0 || max_keyframes < 3 || max_points <= 0) return GMCS_E_INVALID;
    const size_t est = ctx_device_bytes(max_particles, max_keyframes, max_points) + (size_t)table_bytes;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if ((int)s->sessions.size() >= s->max_sessions || s->used + est > s->budget) return GMCS_E_BUDGET;
        s->used += est;   // reserved while the context is created
    }
    Session* ss = new (std::nothrow) Session();
    int rc = ss ? GMCS_OK : GMCS_E_OOM;
    gmcs_config cfg = s->cfg;
    cfg.seed = seed;
    if (!rc) rc = gmcs_create(&cfg, max_particles, max_keyframes, max_points, s->setup_stream, &ss->ctx);
    if (!rc && cudaMallocHost((void**)&ss->ring, sizeof(float) * 3 * (size_t)max_points * kRingSlots) != cudaSuccess) {
        cudaGetLastError();
        rc = GMCS_E_OOM;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (rc) {
        s->used -= est;
        if (ss) {
            if (ss->ctx) gmcs_destroy(ss->ctx);
            if (ss->ring) cudaFreeHost(ss->ring);
            delete ss;
        }
        return rc;
    }
    ss->id = s->next_sid++;
    ss->bytes = est;
    ss->Nmax = max_points;
    for (int k = kRingSlots - 1; k >= 0; --k) ss->free_slots.push_back(k);
    s->sessions[ss->id] = ss;
    *sid = ss->id;
    return GMCS_OK;
}

int gmcs_server_context(gmcs_server* s, int sid, gmcs_ctx** ctx) {
    if (!s || !ctx) return GMCS_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->sessions.find(sid);
    if (it == s->sessions.end()) return GMCS_E_INVALID;
    *ctx = it->second->ctx;
    return GMCS_OK;
}

int gmcs_server_ready(gmcs_server* s, int sid) {
    if (!s) return GMCS_E_INVALID;
    Session* ss = nullptr;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->sessions.find(sid);
        if (it == s->sessions.end()) return GMCS_E_INVALID;
        ss = it->second;
    }
    if (cudaStreamSynchronize(s->setup_stream) != cudaSuccess) return GMCS_E_CUDA;
    if (!ss->ctx->have_particles || ss->ctx->K < 3) return GMCS_E_STATE;
    std::lock_guard<std::mutex> lock(s->mu);
    // replace the estimate by what the session actually holds
    const size_t actual = ss->ctx->dev_bytes;
    s->used = s->used - ss->bytes + actual;
    ss->bytes = actual;
    ss->ready = true;
    return GMCS_OK;
}

int gmcs_server_submit(gmcs_server* s, int sid, const float* scan, int N, const double delta_T[12],
                       const double cov[36], uint64_t* ticket) {
    if (!s || !delta_T || !cov || !ticket || N < 0 || (N > 0 && !scan)) return GMCS_E_INVALID;
    for (int e = 0; e < 12; ++e)
        if (!std::isfinite(delta_T[e])) return GMCS_E_INVALID;
    for (int e = 0; e < 36; ++e)
        if (!std::isfinite(cov[e])) return GMCS_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->sessions.find(sid);
    if (it == s->sessions.end()) return GMCS_E_INVALID;
    Session* ss = it->second;
    if (!ss->ready) return GMCS_E_STATE;
    if (N > ss->Nmax) return GMCS_E_CAPACITY;
    if (ss->free_slots.empty()) return GMCS_E_CAPACITY;   // backpressure: too many frames queued
    Frame f;
    f.ticket = s->next_ticket++;
    f.sid = sid;
    f.ring_slot = ss->free_slots.back();
    ss->free_slots.pop_back();
    f.N = N;
    std::memcpy(f.dT, delta_T, sizeof(f.dT));
    std::memcpy(f.cov, cov, sizeof(f.cov));
    if (N > 0) std::memcpy(ss->ring + (size_t)f.ring_slot * ss->Nmax * 3, scan, sizeof(float) * 3 * (size_t)N);
    f.t_arrive = now_s();
    if (s->t_first == 0.0) s->t_first = f.t_arrive;
    ss->pending.push_back(f);
    *ticket = f.ticket;
    s->cv.notify_all();
    return GMCS_OK;
}

int gmcs_server_poll(gmcs_server* s, uint64_t ticket, gmcs_step_out* out, double* latency_s) {
    if (!s) return GMCS_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->running.load()) pump_locked(s);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return GMCS_PENDING;
    if (out) *out = it->second.out;
    if (latency_s) *latency_s = it->second.latency;
    const int st = it->second.status;
    s->results.erase(it);
    return st == GMCS_E_NONFINITE ? GMCS_OK : st;
}

int gmcs_server_close(gmcs_server* s, int sid) {
    if (!s) return GMCS_E_INVALID;
    Session* ss = nullptr;
    {
        std::unique_lock<std::mutex> lock(s->mu);
        auto it = s->sessions.find(sid);
        if (it == s->sessions.end()) return GMCS_E_INVALID;
        ss = it->second;
        // frames still queued are dropped; a frame on the GPU is waited for
        for (const Frame& f : ss->pending) {
            Result r;
            std::memset(&r, 0, sizeof(r));
            r.status = GMCS_E_STATE;
            s->results[f.ticket] = r;
        }
        ss->pending.clear();
        while (ss->inflight) {
            if (s->running.load()) {
                s->cv.wait_for(lock, std::chrono::milliseconds(1));
            } else {
                lock.unlock();
                for (TickSet& t : s->sets)
                    if (t.busy) cudaEventSynchronize(t.done);
                lock.lock();
                pump_locked(s);
            }
        }
        s->sessions.erase(sid);
        s->used -= std::min(s->used, ss->bytes);
    }
    gmcs_destroy(ss->ctx);
    cudaFreeHost(ss->ring);
    delete ss;
    return GMCS_OK;
}

int gmcs_server_drain(gmcs_server* s) {
    if (!s) return GMCS_E_INVALID;
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            pump_locked(s);
            bool idle = !s->sets[0].busy && !s->sets[1].busy;
            for (auto& kv : s->sessions) idle = idle && kv.second->pending.empty();
            if (idle) return GMCS_OK;
        }
        for (TickSet& t : s->sets)
            if (t.busy) cudaEventSynchronize(t.done);
    }
}

int gmcs_server_get_stats(gmcs_server* s, gmcs_server_stats* out) {
    if (!s || !out) return GMCS_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->frames = s->frames_done;
    out->ticks = s->ticks;
    out->sessions = (int)s->sessions.size();
    out->used_bytes = s->used;
    out->budget_bytes = s->budget;
    out->evals = s->evals;
    out->span_s = (s->t_last > s->t_first) ? s->t_last - s->t_first : 0.0;
    out->mean_sessions_per_tick = s->ticks ? (double)s->slots_used / s->ticks : 0.0;
    {   // union of the tick intervals: time with at least one tick on the GPU
        std::vector<std::pair<double, double>> b = s->busy;
        std::sort(b.begin(), b.end());
        double total = 0.0, cs = 0.0, ce = -1.0;
        for (auto& iv : b) {
            if (iv.first > ce) {
                if (ce > cs) total += ce - cs;
                cs = iv.first;
                ce = iv.second;
            } else {
                ce = std::max(ce, iv.second);
            }
        }
        if (ce > cs) total += ce - cs;
        out->busy_s = total;
    }
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            const double pos = q * (l.size() - 1);
            const size_t lo = (size_t)std::floor(pos), hi = std::min(l.size() - 1, lo + 1);
            return l[lo] + (l[hi] - l[lo]) * (pos - lo);
        };
        out->latency_p50_s = pct(0.50);
        out->latency_p99_s = pct(0.99);
        out->latency_max_s = l.back();
        double m = 0.0;
        for (double v : l) m += v;
        out->latency_mean_s = m / l.size();
    }
    return GMCS_OK;
}

int gmcs_server_reset_stats(gmcs_server* s) {
    if (!s) return GMCS_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    s->latencies.clear();
    s->busy.clear();
    s->frames_done = s->ticks = s->slots_used = 0;
    s->evals = 0.0;
    s->t_first = s->t_last = 0.0;
    return GMCS_OK;
}

int gmcs_server_destroy(gmcs_server* s) {
    if (!s) return GMCS_OK;
    gmcs_server_stop(s);
    std::vector<int> ids;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (auto& kv : s->sessions) ids.push_back(kv.first);
    }
    for (int id : ids) gmcs_server_close(s, id);
    for (TickSet& t : s->sets) {
        if (t.stream) cudaStreamSynchronize(t.stream);
        if (t.exec) cudaGraphExecDestroy(t.exec);
        if (t.done) cudaEventDestroy(t.done);
        if (t.stream) cudaStreamDestroy(t.stream);
        if (t.h_desc) cudaFreeHost(t.h_desc);
        if (t.h_res) cudaFreeHost(t.h_res);
        if (t.d_desc) cudaFree(t.d_desc);
        if (t.d_res) cudaFree(t.d_res);
    }
    if (s->setup_stream) cudaStreamDestroy(s->setup_stream);
    cudaGetLastError();
    delete s;
    return GMCS_OK;
}

}  // extern "C"
