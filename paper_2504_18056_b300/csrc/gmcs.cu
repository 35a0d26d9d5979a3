// gmcs.cu -- the C ABI (include/gmcs.h): context, state, and the frame driver.
//
// The host side only validates arguments, moves caller buffers into the
// context's device layout and enqueues kernels on the context stream; every
// step of the per-frame path runs in the kernels of k_filter.cu and
// k_weights.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gmcs.h"
#include "context.h"
#include "kernels.h"

using namespace gmcs;

static_assert(sizeof(gmcs_config) == 104, "gmcs_config layout is part of the ABI");
static_assert(sizeof(gmcs_step_out) == 152, "gmcs_step_out layout is part of the ABI");
static_assert(sizeof(gmcs_grid) == 48, "gmcs_grid layout is part of the ABI");

namespace {

const char* kKindName[K_COUNT] = {"predict", "select", "pass_grad", "pass_value", "finish",
                                  "weigh", "resample", "gather", "table", "layout"};

}  // namespace

namespace gmcs {

// Chunking of the scan for the lookup pass: a CTA covers kPassTW particle tiles
// x kPassCW point chunks; the number of chunk groups G gives several waves of
// CTAs on 148 SMs, at most kMaxGroups (the partial-sum scratch), chunks >= 8 points.
void pass_shape(int P, int N, int* ntiles, int* groups, int* chunk_len, int max_groups) {
    const int nt = (P + 31) / 32;
    const int ntg = (nt + kPassTW - 1) / kPassTW;
    const int target = 148 * 8 * 4;
    int g = (target + ntg - 1) / ntg;
    g = std::max(1, std::min(g, max_groups));
#ifdef GMCS_FORCE_GROUPS
    g = std::max(1, std::min(GMCS_FORCE_GROUPS, max_groups));
#endif
    const int max_chunks = std::max(1, (N + 7) / 8);
    while (g > 1 && g * kPassCW > max_chunks) --g;
    const int chunks = g * kPassCW;
    *ntiles = nt;
    *groups = g;
    *chunk_len = std::max(1, (N + chunks - 1) / chunks);
}

// Device bytes gmcs_create allocates for these capacities (tables excluded).
size_t ctx_device_bytes(int max_particles, int max_keyframes, int max_points) {
    const size_t ld = ((size_t)max_particles + 31) / 32 * 32;
    const size_t nb = (max_particles + kScanBlock - 1) / kScanBlock;
    const size_t part = std::max((size_t)kMaxGroups * kAccGrad * ld, (size_t)12 * ld);
    const size_t stage = std::max((size_t)3 * max_points, (size_t)6 * ld);
    size_t b = 0;
    b += 2 * (sizeof(float) * kPoseC * ld + sizeof(float) * kPoseC * ld * max_keyframes);
    b += sizeof(double) * ld * 2 + sizeof(float) * ld + sizeof(float) * 6 * ld;   // logw, w, ll, gbuf
    b += sizeof(int) * GMCS_MAX_NB * ld + sizeof(float) * part + sizeof(float4) * 2 * max_points + sizeof(float) * stage;
    b += sizeof(double) * kWeighPart * kWeighMaxBlocks + sizeof(unsigned) + sizeof(WeighResult);
    b += sizeof(unsigned long long) * (ld + 2 * (nb + 1)) + sizeof(int) * ld;
    b += sizeof(TableDesc) * max_keyframes + sizeof(float) * max_keyframes + sizeof(int) * 8 + sizeof(unsigned);
    return b;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GMCS_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return GMCS_E_OOM;
    }
    return GMCS_E_CUDA;
}

}  // namespace gmcs

namespace {

#define CK(expr)                                   \
    do {                                           \
        cudaError_t _e = (expr);                   \
        if (_e != cudaSuccess) return cuda_status(_e); \
    } while (0)

template <typename T>
int dalloc(gmcs_ctx* c, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return GMCS_E_OOM;
    }
    c->dev_bytes += count * sizeof(T);
    return GMCS_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaEvent_t take_event(gmcs_ctx* c) {
    if (!c->free_events.empty()) {
        cudaEvent_t e = c->free_events.back();
        c->free_events.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Bracket one launch: count it, and time it with events when profiling.
struct Launch {
    gmcs_ctx* c;
    int kind;
    cudaEvent_t a = nullptr;
    Launch(gmcs_ctx* ctx, int k) : c(ctx), kind(k) {
        nvtxRangePushA(kKindName[k]);   // an NVTX range per launch, for timeline tools
        if (c->profiling) {
            a = take_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~Launch() {
        nvtxRangePop();
        c->launches++;
        c->kind_launches[kind]++;
        if (c->profiling) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, c->stream);
            c->pending.push_back({kind, a, b});
        }
    }
};

int check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GMCS_OK : cuda_status(e);
}

void harvest(gmcs_ctx* c) {
    for (auto& p : c->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            c->kind_ms[p.kind] += ms;
        c->free_events.push_back(p.a);
        c->free_events.push_back(p.b);
    }
    c->pending.clear();
    cudaGetLastError();
}

int upload_scan(gmcs_ctx* c, const float* scan, int N) {
    if (N < 0 || (N > 0 && !scan)) return GMCS_E_INVALID;
    if (N > c->Nmax) return GMCS_E_CAPACITY;
    if (N == 0) return GMCS_OK;
    const float* src = scan;
    if (!is_device_ptr(scan)) {
        CK(cudaMemcpyAsync(c->stage, scan, sizeof(float) * 3 * (size_t)N, cudaMemcpyHostToDevice, c->stream));
        src = c->stage;
    }
    {
        Launch L(c, K_MISC);
        launch_scan_pack(src, N, c->scan, c->stream);
    }
    int rc = check_launch();
    if (rc || c->cfg.model != GMCS_MODEL_GICP) return rc;
    // GICP: per-point covariances of the scan (k nearest points of the scan itself)
    KnnCovArgs ka;
    ka.pts = c->scan;
    ka.n = N;
    ka.k = c->cfg.knn;
    ka.eps = (double)c->cfg.cov_eps;
    ka.cov64 = nullptr;
    ka.nrm32 = c->scov;
    {
        Launch L(c, K_MISC);
        launch_knn_cov(ka, c->stream);
    }
    return check_launch();
}

}  // namespace

// ------------------------------------------------------------------ argument records
namespace gmcs {

void pass_args(gmcs_ctx* c, int N, bool grad, bool move, float* out_ll, float* out_g, float* out_mom, double* logw,
               const float* pose_override, PassArgs* pa_out, FinishArgs* fa_out) {
    int nt, groups, chunk;
    const bool gicp = c->cfg.model == GMCS_MODEL_GICP;
    // the partial-sum scratch holds kMaxGroups x kAccGrad accumulators per particle
    pass_shape(c->P, N, &nt, &groups, &chunk, gicp ? kMaxGroups * kAccGrad / kAccGicp : kMaxGroups);
    PassArgs pa;
    pa.pose = pose_override ? pose_override : c->pose[c->cur];
    pa.kf = c->kf[c->cur];
    pa.nbr = c->nbr;
    pa.tables = c->d_tables;
    pa.scan = c->scan;
    pa.scov = c->scov;
    pa.cov_w = 1.f - c->cfg.cov_eps;
    pa.cov_eps = c->cfg.cov_eps;
    pa.tau = c->cfg.gicp_tau;
    pa.model = c->cfg.model;
    pa.part = c->part;
    pa.ld = c->ld;
    pa.P = c->P;
    pa.N = N;
    pa.k_nb = std::min(c->cfg.k_nb, c->K);
    pa.ntiles = nt;
    pa.groups = groups;
    pa.chunk_len = chunk;
    pa.eps = c->cfg.eps;
    pa.want_ll = (!grad || out_ll) ? 1 : 0;
    pa.sparse = c->cfg.table_layout == GMCS_LAYOUT_COLUMNS ? 1 : 0;
    pa.perm = nullptr;
    FinishArgs fa;
    fa.part = c->part;
    fa.pose = c->pose[c->cur];
    fa.ld = c->ld;
    fa.P = c->P;
    fa.groups = groups;
    fa.do_move = move ? 1 : 0;
    fa.sigma = c->cfg.sigma;
    fa.lambda = c->cfg.lambda;
    fa.theta_max = c->cfg.theta_max;
    fa.t_max = c->cfg.t_max;
    fa.w_min = c->cfg.w_min;
    fa.out_ll = out_ll;
    fa.out_g = out_g;
    fa.out_mom = out_mom;
    fa.logw = logw;
    fa.kf = c->kf[c->cur];
    fa.nbr = c->nbr;
    fa.kf_path = c->d_kf_path;
    fa.path_now = (float)c->path_now;
    fa.K = c->K;
    fa.k_nb = std::min(c->cfg.k_nb, c->K);
    fa.propagate = c->cfg.propagate;
    fa.loop_recent = c->cfg.loop_recent;
    fa.model = c->cfg.model;
    *pa_out = pa;
    *fa_out = fa;
}

SelectArgs select_args(gmcs_ctx* c, int* nbr_out) {
    SelectArgs sa;
    sa.pose = c->pose[c->cur];
    sa.kf = c->kf[c->cur];
    sa.ld = c->ld;
    sa.P = c->P;
    sa.K = c->K;
    sa.k_nb = std::min(c->cfg.k_nb, std::max(c->K, 1));
    sa.nbr = c->nbr;
    sa.nbr_out = nbr_out;
    return sa;
}

PredictArgs predict_args(gmcs_ctx* c, const double dT[12], const double cov[36], const float* z, uint32_t frame) {
    PredictArgs a;
    a.pose = c->pose[c->cur];
    a.ld = c->ld;
    a.P = c->P;
    for (int e = 0; e < 12; ++e) a.dT[e] = (float)dT[e];
    for (int e = 0; e < 36; ++e) a.cov[e] = (float)cov[e];
    a.z = z;
    a.seed = c->cfg.seed;
    a.frame = frame;
    return a;
}

WeighArgs weigh_args(gmcs_ctx* c, const float* ll, WeighResult* res) {
    WeighArgs a;
    a.logw = c->logw;
    a.ll = ll;
    a.P = c->P;
    a.policy = c->cfg.resample;
    a.llm = (c->cfg.resample == GMCS_RESAMPLE_PRUNE && c->cfg.prune_lr > 0.f) ? c->ll : nullptr;
    a.part = c->wpart;
    a.counter = c->counter;
    a.res = res;
    a.pose = c->pose[c->cur];
    a.ld = c->ld;
    return a;
}

void resample_args(gmcs_ctx* c, int P, const double* w, const WeighResult* res, double* w_out, double u,
                   int u_from_philox, uint32_t frame, int* anc, ScanArgs* sa, TotalsArgs* ta, SearchArgs* se) {
    const int nb = (P + kScanBlock - 1) / kScanBlock;
    sa->logw = c->logw;
    sa->w = w;
    sa->res = res;
    sa->w_out = w_out;
    sa->P = P;
    sa->cl = c->cl;
    sa->btot = c->btot;
    ta->btot = c->btot;
    ta->nblocks = nb;
    se->cl = c->cl;
    se->boff = c->btot;
    se->nblocks = nb;
    se->P = P;
    se->u = u;
    se->u_from_philox = u_from_philox;
    se->seed = c->cfg.seed;
    se->frame = frame;
    se->res = res;
    se->anc = anc;
}

PruneArgs prune_args(gmcs_ctx* c, int P, WeighResult* res, const double* w, const float* ll, double u,
                     int u_from_philox, uint32_t frame, bool refill) {
    PruneArgs a;
    a.logw = c->logw;
    a.w = w;
    a.w_out = c->w;
    a.ll = ll;
    a.res = res;
    a.pose = refill ? c->pose[c->cur] : nullptr;
    a.kf = refill ? c->kf[c->cur] : nullptr;
    a.ld = c->ld;
    a.P = P;
    a.K = c->K;
    a.nblocks = (P + kScanBlock - 1) / kScanBlock;
    a.cl = c->cl;
    a.btot = c->btot;
    a.dtot = c->dtot;
    a.anc = c->anc;
    a.prune_w = (double)c->cfg.prune_w;
    a.ll_cut = c->cfg.prune_lr > 0.f ? std::log((double)c->cfg.prune_lr) : -INFINITY;
    a.u = u;
    a.u_from_philox = u_from_philox;
    a.frame = frame;
    a.seed = c->cfg.seed;
    return a;
}

GatherArgs gather_args(gmcs_ctx* c, const WeighResult* res) {
    GatherArgs g;
    g.pose_src = c->pose[c->cur];
    g.pose_dst = c->pose[1 - c->cur];
    g.kf_src = c->kf[c->cur];
    g.kf_dst = c->kf[1 - c->cur];
    g.ld = c->ld;
    g.P = c->P;
    g.K = c->K;
    g.anc = c->anc;
    g.logw = c->logw;
    g.res = res;
    return g;
}

}  // namespace gmcs

namespace {

int run_pass(gmcs_ctx* c, int N, bool grad, bool move, float* out_ll, float* out_g, float* out_mom, double* logw,
             const float* pose_override = nullptr, const int* perm = nullptr) {
    PassArgs pa;
    FinishArgs fa;
    pass_args(c, N, grad, move, out_ll, out_g, out_mom, logw, pose_override, &pa, &fa);
    pa.perm = perm;
    {
        Launch L(c, grad ? K_PASS_GRAD : K_PASS_VALUE);
        if (pa.model == GMCS_MODEL_GICP) launch_gicp_pass(pa, grad, c->stream);
        else launch_pass(pa, c->cfg.table_dtype, grad, c->stream);
    }
    int rc = check_launch();
    if (rc) return rc;
    {
        Launch L(c, K_FINISH);
        launch_finish(fa, grad, c->stream);
    }
    return check_launch();
}

int run_select(gmcs_ctx* c, int* nbr_out_dev) {
    const SelectArgs sa = select_args(c, nbr_out_dev);
    {
        Launch L(c, K_SELECT);
        launch_select(sa, c->stream);
    }
    c->nbr_K = c->K;
    return check_launch();
}

// The passes read the neighbour sets: they must have been selected since the
// context was created or loaded (before, the sets hold zeros or indices of the
// keyframes the context held before a failed load).
bool nbr_ready(const gmcs_ctx* c) { return c->nbr_K > 0 && c->nbr_K <= c->K; }

int check_pass_state(const gmcs_ctx* c) {
    if (!c->have_particles || c->K == 0 || !nbr_ready(c)) return GMCS_E_STATE;
    return GMCS_OK;
}

int run_predict(gmcs_ctx* c, const double dT[12], const double cov[36], const float* z_dev, uint32_t frame) {
    for (int e = 0; e < 12; ++e)
        if (!std::isfinite(dT[e])) return GMCS_E_INVALID;
    for (int e = 0; e < 36; ++e)
        if (!std::isfinite(cov[e])) return GMCS_E_INVALID;
    const PredictArgs a = predict_args(c, dT, cov, z_dev, frame);
    {
        Launch L(c, K_PREDICT);
        launch_predict(a, c->stream);
    }
    return check_launch();
}

int run_weigh(gmcs_ctx* c, const float* ll_dev) {
    const WeighArgs a = weigh_args(c, ll_dev, c->d_res);
    {
        Launch L(c, K_WEIGH);
        launch_weigh(a, weigh_blocks(c->P), c->stream);
    }
    return check_launch();
}

// Quantise, scan, search (ancestors into anc_dev). w_dev: given weights or null.
int run_resample_core(gmcs_ctx* c, int P, const double* w_dev, const WeighResult* res, double* w_out,
                      double u, int u_from_philox, uint32_t frame, int* anc_dev) {
    ScanArgs sa;
    TotalsArgs ta;
    SearchArgs se;
    resample_args(c, P, w_dev, res, w_out, u, u_from_philox, frame, anc_dev, &sa, &ta, &se);
    {
        Launch L(c, K_RESAMPLE);
        launch_resample_scan(sa, c->stream);
    }
    int rc = check_launch();
    if (rc) return rc;
    {
        Launch L(c, K_RESAMPLE);
        launch_scan_totals(ta.btot, ta.nblocks, c->stream);
    }
    rc = check_launch();
    if (rc) return rc;
    {
        Launch L(c, K_RESAMPLE);
        launch_resample_search(se, c->stream);
    }
    return check_launch();
}

// Dead-particle pruning: mark + scans, totals, refill of dead slots, weight split.
int run_prune(gmcs_ctx* c, const PruneArgs& a) {
    {
        Launch L(c, K_RESAMPLE);
        launch_prune_mark(a, c->stream);
    }
    int rc = check_launch();
    if (rc) return rc;
    {
        Launch L(c, K_RESAMPLE);
        launch_prune_totals(a, c->stream);
    }
    if ((rc = check_launch())) return rc;
    {
        Launch L(c, K_GATHER);
        launch_prune_spawn(a, c->stream);
    }
    if ((rc = check_launch())) return rc;
    {
        Launch L(c, K_RESAMPLE);
        launch_prune_reweigh(a, c->stream);
    }
    return check_launch();
}

int run_gather(gmcs_ctx* c, const WeighResult* res) {
    const GatherArgs g = gather_args(c, res);
    {
        Launch L(c, K_GATHER);
        launch_gather(g, c->stream);
    }
    int rc = check_launch();
    if (rc == GMCS_OK) c->cur = 1 - c->cur;
    return rc;
}

}  // namespace

namespace gmcs {

void fill_out(const WeighResult& r, uint32_t frame, gmcs_step_out* o) {
    for (int e = 0; e < 12; ++e) o->estimate[e] = r.est[e];
    o->ess = r.ess;
    o->max_w = r.max_w;
    o->log_norm = r.M + r.logS;
    o->argmax = r.argmax;
    o->resampled = r.do_resample;
    o->frame = frame;
    o->status = r.nonfinite ? GMCS_E_NONFINITE : GMCS_OK;
    o->pruned = r.pruned;
    o->kf_inserted = 0;
    o->overlap = -1.0;
}

}  // namespace gmcs

namespace {

// Copy n bytes from device src to dst (host or device); host destinations synchronise.
int copy_out(gmcs_ctx* c, void* dst, const void* src, size_t n) {
    const bool dev = is_device_ptr(dst);
    CK(cudaMemcpyAsync(dst, src, n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!dev) CK(cudaStreamSynchronize(c->stream));
    return GMCS_OK;
}

}  // namespace

// =============================================================================
extern "C" {

void gmcs_config_default(gmcs_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->sigma = 0.2f;
    cfg->r_t = 1.0f;
    cfg->eps = 1e-3f;
    cfg->lambda = 1e-3f;
    cfg->theta_max = (float)(2.0 * M_PI / 180.0);
    cfg->t_max = 0.1f;
    cfg->w_min = 1e-6f;
    cfg->k_nb = 3;
    cfg->steps = 3;
    cfg->table_dtype = GMCS_TABLE_F32;
    cfg->resample = GMCS_RESAMPLE_ALWAYS;
    cfg->prune_w = 1e-8f;
    cfg->prune_lr = 1e-16f;
    cfg->model = GMCS_MODEL_FIELD;
    cfg->knn = 10;
    cfg->cov_eps = 1e-3f;
    cfg->gicp_tau = 20.f;
    cfg->kf_overlap = 0.f;
    cfg->kf_voxel = 1.f;
    cfg->kf_h = 0.2f;
    cfg->seed = 0;
}

const char* gmcs_strerror(int code) {
    switch (code) {
        case GMCS_OK: return "ok";
        case GMCS_E_INVALID: return "invalid argument";
        case GMCS_E_OOM: return "out of device memory";
        case GMCS_E_CUDA: return "CUDA error";
        case GMCS_E_CAPACITY: return "capacity exceeded";
        case GMCS_E_STATE: return "call out of order";
        case GMCS_E_NONFINITE: return "weights degenerated (reset to uniform)";
        case GMCS_E_BUDGET: return "session does not fit the serving budget";
        case GMCS_E_IO: return "checkpoint file error";
        case GMCS_PENDING: return "pending";
        default: return "unknown error";
    }
}

}  // extern "C"

namespace gmcs {

bool config_valid(const gmcs_config* c) {
    return c && c->sigma > 0.f && c->r_t > 0.f && c->eps > 0.f && c->lambda >= 0.f && c->theta_max > 0.f &&
           (c->propagate == 0 || c->propagate == 1) && c->loop_recent >= 0 &&
           c->t_max > 0.f && c->w_min >= 0.f && c->k_nb >= 1 && c->k_nb <= GMCS_MAX_NB && c->steps >= 0 &&
           c->steps <= 64 && c->table_dtype >= 0 && c->table_dtype <= 2 && c->resample >= 0 && c->resample <= 3 &&
           c->prune_w >= 0.f && c->prune_w < 1.f && c->prune_lr >= 0.f && c->prune_lr < 1.f &&
           (c->model == GMCS_MODEL_FIELD || c->model == GMCS_MODEL_GICP) && c->knn >= 1 && c->knn <= kKnnMax &&
           c->cov_eps > 0.f && c->cov_eps <= 1.f && c->gicp_tau > 0.f && c->kf_overlap >= 0.f &&
           c->kf_overlap <= 1.f && c->kf_voxel > 0.f && c->kf_h > 0.f &&
           (c->table_layout == GMCS_LAYOUT_DENSE ||
            (c->table_layout == GMCS_LAYOUT_COLUMNS && c->model == GMCS_MODEL_FIELD));
}

}  // namespace gmcs

extern "C" {

int gmcs_create(const gmcs_config* cfg, int max_particles, int max_keyframes, int max_points, void* cuda_stream,
                gmcs_ctx** out) {
    if (!out) return GMCS_E_INVALID;
    *out = nullptr;
    if (!config_valid(cfg) || max_particles <= 0 || max_keyframes <= 0 || max_points <= 0) return GMCS_E_INVALID;
    if ((size_t)max_particles * (size_t)(1 + max_keyframes) > ((size_t)1 << 34)) return GMCS_E_INVALID;
    gmcs_ctx* c = new (std::nothrow) gmcs_ctx();
    if (!c) return GMCS_E_OOM;
    c->cfg = *cfg;
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)cuda_stream;
    c->Pmax = max_particles;
    c->Kmax = max_keyframes;
    c->Nmax = max_points;
    c->ld = ((size_t)max_particles + 31) / 32 * 32;
    const size_t ld = c->ld;
    const int nb = (max_particles + kScanBlock - 1) / kScanBlock;
    c->part_floats = std::max((size_t)kMaxGroups * kAccGrad * ld, (size_t)12 * ld);
    c->stage_floats = std::max((size_t)3 * max_points, (size_t)6 * ld);
    int rc = GMCS_OK;
    for (int b = 0; b < 2 && !rc; ++b) {
        rc = dalloc(c, &c->pose[b], (size_t)kPoseC * ld);
        if (!rc) rc = dalloc(c, &c->kf[b], (size_t)kPoseC * ld * max_keyframes);
    }
    if (!rc) rc = dalloc(c, &c->logw, ld);
    if (!rc) rc = dalloc(c, &c->ll, ld);
    if (!rc) rc = dalloc(c, &c->w, ld);
    if (!rc) rc = dalloc(c, &c->gbuf, (size_t)6 * ld);
    if (!rc) rc = dalloc(c, &c->nbr, (size_t)GMCS_MAX_NB * ld);
    if (!rc) rc = dalloc(c, &c->part, c->part_floats);
    if (!rc) rc = dalloc(c, &c->scan, (size_t)max_points);
    if (!rc) rc = dalloc(c, &c->scov, (size_t)max_points);
    if (!rc) rc = dalloc(c, &c->stage, c->stage_floats);
    if (!rc) rc = dalloc(c, &c->wpart, (size_t)kWeighPart * kWeighMaxBlocks);
    if (!rc) rc = dalloc(c, &c->counter, 1);
    if (!rc) rc = dalloc(c, &c->d_res, 1);
    if (!rc) rc = dalloc(c, &c->cl, ld);
    if (!rc) rc = dalloc(c, &c->btot, (size_t)nb + 1);
    if (!rc) rc = dalloc(c, &c->dtot, (size_t)nb + 1);
    if (!rc) rc = dalloc(c, &c->anc, ld);
    if (!rc) rc = dalloc(c, &c->d_tables, (size_t)max_keyframes);
    if (!rc) rc = dalloc(c, &c->d_kf_path, (size_t)max_keyframes);
    if (!rc) rc = dalloc(c, &c->d_mm, 8);
    if (!rc) rc = dalloc(c, &c->d_ovl, 1);
    if (!rc && cudaMallocHost((void**)&c->h_ovl, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        c->h_ovl = nullptr;
        rc = GMCS_E_OOM;
    }
    if (!rc && cudaMallocHost((void**)&c->h_res, sizeof(WeighResult)) != cudaSuccess) {
        cudaGetLastError();
        c->h_res = nullptr;
        rc = GMCS_E_OOM;
    }
    if (!rc && cudaMemsetAsync(c->counter, 0, sizeof(unsigned), c->stream) != cudaSuccess) rc = GMCS_E_CUDA;
    // neighbour sets start as table 0 (never a negative index; see nbr_ready)
    if (!rc && cudaMemsetAsync(c->nbr, 0, sizeof(int) * GMCS_MAX_NB * ld, c->stream) != cudaSuccess) rc = GMCS_E_CUDA;
    if (!rc && cudaMemsetAsync(c->d_tables, 0, sizeof(TableDesc) * (size_t)max_keyframes, c->stream) != cudaSuccess)
        rc = GMCS_E_CUDA;
    if (!rc && cudaMemsetAsync(c->d_res, 0, sizeof(WeighResult), c->stream) != cudaSuccess) rc = GMCS_E_CUDA;
    if (rc) {
        gmcs_destroy(c);
        return rc;
    }
    *out = c;
    return GMCS_OK;
}

int gmcs_destroy(gmcs_ctx* c) {
    if (!c) return GMCS_OK;
    cudaStreamSynchronize(c->stream);
    harvest(c);
    for (auto e : c->free_events) cudaEventDestroy(e);
    for (auto& t : c->tables) {
        cudaFree(t.cells);
        cudaFree(t.occ);
    }
    void* ptrs[] = {c->pose[0], c->pose[1], c->kf[0], c->kf[1], c->logw, c->w, c->gbuf, c->ll, c->nbr, c->part, c->scan,
                    c->stage, c->wpart, c->counter, c->d_res, c->cl, c->btot, c->dtot, c->anc, c->d_tables, c->d2, c->scov, c->d_mm, c->d_ovl,
                    c->d_kf_path, c->perm, c->order_scratch};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_res) cudaFreeHost(c->h_res);
    if (c->h_ovl) cudaFreeHost(c->h_ovl);
    cudaGetLastError();
    delete c;
    return GMCS_OK;
}

int gmcs_init_particles(gmcs_ctx* c, const float* poses, int P, const double* logw) {
    if (!c || !poses || P <= 0) return GMCS_E_INVALID;
    if (P > c->Pmax) return GMCS_E_CAPACITY;
    // stage the P x 12 block in the scratch buffer, then transpose to SoA
    CK(cudaMemcpyAsync(c->part, poses, sizeof(float) * 12 * (size_t)P, cudaMemcpyDefault, c->stream));
    {
        Launch L(c, K_MISC);
        launch_aos_to_soa(c->part, P, 12, c->pose[c->cur], c->ld, c->stream);
    }
    int rc = check_launch();
    if (rc) return rc;
    if (logw) {
        CK(cudaMemcpyAsync(c->logw, logw, sizeof(double) * P, cudaMemcpyDefault, c->stream));
    } else {
        std::vector<double> u(P, -std::log((double)P));
        CK(cudaMemcpyAsync(c->logw, u.data(), sizeof(double) * P, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    c->P = P;
    c->frame = 0;
    c->version++;
    c->have_particles = true;
    c->last_valid = false;
    return GMCS_OK;
}

namespace {

// GICP keyframe: per-point covariances (k nearest keyframe points, FP64), then
// per-voxel means of points and covariances into a dense record lattice.
int build_gicp_map(gmcs_ctx* c, const float* dpts, int n, const gmcs_grid* grid, HostTable* t) {
    const size_t nv = (size_t)grid->n[0] * grid->n[1] * grid->n[2];
    t->bytes = nv * 3 * sizeof(float4);
    if (cudaMalloc(&t->cells, t->bytes) != cudaSuccess) {
        cudaGetLastError();
        t->cells = nullptr;
        return GMCS_E_OOM;
    }
    float4* p4 = nullptr;
    double* cov = nullptr;
    double* sums = nullptr;
    int rc = GMCS_OK;
    if (cudaMalloc((void**)&p4, sizeof(float4) * (size_t)std::max(n, 1)) != cudaSuccess ||
        cudaMalloc((void**)&cov, sizeof(double) * 6 * (size_t)std::max(n, 1)) != cudaSuccess ||
        cudaMalloc((void**)&sums, sizeof(double) * 10 * nv) != cudaSuccess) {
        cudaGetLastError();
        rc = GMCS_E_OOM;
    }
    if (!rc) rc = cuda_status(cudaMemsetAsync(sums, 0, sizeof(double) * 10 * nv, c->stream));
    if (!rc && n > 0) {
        {
            Launch L(c, K_TABLE);
            launch_scan_pack(dpts, n, p4, c->stream);
        }
        KnnCovArgs ka;
        ka.pts = p4;
        ka.n = n;
        ka.k = c->cfg.knn;
        ka.eps = (double)c->cfg.cov_eps;
        ka.cov64 = cov;
        ka.nrm32 = nullptr;
        {
            Launch L(c, K_TABLE);
            launch_knn_cov(ka, c->stream);
        }
        rc = check_launch();
    }
    VoxelArgs va;
    va.pts = p4;
    va.cov = cov;
    va.n = n;
    va.ox = grid->origin[0];
    va.oy = grid->origin[1];
    va.oz = grid->origin[2];
    va.h = grid->h;
    va.nx = grid->n[0];
    va.ny = grid->n[1];
    va.nz = grid->n[2];
    va.sums = sums;
    va.rec = reinterpret_cast<float4*>(t->cells);
    if (!rc) {
        {
            Launch L(c, K_TABLE);
            launch_voxel_accum(va, c->stream);
        }
        rc = check_launch();
    }
    if (!rc) {
        {
            Launch L(c, K_TABLE);
            launch_voxel_final(va, c->stream);
        }
        rc = check_launch();
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(p4);
    cudaFree(cov);
    cudaFree(sums);
    if (rc) {
        cudaFree(t->cells);
        t->cells = nullptr;
    }
    return rc;
}

// Bounding box of n device points (n x 3 floats), synchronising.
int device_bbox(gmcs_ctx* c, const float* dpts, int n, float4* p4, float mn[3], float mx[3]) {
    {
        Launch L(c, K_TABLE);
        launch_scan_pack(dpts, n, p4, c->stream);
    }
    BBoxArgs ba{p4, n, c->d_mm};
    {
        Launch L(c, K_TABLE);
        launch_bbox(ba, c->stream);
    }
    int rc = check_launch();
    if (rc) return rc;
    int mm[6];
    CK(cudaMemcpyAsync(mm, c->d_mm, sizeof(mm), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int d = 0; d < 6; ++d) {
        const int i = mm[d] >= 0 ? mm[d] : mm[d] ^ 0x7fffffff;   // back from the order-preserving image
        float f;
        std::memcpy(&f, &i, sizeof(f));
        (d < 3 ? mn[d] : mx[d - 3]) = f;
    }
    return GMCS_OK;
}

// Occupancy lattice of a keyframe (voxel edge kf_voxel; per axis lo = floor(min/h) - 1,
// hi = floor(max/h) + 1, origin lo h, hi - lo + 1 voxels), for the overlap rate.
int build_occupancy(gmcs_ctx* c, const float* dpts, int n, HostTable& t) {
    const double h = (double)c->cfg.kf_voxel;
    float4* p4 = nullptr;
    if (cudaMalloc((void**)&p4, sizeof(float4) * (size_t)std::max(n, 1)) != cudaSuccess) {
        cudaGetLastError();
        return GMCS_E_OOM;
    }
    float mn[3] = {0.f, 0.f, 0.f}, mx[3] = {0.f, 0.f, 0.f};
    int rc = n > 0 ? device_bbox(c, dpts, n, p4, mn, mx) : GMCS_OK;
    size_t nv = 1;
    for (int a = 0; a < 3 && !rc; ++a) {
        const double lo = std::floor((double)mn[a] / h) - 1.0, hi = std::floor((double)mx[a] / h) + 1.0;
        t.occ_grid.origin[a] = lo * h;
        t.occ_grid.n[a] = (int)(hi - lo) + 1;
        nv *= (size_t)t.occ_grid.n[a];
    }
    t.occ_grid.h = h;
    if (!rc && nv >= ((size_t)1 << 32)) rc = GMCS_E_INVALID;
    if (!rc && cudaMalloc((void**)&t.occ, nv) != cudaSuccess) {
        cudaGetLastError();
        t.occ = nullptr;
        rc = GMCS_E_OOM;
    }
    if (!rc) rc = cuda_status(cudaMemsetAsync(t.occ, 0, nv, c->stream));
    if (!rc && n > 0) {
        OccArgs oa{p4, n, t.occ_grid.origin[0], t.occ_grid.origin[1], t.occ_grid.origin[2], h,
                   t.occ_grid.n[0], t.occ_grid.n[1], t.occ_grid.n[2], t.occ};
        {
            Launch L(c, K_TABLE);
            launch_occ_fill(oa, c->stream);
        }
        rc = check_launch();
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(p4);
    if (rc && t.occ) {
        cudaFree(t.occ);
        t.occ = nullptr;
    }
    t.occ_bytes = rc ? 0 : nv;
    return rc;
}

// Table descriptor, occupancy lattice, per-particle keyframe poses and path
// length of a new keyframe whose table t is built; frees t on failure. The
// odometry since the last keyframe restarts (the keyframe is the current frame).
int register_keyframe(gmcs_ctx* c, HostTable& t, const gmcs_grid* grid, int ncx, int ncy, int ncz,
                      const float* kf_poses, int* kf_id, const float* dpts, int n) {
    int rc = build_occupancy(c, dpts, n, t);
    if (rc) {
        cudaFree(t.cells);
        return rc;
    }
    TableDesc td;
    std::memset(&td, 0, sizeof(td));
    td.cells = table_records(t);
    td.dir = table_dir(t);
    td.ox = (float)grid->origin[0];
    td.oy = (float)grid->origin[1];
    td.oz = (float)grid->origin[2];
    td.inv_h = (float)(1.0 / grid->h);
    td.h = (float)grid->h;
    td.ncx = ncx;
    td.ncy = ncy;
    td.ncz = ncz;
    td.dtype = t.dtype;
    const int k = c->K;
    rc = cuda_status(cudaMemcpyAsync(c->d_tables + k, &td, sizeof(td), cudaMemcpyHostToDevice, c->stream));
    if (!rc) {
        float* dst = c->kf[c->cur] + (size_t)k * kPoseC * c->ld;
        if (kf_poses) {
            rc = cuda_status(cudaMemcpyAsync(c->part, kf_poses, sizeof(float) * 12 * (size_t)c->P, cudaMemcpyDefault,
                                             c->stream));
            if (!rc) {
                Launch L(c, K_MISC);
                launch_aos_to_soa(c->part, c->P, 12, dst, c->ld, c->stream);
            }
        } else {
            rc = cuda_status(cudaMemcpy2DAsync(dst, c->ld * sizeof(float), c->pose[c->cur], c->ld * sizeof(float),
                                               c->P * sizeof(float), kPoseC, cudaMemcpyDeviceToDevice, c->stream));
        }
        if (!rc) rc = check_launch();
    }
    if (!rc) rc = cuda_status(cudaStreamSynchronize(c->stream));   // td lives on this stack frame
    if (rc) {
        cudaFree(t.cells);
        cudaFree(t.occ);
        return rc;
    }
    {
        const float d = (float)c->path_now;
        if (cudaMemcpy(c->d_kf_path + k, &d, sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(t.cells);
            cudaFree(t.occ);
            return GMCS_E_CUDA;
        }
    }
    c->kf_path.push_back(c->path_now);
    c->dev_bytes += t.bytes + t.occ_bytes;
    c->tables.push_back(t);
    c->K = k + 1;
    c->version++;
    for (int e = 0; e < 12; ++e) c->odo[e] = (e % 5 == 0) ? 1.0 : 0.0;   // identity
    if (kf_id) *kf_id = k;
    return GMCS_OK;
}

// Stage host points on the device (device points are used in place).
int stage_points(gmcs_ctx* c, const float* pts, int n, const float** dpts, float** tmp) {
    *dpts = pts;
    *tmp = nullptr;
    if (n > 0 && !is_device_ptr(pts)) {
        if (cudaMalloc((void**)tmp, sizeof(float) * 3 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            *tmp = nullptr;
            return GMCS_E_OOM;
        }
        if (cudaMemcpyAsync(*tmp, pts, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess) {
            cudaFree(*tmp);
            *tmp = nullptr;
            return GMCS_E_CUDA;
        }
        *dpts = *tmp;
    }
    return GMCS_OK;
}

int add_keyframe_gicp(gmcs_ctx* c, const float* pts, int n, const gmcs_grid* grid, const float* kf_poses, int* kf_id) {
    for (int a = 0; a < 3; ++a)
        if (grid->n[a] < 1 || !std::isfinite(grid->origin[a])) return GMCS_E_INVALID;
    if (!(grid->h > 0.0) || !std::isfinite(grid->h)) return GMCS_E_INVALID;
    const size_t nv = (size_t)grid->n[0] * grid->n[1] * grid->n[2];
    if (nv >= ((size_t)1 << 31)) return GMCS_E_INVALID;
    const float* dpts = nullptr;
    float* tmp = nullptr;
    int rc = stage_points(c, pts, n, &dpts, &tmp);
    if (rc) return rc;
    HostTable t;
    t.grid = *grid;
    t.dtype = 3;
    rc = build_gicp_map(c, dpts, n, grid, &t);
    if (!rc) rc = register_keyframe(c, t, grid, grid->n[0], grid->n[1], grid->n[2], kf_poses, kf_id, dpts, n);
    if (tmp) {
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
    }
    return rc;
}

}  // namespace

namespace {

// Column-sparse layout of a table whose squared distances are in c->d2: the
// per-column runs (device), read back to build the directory of first-record
// offsets on the host; allocates the table (directory, then the records) into t.
int build_columns(gmcs_ctx* c, HostTable& t, int nx, int ny, int nz, float inv_two_sigma2, float r_t2, size_t rec) {
    const size_t ncol = (size_t)col_tiles(nx - 1) * col_tiles(ny - 1);   // tiles of columns
    uint32_t* d_run = nullptr;
    if (cudaMalloc((void**)&d_run, ncol * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return GMCS_E_OOM;
    }
    {
        Launch L(c, K_TABLE);
        launch_col_range(c->d2, nx, ny, nz, inv_two_sigma2, r_t2, d_run, c->stream);
    }
    int rc = check_launch();
    std::vector<uint32_t> run;
    std::vector<uint2> dir;
    try {
        run.resize(ncol);
        dir.resize(ncol);
    } catch (...) {
        rc = GMCS_E_OOM;
    }
    if (!rc) rc = cuda_status(cudaMemcpyAsync(run.data(), d_run, ncol * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                              c->stream));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(c->stream));
    cudaFree(d_run);
    if (rc) return rc;
    uint64_t total = 0;
    for (size_t k = 0; k < ncol; ++k) {
        dir[k] = make_uint2((uint32_t)total, run[k]);
        total += (uint64_t)(run[k] >> 16) * kColTile * kColTile;
    }
    if (total >= ((uint64_t)1 << 31)) return GMCS_E_INVALID;
    t.dir_bytes = (ncol * sizeof(uint2) + 255) / 256 * 256;   // records start 256-byte aligned
    t.bytes = t.dir_bytes + (size_t)std::max<uint64_t>(total, 1) * rec;
    if (cudaMalloc(&t.cells, t.bytes) != cudaSuccess) {
        cudaGetLastError();
        t.cells = nullptr;
        return GMCS_E_OOM;
    }
    rc = cuda_status(cudaMemcpyAsync(t.cells, dir.data(), ncol * sizeof(uint2), cudaMemcpyHostToDevice, c->stream));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(c->stream));   // dir lives on this stack frame
    if (rc) {
        cudaFree(t.cells);
        t.cells = nullptr;
    }
    return rc;
}

}  // namespace

int gmcs_add_keyframe(gmcs_ctx* c, const float* pts, int n, const gmcs_grid* grid, const float* kf_poses, int* kf_id) {
    if (!c || !grid || n < 0 || (n > 0 && !pts)) return GMCS_E_INVALID;
    if (!c->have_particles) return GMCS_E_STATE;
    if (c->K >= c->Kmax) return GMCS_E_CAPACITY;
    if (c->cfg.model == GMCS_MODEL_GICP) return add_keyframe_gicp(c, pts, n, grid, kf_poses, kf_id);
    for (int a = 0; a < 3; ++a)   // the lookup's floor is exact below 2^22 cells per axis
        if (grid->n[a] < 2 || grid->n[a] > (1 << 22) || !std::isfinite(grid->origin[a])) return GMCS_E_INVALID;
    if (!(grid->h > 0.0) || !std::isfinite(grid->h)) return GMCS_E_INVALID;
    const bool cols = c->cfg.table_layout == GMCS_LAYOUT_COLUMNS;
    if (cols && grid->n[2] > 65536) return GMCS_E_INVALID;   // a column run is 16-bit
    const size_t nx = grid->n[0], ny = grid->n[1], nz = grid->n[2];
    const size_t nv = nx * ny * nz;
    const size_t ncell = (nx - 1) * (ny - 1) * (nz - 1);
    if (ncell >= ((size_t)1 << 31)) return GMCS_E_INVALID;
    const int dtype = c->cfg.table_dtype;
    const size_t rec = dtype == 0 ? 32 : 16;
    HostTable t;
    t.grid = *grid;
    t.dtype = dtype;
    t.layout = cols ? GMCS_LAYOUT_COLUMNS : GMCS_LAYOUT_DENSE;
    // squared-distance scratch, grown to the largest table seen
    if (c->d2_cap < nv) {
        if (c->d2) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->d2);
            c->dev_bytes -= c->d2_cap * sizeof(unsigned);
            c->d2 = nullptr;
            c->d2_cap = 0;
        }
        if (cudaMalloc((void**)&c->d2, nv * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            return GMCS_E_OOM;
        }
        c->d2_cap = nv;
        c->dev_bytes += nv * sizeof(unsigned);
    }
    // points: device pointer used in place, host points staged
    const float* dpts = pts;
    float* tmp = nullptr;
    if (n > 0 && !is_device_ptr(pts)) {
        if (cudaMalloc((void**)&tmp, sizeof(float) * 3 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return GMCS_E_OOM;
        }
        if (cudaMemcpyAsync(tmp, pts, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            cudaFree(tmp);
            return GMCS_E_CUDA;
        }
        dpts = tmp;
    }
    auto release_tmp = [&]() {
        if (tmp) {
            cudaStreamSynchronize(c->stream);
            cudaFree(tmp);
            tmp = nullptr;
        }
    };
    {
        Launch L(c, K_TABLE);
        launch_fill_u32(c->d2, nv, 0x7f800000u, c->stream);
    }
    SplatArgs sa;
    sa.pts = dpts;
    sa.n = n;
    for (int a = 0; a < 3; ++a) {
        sa.o_hi[a] = (float)grid->origin[a];
        sa.o_lo[a] = (float)(grid->origin[a] - (double)sa.o_hi[a]);
    }
    sa.h_hi = (float)grid->h;
    sa.h_lo = (float)(grid->h - (double)sa.h_hi);
    sa.nx = (int)nx;
    sa.ny = (int)ny;
    sa.nz = (int)nz;
    sa.r_t = c->cfg.r_t;
    sa.d2 = c->d2;
    {
        Launch L(c, K_TABLE);
        launch_splat(sa, c->stream);
    }
    int rc = check_launch();
    const float inv_two_sigma2 = 1.0f / (2.0f * c->cfg.sigma * c->cfg.sigma);
    const float r_t2 = c->cfg.r_t * c->cfg.r_t;
    if (!rc) {
        if (cols) {
            rc = build_columns(c, t, (int)nx, (int)ny, (int)nz, inv_two_sigma2, r_t2, rec);
        } else {
            t.bytes = ncell * rec;
            if (cudaMalloc(&t.cells, t.bytes) != cudaSuccess) {
                cudaGetLastError();
                t.cells = nullptr;
                rc = GMCS_E_OOM;
            }
        }
    }
    if (rc) {
        release_tmp();
        return rc;
    }
    PackArgs pa;
    pa.d2 = c->d2;
    pa.nx = (int)nx;
    pa.ny = (int)ny;
    pa.nz = (int)nz;
    pa.inv_two_sigma2 = inv_two_sigma2;
    pa.r_t2 = r_t2;
    pa.cells = table_records(t);
    pa.dtype = dtype;
    pa.dir = table_dir(t);
    {
        Launch L(c, K_TABLE);
        launch_pack(pa, c->stream);
    }
    rc = check_launch();
    if (rc) {
        release_tmp();
        cudaFree(t.cells);
        return rc;
    }
    rc = register_keyframe(c, t, grid, (int)nx - 1, (int)ny - 1, (int)nz - 1, kf_poses, kf_id, dpts, n);
    release_tmp();
    return rc;
}

namespace {

// Enqueue the overlap count of the packed scan (c->scan) against the last keyframe.
int enqueue_overlap(gmcs_ctx* c, int N, const double T[12]) {
    const HostTable& t = c->tables[c->K - 1];
    OverlapArgs oa;
    oa.scan = c->scan;
    oa.n = N;
    for (int e = 0; e < 12; ++e) oa.T[e] = T[e];
    oa.occ = t.occ;
    oa.ox = t.occ_grid.origin[0];
    oa.oy = t.occ_grid.origin[1];
    oa.oz = t.occ_grid.origin[2];
    oa.h = t.occ_grid.h;
    oa.nx = t.occ_grid.n[0];
    oa.ny = t.occ_grid.n[1];
    oa.nz = t.occ_grid.n[2];
    oa.count = c->d_ovl;
    CK(cudaMemsetAsync(c->d_ovl, 0, sizeof(unsigned), c->stream));
    {
        Launch L(c, K_MISC);
        launch_overlap(oa, c->stream);
    }
    int rc = check_launch();
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->h_ovl, c->d_ovl, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    return GMCS_OK;
}

void pose_mul_d(const double* A, const double* B, double* C) {
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 4; ++k) {
            double v = A[r * 4] * B[k] + A[r * 4 + 1] * B[4 + k] + A[r * 4 + 2] * B[8 + k];
            if (k == 3) v += A[r * 4 + 3];
            C[r * 4 + k] = v;
        }
}

// Insert the frame's scan as a keyframe: every particle's current pose, a
// lattice (field: step kf_h, margin r_t; GICP: voxels of edge kf_h, margin one
// voxel) over the scan's bounding box.
int insert_scan_keyframe(gmcs_ctx* c, const float* scan, int N) {
    const float* dpts = nullptr;
    float* tmp = nullptr;
    int rc = stage_points(c, scan, N, &dpts, &tmp);
    float4* p4 = nullptr;
    if (!rc && cudaMalloc((void**)&p4, sizeof(float4) * (size_t)N) != cudaSuccess) {
        cudaGetLastError();
        rc = GMCS_E_OOM;
    }
    float mn[3], mx[3];
    if (!rc) rc = device_bbox(c, dpts, N, p4, mn, mx);
    cudaFree(p4);
    if (!rc) {
        const bool gicp = c->cfg.model == GMCS_MODEL_GICP;
        const double h = (double)c->cfg.kf_h, margin = gicp ? h : (double)c->cfg.r_t;
        gmcs_grid g;
        for (int a = 0; a < 3; ++a) {
            const double i0 = std::floor(((double)mn[a] - margin) / h), i1 = std::ceil(((double)mx[a] + margin) / h);
            g.origin[a] = i0 * h;
            g.n[a] = (int)(i1 - i0) + 1;
        }
        g.h = h;
        int kid = 0;
        rc = gmcs_add_keyframe(c, dpts, N, &g, nullptr, &kid);
    }
    if (tmp) {
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
    }
    return rc;
}

}  // namespace

static int locality_order(gmcs_ctx* c, const int** perm);

// The frame's lookup passes with the particles in the locality order (1), or in
// their own order (0): after resampling, copies of one parent sit side by side
// and a warp reads fewer distinct cells than the pose-space order gives it (FP32
// gradient / value pass 1.534 / 1.015 -> 1.565 / 1.048 ms ordered; GICP value
// pass 2.37 -> 2.44 ms).
#ifndef GMCS_STEP_ORDER
#define GMCS_STEP_ORDER 0
#endif

int gmcs_step(gmcs_ctx* c, const float* scan, int N, const double delta_T[12], const double cov[36],
              const double* u_override, gmcs_step_out* out) {
    if (!c || !delta_T || !cov) return GMCS_E_INVALID;
    if (!c->have_particles || c->K == 0) return GMCS_E_STATE;
    if (u_override && !(*u_override >= 0.0 && *u_override < 1.0)) return GMCS_E_INVALID;
    int rc = upload_scan(c, scan, N);
    if (rc) return rc;
    c->version++;
    const uint32_t frame = c->frame;
    // odometry path length of this frame (Eq. 9 along the odometry trajectory)
    c->path_now += std::sqrt(delta_T[3] * delta_T[3] + delta_T[7] * delta_T[7] + delta_T[11] * delta_T[11]);
    // odometry pose of this frame in the last keyframe's frame, and its overlap rate (Sec. III-E)
    {
        double o[12];
        pose_mul_d(c->odo, delta_T, o);
        std::memcpy(c->odo, o, sizeof(o));
    }
    c->ovl_valid = c->cfg.kf_overlap > 0.f && c->K > 0 && N > 0;
    if (c->ovl_valid && (rc = enqueue_overlap(c, N, c->odo))) return rc;
    if ((rc = run_predict(c, delta_T, cov, nullptr, frame))) return rc;
    if ((rc = run_select(c, nullptr))) return rc;
    const int* perm = nullptr;
    if (GMCS_STEP_ORDER && (rc = locality_order(c, &perm))) return rc;
    for (int s = 0; s < c->cfg.steps; ++s)
        if ((rc = run_pass(c, N, true, true, nullptr, nullptr, nullptr, nullptr, nullptr, perm))) return rc;
    if ((rc = run_pass(c, N, false, false, c->ll, nullptr, nullptr, c->logw, nullptr, perm))) return rc;
    if ((rc = run_weigh(c, nullptr))) return rc;
    if (c->cfg.resample == GMCS_RESAMPLE_NEVER) {
        {
            Launch L(c, K_WEIGH);
            launch_normalize(c->logw, c->P, c->d_res, c->w, c->anc, c->stream);
        }
        if ((rc = check_launch())) return rc;
    } else if (c->cfg.resample == GMCS_RESAMPLE_PRUNE) {
        const double u = u_override ? *u_override : 0.0;
        const PruneArgs pa = prune_args(c, c->P, c->d_res, nullptr, c->ll, u, u_override ? 0 : 1, frame, true);
        if ((rc = run_prune(c, pa))) return rc;
    } else {
        const double u = u_override ? *u_override : 0.0;
        if ((rc = run_resample_core(c, c->P, nullptr, c->d_res, c->w, u, u_override ? 0 : 1, frame, c->anc)))
            return rc;
        if ((rc = run_gather(c, c->d_res))) return rc;
    }
    CK(cudaMemcpyAsync(c->h_res, c->d_res, sizeof(WeighResult), cudaMemcpyDeviceToHost, c->stream));
    c->frame = frame + 1;
    c->frames++;
    c->version++;
    c->last_valid = true;
    c->last_N = N;
    c->last_inserted = 0;
    if (out) {
        CK(cudaStreamSynchronize(c->stream));
        fill_out(*c->h_res, frame, out);
        if (c->ovl_valid) {
            out->overlap = (double)*c->h_ovl / (double)N;
            if (out->overlap < (double)c->cfg.kf_overlap && c->K < c->Kmax) {
                if ((rc = insert_scan_keyframe(c, scan, N))) return rc;
                out->kf_inserted = 1;
                c->last_inserted = 1;
            }
        }
        c->last = *out;
    }
    return GMCS_OK;
}

int gmcs_set_path(gmcs_ctx* c, double now, const double* kf_path) {
    if (!c || !std::isfinite(now)) return GMCS_E_INVALID;
    if (kf_path) {
        std::vector<float> f(c->K);
        for (int k = 0; k < c->K; ++k) {
            if (!std::isfinite(kf_path[k])) return GMCS_E_INVALID;
            f[k] = (float)kf_path[k];
        }
        if (c->K > 0) {
            CK(cudaMemcpyAsync(c->d_kf_path, f.data(), sizeof(float) * c->K, cudaMemcpyHostToDevice, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        c->kf_path.assign(kf_path, kf_path + c->K);
    }
    c->path_now = now;
    return GMCS_OK;
}

int gmcs_last_result(gmcs_ctx* c, gmcs_step_out* out) {
    if (!c || !out) return GMCS_E_INVALID;
    if (!c->last_valid) return GMCS_E_STATE;
    CK(cudaStreamSynchronize(c->stream));
    fill_out(*c->h_res, c->frame - 1, out);
    if (c->ovl_valid && c->last_N > 0) out->overlap = (double)*c->h_ovl / (double)c->last_N;
    out->kf_inserted = c->last_inserted;
    return GMCS_OK;
}

int gmcs_predict(gmcs_ctx* c, const double delta_T[12], const double cov[36], const float* z, uint32_t frame) {
    if (!c || !delta_T || !cov) return GMCS_E_INVALID;
    if (!c->have_particles) return GMCS_E_STATE;
    const float* zd = z;
    if (z && !is_device_ptr(z)) {
        CK(cudaMemcpyAsync(c->stage, z, sizeof(float) * 6 * (size_t)c->P, cudaMemcpyHostToDevice, c->stream));
        zd = c->stage;
    }
    c->version++;
    return run_predict(c, delta_T, cov, zd, frame);
}

int gmcs_select(gmcs_ctx* c, int* nbr_out) {
    if (!c) return GMCS_E_INVALID;
    if (!c->have_particles) return GMCS_E_STATE;
    const int knb = std::min(c->cfg.k_nb, std::max(c->K, 1));
    const bool dev = nbr_out && is_device_ptr(nbr_out);
    int* tmp = nullptr;
    if (nbr_out && !dev) tmp = reinterpret_cast<int*>(c->part);   // P x k_nb ints fit in the scratch
    c->version++;
    int rc = run_select(c, dev ? nbr_out : tmp);
    if (rc) return rc;
    if (tmp) return copy_out(c, nbr_out, tmp, sizeof(int) * (size_t)c->P * knb);
    return GMCS_OK;
}

int gmcs_eval(gmcs_ctx* c, const float* scan, int N, float* ll, float* g, float* mom) {
    if (!c) return GMCS_E_INVALID;
    int rc = check_pass_state(c);
    if (rc) return rc;
    rc = upload_scan(c, scan, N);
    if (rc) return rc;
    // outputs go to device staging (ll: c->ll; g and mom: the stage buffer) unless device pointers were given
    const bool gd = g && is_device_ptr(g), md = mom && is_device_ptr(mom), ld_ = ll && is_device_ptr(ll);
    float* dg = g ? (gd ? g : nullptr) : nullptr;
    float* dm = mom ? (md ? mom : nullptr) : nullptr;
    float* tmp = nullptr;
    if ((g && !gd) || (mom && !md)) {
        if (cudaMalloc((void**)&tmp, sizeof(float) * 28 * (size_t)c->P) != cudaSuccess) {
            cudaGetLastError();
            return GMCS_E_OOM;
        }
        if (g && !gd) dg = tmp;
        if (mom && !md) dm = tmp + 6 * (size_t)c->P;
    }
    float* dl = ll ? (ld_ ? ll : c->ll) : nullptr;
    const bool grad = (g != nullptr) || (mom != nullptr);
    rc = run_pass(c, N, grad, false, dl, dg, dm, nullptr);
    if (!rc && ll && !ld_) rc = copy_out(c, ll, c->ll, sizeof(float) * c->P);
    if (!rc && g && !gd) rc = copy_out(c, g, dg, sizeof(float) * 6 * (size_t)c->P);
    const size_t nm = c->cfg.model == GMCS_MODEL_GICP ? 22 : 10;
    if (!rc && mom && !md) rc = copy_out(c, mom, dm, sizeof(float) * nm * (size_t)c->P);
    if (tmp) {
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
    }
    return rc;
}

// Poses T0 exp(xi) into the alternate pose buffer (xi staged when on the host).
// The particles in a locality order (k_order.cu) for the passes of the
// differentiable log-likelihood, whose poses need not be clustered; computed
// from the current poses once per state version.
static int locality_order(gmcs_ctx* c, const int** perm) {
    *perm = nullptr;
    if (!c->perm) {
        if (cudaMalloc((void**)&c->perm, sizeof(int) * c->ld) != cudaSuccess ||
            cudaMalloc((void**)&c->order_scratch, sizeof(uint32_t) * order_scratch_words((int)c->ld)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->perm);
            c->perm = nullptr;
            return GMCS_E_OOM;
        }
        c->dev_bytes += sizeof(int) * c->ld + sizeof(uint32_t) * order_scratch_words((int)c->ld);
    }
    if (c->perm_version != c->version) {
        {
            Launch L(c, K_MISC);
            launch_locality_order(c->pose[c->cur], c->ld, c->P, c->order_scratch, c->perm, c->stream);
        }
        const int rc = check_launch();
        if (rc) return rc;
        c->perm_version = c->version;
    }
    *perm = c->perm;
    return GMCS_OK;
}

static int perturbed_poses(gmcs_ctx* c, const float* xi, const float** pose_out) {
    const float* dxi = xi;
    if (!is_device_ptr(xi)) {
        CK(cudaMemcpyAsync(c->stage, xi, sizeof(float) * 6 * (size_t)c->P, cudaMemcpyHostToDevice, c->stream));
        dxi = c->stage;
    }
    float* dst = c->pose[1 - c->cur];
    {
        Launch L(c, K_MISC);
        launch_perturb(c->pose[c->cur], dxi, c->P, c->ld, dst, c->stream);
    }
    *pose_out = dst;
    return check_launch();
}

int gmcs_loglik(gmcs_ctx* c, const float* xi, const float* scan, int N, float* ll) {
    if (!c || !xi || !ll) return GMCS_E_INVALID;
    int rc = check_pass_state(c);
    if (rc) return rc;
    rc = upload_scan(c, scan, N);
    if (rc) return rc;
    const float* T = nullptr;
    const int* perm = nullptr;
    if ((rc = perturbed_poses(c, xi, &T))) return rc;
    if ((rc = locality_order(c, &perm))) return rc;
    const bool dev = is_device_ptr(ll);
    if ((rc = run_pass(c, N, false, false, dev ? ll : c->ll, nullptr, nullptr, nullptr, T, perm))) return rc;
    if (!dev) return copy_out(c, ll, c->ll, sizeof(float) * c->P);
    return GMCS_OK;
}

int gmcs_loglik_backward(gmcs_ctx* c, const float* xi, const float* scan, int N, const float* grad_ll, float* grad_xi) {
    if (!c || !xi || !grad_ll || !grad_xi) return GMCS_E_INVALID;
    int rc = check_pass_state(c);
    if (rc) return rc;
    rc = upload_scan(c, scan, N);
    if (rc) return rc;
    const float* T = nullptr;
    const int* perm = nullptr;
    if ((rc = perturbed_poses(c, xi, &T))) return rc;
    if ((rc = locality_order(c, &perm))) return rc;
    if ((rc = run_pass(c, N, true, false, nullptr, c->gbuf, nullptr, nullptr, T, perm))) return rc;
    const float* dxi = is_device_ptr(xi) ? xi : c->stage;
    const float* dgl = grad_ll;
    if (!is_device_ptr(grad_ll)) {
        CK(cudaMemcpyAsync(c->ll, grad_ll, sizeof(float) * c->P, cudaMemcpyHostToDevice, c->stream));
        dgl = c->ll;
    }
    const bool dev = is_device_ptr(grad_xi);
    float* out = dev ? grad_xi : reinterpret_cast<float*>(c->part);
    {
        Launch L(c, K_MISC);
        launch_chain(dxi, c->gbuf, dgl, c->P, out, c->stream);
    }
    if ((rc = check_launch())) return rc;
    if (!dev) return copy_out(c, grad_xi, out, sizeof(float) * 6 * (size_t)c->P);
    return GMCS_OK;
}

int gmcs_move(gmcs_ctx* c, const float* scan, int N) {
    if (!c) return GMCS_E_INVALID;
    int rc = check_pass_state(c);
    if (rc) return rc;
    rc = upload_scan(c, scan, N);
    if (rc) return rc;
    c->version++;
    return run_pass(c, N, true, true, nullptr, nullptr, nullptr, nullptr);
}

int gmcs_weigh(gmcs_ctx* c, const float* ll, double* w_out, gmcs_step_out* res) {
    if (!c || !ll) return GMCS_E_INVALID;
    if (!c->have_particles) return GMCS_E_STATE;
    const float* dll = ll;
    if (!is_device_ptr(ll)) {
        CK(cudaMemcpyAsync(c->ll, ll, sizeof(float) * c->P, cudaMemcpyHostToDevice, c->stream));
        dll = c->ll;
    }
    int rc = run_weigh(c, dll);
    if (rc) return rc;
    if (w_out) {
        const bool dev = is_device_ptr(w_out);
        double* dw = dev ? w_out : reinterpret_cast<double*>(c->part);
        ScanArgs sa;   // the scan kernel's first half writes the normalised weights
        sa.logw = c->logw;
        sa.w = nullptr;
        sa.res = c->d_res;
        sa.w_out = dw;
        sa.P = c->P;
        sa.cl = c->cl;
        sa.btot = c->btot;
        {
            Launch L(c, K_RESAMPLE);
            launch_resample_scan(sa, c->stream);
        }
        if ((rc = check_launch())) return rc;
        if (!dev && (rc = copy_out(c, w_out, dw, sizeof(double) * c->P))) return rc;
    }
    if (res) {
        CK(cudaMemcpyAsync(c->h_res, c->d_res, sizeof(WeighResult), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        fill_out(*c->h_res, c->frame, res);
    }
    return GMCS_OK;
}

int gmcs_resample(gmcs_ctx* c, const double* w, int P, double u, int* anc) {
    if (!c || !w || !anc || P <= 0) return GMCS_E_INVALID;
    if (P > c->Pmax) return GMCS_E_CAPACITY;
    if (!(u >= 0.0 && u < 1.0)) return GMCS_E_INVALID;
    const double* dw = w;
    if (!is_device_ptr(w)) {
        CK(cudaMemcpyAsync(c->part, w, sizeof(double) * P, cudaMemcpyHostToDevice, c->stream));
        dw = reinterpret_cast<const double*>(c->part);
    }
    const bool dev = is_device_ptr(anc);
    int rc = run_resample_core(c, P, dw, nullptr, nullptr, u, 0, 0, dev ? anc : c->anc);
    if (rc) return rc;
    if (!dev) return copy_out(c, anc, c->anc, sizeof(int) * P);
    return GMCS_OK;
}

int gmcs_prune(gmcs_ctx* c, const double* x, const double* w, const float* ll, int P, int argmax, double u,
               int* anc, double* logw, int* n_dead) {
    if (!c || !x || !w || !anc || !logw || P <= 0) return GMCS_E_INVALID;
    if (P > c->Pmax) return GMCS_E_CAPACITY;
    if (argmax < 0 || argmax >= P || !(u >= 0.0 && u < 1.0)) return GMCS_E_INVALID;
    // inputs into scratch (the context's particles and diagnostics stay as they are):
    // w and x as doubles in the partial-sum buffer, ll in the staging buffer
    double* dw = reinterpret_cast<double*>(c->part);
    double* dx = dw + c->ld;
    float* dll = ll ? c->stage : nullptr;
    CK(cudaMemcpyAsync(dx, x, sizeof(double) * P, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(dw, w, sizeof(double) * P, cudaMemcpyDefault, c->stream));
    WeighResult* hr = c->h_res;
    CK(cudaStreamSynchronize(c->stream));   // h_res may still be the target of an earlier copy
    std::memset(hr, 0, sizeof(WeighResult));
    hr->M = 0.0;                             // x is normalised: x - 0 - 0 = x exactly
    hr->logS = 0.0;
    hr->argmax = argmax;
    hr->ll_max = -INFINITY;
    if (ll) {
        std::vector<float> h(P);
        CK(cudaMemcpy(h.data(), ll, sizeof(float) * P, cudaMemcpyDefault));
        CK(cudaMemcpyAsync(dll, ll, sizeof(float) * P, cudaMemcpyDefault, c->stream));
        for (int i = 0; i < P; ++i)
            if ((double)h[i] > hr->ll_max) hr->ll_max = (double)h[i];
    }
    CK(cudaMemcpyAsync(c->d_res, hr, sizeof(WeighResult), cudaMemcpyHostToDevice, c->stream));
    PruneArgs pa = prune_args(c, P, c->d_res, dw, dll, u, 0, 0, false);
    pa.logw = dx;
    pa.w_out = nullptr;
    int rc = run_prune(c, pa);
    if (rc) return rc;
    if ((rc = copy_out(c, anc, c->anc, sizeof(int) * P))) return rc;
    if ((rc = copy_out(c, logw, dx, sizeof(double) * P))) return rc;
    CK(cudaMemcpyAsync(hr, c->d_res, sizeof(WeighResult), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (n_dead) *n_dead = hr->pruned;
    return GMCS_OK;
}

int gmcs_overlap(gmcs_ctx* c, const float* scan, int N, const double T_rel[12], double* rate) {
    if (!c || !T_rel || !rate || N <= 0) return GMCS_E_INVALID;
    if (c->K == 0) return GMCS_E_STATE;
    for (int e = 0; e < 12; ++e)
        if (!std::isfinite(T_rel[e])) return GMCS_E_INVALID;
    c->ovl_valid = false;   // the count buffer is shared with the step's rate
    int rc = upload_scan(c, scan, N);
    if (!rc) rc = enqueue_overlap(c, N, T_rel);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    *rate = (double)*c->h_ovl / (double)N;
    return GMCS_OK;
}

int gmcs_get_particles(gmcs_ctx* c, float* poses, double* logw) {
    if (!c) return GMCS_E_INVALID;
    if (!c->have_particles) return GMCS_E_STATE;
    if (poses) {
        {
            Launch L(c, K_MISC);
            launch_soa_to_aos(c->pose[c->cur], c->ld, c->P, 12, c->part, c->stream);
        }
        int rc = check_launch();
        if (rc) return rc;
        if ((rc = copy_out(c, poses, c->part, sizeof(float) * 12 * (size_t)c->P))) return rc;
    }
    if (logw) return copy_out(c, logw, c->logw, sizeof(double) * c->P);
    return GMCS_OK;
}

int gmcs_get_kf_poses(gmcs_ctx* c, int k, float* poses) {
    if (!c || !poses || k < 0 || k >= c->K) return GMCS_E_INVALID;
    {
        Launch L(c, K_MISC);
        launch_soa_to_aos(c->kf[c->cur] + (size_t)k * kPoseC * c->ld, c->ld, c->P, 12, c->part, c->stream);
    }
    int rc = check_launch();
    if (rc) return rc;
    return copy_out(c, poses, c->part, sizeof(float) * 12 * (size_t)c->P);
}

int gmcs_set_kf_poses(gmcs_ctx* c, int k, const float* poses) {
    if (!c || !poses || k < 0 || k >= c->K) return GMCS_E_INVALID;
    c->version++;
    CK(cudaMemcpyAsync(c->part, poses, sizeof(float) * 12 * (size_t)c->P, cudaMemcpyDefault, c->stream));
    {
        Launch L(c, K_MISC);
        launch_aos_to_soa(c->part, c->P, 12, c->kf[c->cur] + (size_t)k * kPoseC * c->ld, c->ld, c->stream);
    }
    int rc = check_launch();
    if (!rc) rc = cuda_status(cudaStreamSynchronize(c->stream));
    return rc;
}

int gmcs_get_frame_diag(gmcs_ctx* c, float* ll, double* w, int* anc, int* nbr) {
    if (!c) return GMCS_E_INVALID;
    if (!c->last_valid) return GMCS_E_STATE;
    int rc = GMCS_OK;
    if (ll && (rc = copy_out(c, ll, c->ll, sizeof(float) * c->P))) return rc;
    if (w && (rc = copy_out(c, w, c->w, sizeof(double) * c->P))) return rc;
    if (anc && (rc = copy_out(c, anc, c->anc, sizeof(int) * c->P))) return rc;
    if (nbr) {
        const int knb = std::min(c->cfg.k_nb, std::max(c->K, 1));
        {
            Launch L(c, K_MISC);   // [k_nb][ld] -> P x k_nb, bit copies
            launch_soa_to_aos(reinterpret_cast<const float*>(c->nbr), c->ld, c->P, knb, c->part, c->stream);
        }
        if ((rc = check_launch())) return rc;
        if ((rc = copy_out(c, nbr, c->part, sizeof(int) * (size_t)c->P * knb))) return rc;
    }
    return GMCS_OK;
}

int gmcs_point_covariances(gmcs_ctx* c, const float* pts, int n, double* cov) {
    if (!c || n < 0 || (n > 0 && (!pts || !cov))) return GMCS_E_INVALID;
    if (n == 0) return GMCS_OK;
    const float* dpts = nullptr;
    float* tmp = nullptr;
    int rc = stage_points(c, pts, n, &dpts, &tmp);
    if (rc) return rc;
    float4* p4 = nullptr;
    double* dcov = is_device_ptr(cov) ? cov : nullptr;
    double* tcov = nullptr;
    if (cudaMalloc((void**)&p4, sizeof(float4) * (size_t)n) != cudaSuccess ||
        (!dcov && cudaMalloc((void**)&tcov, sizeof(double) * 6 * (size_t)n) != cudaSuccess)) {
        cudaGetLastError();
        rc = GMCS_E_OOM;
    }
    if (!rc) {
        if (!dcov) dcov = tcov;
        {
            Launch L(c, K_MISC);
            launch_scan_pack(dpts, n, p4, c->stream);
        }
        KnnCovArgs ka;
        ka.pts = p4;
        ka.n = n;
        ka.k = c->cfg.knn;
        ka.eps = (double)c->cfg.cov_eps;
        ka.cov64 = dcov;
        ka.nrm32 = nullptr;
        {
            Launch L(c, K_MISC);
            launch_knn_cov(ka, c->stream);
        }
        rc = check_launch();
        if (!rc && tcov) rc = copy_out(c, cov, tcov, sizeof(double) * 6 * (size_t)n);
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(p4);
    cudaFree(tcov);
    cudaFree(tmp);
    return rc ? rc : cuda_status(cudaGetLastError());
}

int gmcs_get_table(gmcs_ctx* c, int k, float* vals) {
    if (!c || !vals || k < 0 || k >= c->K) return GMCS_E_INVALID;
    const HostTable& t = c->tables[k];
    if (t.dtype == 3) return copy_out(c, vals, t.cells, t.bytes);   // GICP voxel records as stored
    const size_t nv = (size_t)t.grid.n[0] * t.grid.n[1] * t.grid.n[2];
    const bool dev = is_device_ptr(vals);
    float* dst = dev ? vals : nullptr;
    if (!dev) {
        if (cudaMalloc((void**)&dst, nv * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return GMCS_E_OOM;
        }
    }
    {
        Launch L(c, K_MISC);
        launch_unpack(table_records(t), table_dir(t), t.dtype, t.grid.n[0], t.grid.n[1], t.grid.n[2], dst, c->stream);
    }
    int rc = check_launch();
    if (!rc && !dev) rc = copy_out(c, vals, dst, nv * sizeof(float));
    if (!dev) cudaFree(dst);
    return rc;
}

int gmcs_get_records(gmcs_ctx* c, int k, uint64_t c0, uint64_t n, float* coef) {
    if (!c || !coef || k < 0 || k >= c->K) return GMCS_E_INVALID;
    const HostTable& t = c->tables[k];
    if (t.dtype == 3) return GMCS_E_INVALID;
    const uint64_t ncell = (uint64_t)(t.grid.n[0] - 1) * (t.grid.n[1] - 1) * (t.grid.n[2] - 1);
    if (c0 > ncell || n > ncell - c0) return GMCS_E_INVALID;
    if (n == 0) return GMCS_OK;
    const bool dev = is_device_ptr(coef);
    float* dst = dev ? coef : nullptr;
    if (!dev && cudaMalloc((void**)&dst, n * 8 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return GMCS_E_OOM;
    }
    {
        Launch L(c, K_MISC);
        launch_records(table_records(t), table_dir(t), t.dtype, t.grid.n[0], t.grid.n[1], t.grid.n[2], c0, n, dst,
                       c->stream);
    }
    int rc = check_launch();
    if (!rc && !dev) rc = copy_out(c, coef, dst, n * 8 * sizeof(float));
    if (!dev) cudaFree(dst);
    return rc;
}

int gmcs_state_version(gmcs_ctx* c, uint64_t* version) {
    if (!c || !version) return GMCS_E_INVALID;
    *version = c->version;
    return GMCS_OK;
}

int gmcs_get_sizes(gmcs_ctx* c, int* P, int* K, uint32_t* frame) {
    if (!c) return GMCS_E_INVALID;
    if (P) *P = c->P;
    if (K) *K = c->K;
    if (frame) *frame = c->frame;
    return GMCS_OK;
}

int gmcs_set_profiling(gmcs_ctx* c, int on) {
    if (!c) return GMCS_E_INVALID;
    c->profiling = on != 0;
    return GMCS_OK;
}

int gmcs_get_stats(gmcs_ctx* c, gmcs_stats* out) {
    if (!c || !out) return GMCS_E_INVALID;
    harvest(c);
    std::memset(out, 0, sizeof(*out));
    out->launches = c->launches;
    out->frames = c->frames;
    out->profiling = c->profiling ? 1 : 0;
    out->n_kinds = K_COUNT;
    for (int k = 0; k < K_COUNT; ++k) {
        out->kind[k] = kKindName[k];
        out->kind_launches[k] = c->kind_launches[k];
        out->kind_ms[k] = c->kind_ms[k];
    }
    return GMCS_OK;
}

int gmcs_reset_stats(gmcs_ctx* c) {
    if (!c) return GMCS_E_INVALID;
    harvest(c);
    c->launches = 0;
    c->frames = 0;
    for (int k = 0; k < K_COUNT; ++k) {
        c->kind_launches[k] = 0;
        c->kind_ms[k] = 0.0;
    }
    return GMCS_OK;
}

int gmcs_device_bytes(gmcs_ctx* c, uint64_t* bytes) {
    if (!c || !bytes) return GMCS_E_INVALID;
    *bytes = c->dev_bytes;
    return GMCS_OK;
}

}  // extern "C"
