// kernels.h -- argument records and host launchers of the device kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gmcs {

constexpr int kPassWarps = 4;           // warps per CTA of the lookup pass
constexpr int kPassThreads = 32 * kPassWarps;
#ifndef GMCS_TW
#define GMCS_TW 1
#endif
// A CTA's warps cover kPassTW particle tiles (32 particles each) times
// kPassCW point chunks; warps on the same chunk walk the same points together.
constexpr int kPassTW = GMCS_TW;
constexpr int kPassCW = kPassWarps / kPassTW;
static_assert(kPassTW * kPassCW == kPassWarps, "tile x chunk split of the CTA");
constexpr int kAccGrad = 17;            // ll, d ll/d omega (3), d ll/d v (3), moments (10)
constexpr int kAccGicp = 29;            // GICP: ll, b (6), H upper triangle (21), inlier count
constexpr int kMaxGroups = 8;           // point-chunk groups per particle tile (scratch bound)

// ------------------------------------------------------------------ tables
struct SplatArgs {
    const float* pts;   // n x 3
    int n;
    float o_hi[3], o_lo[3];   // lattice origin as an unevaluated float pair (hi + lo)
    float h_hi, h_lo;         // lattice step likewise
    int nx, ny, nz;
    float r_t;
    unsigned* d2;       // [nz][ny][nx] squared distance as float bits
};

struct PackArgs {
    const unsigned* d2;
    int nx, ny, nz;
    float inv_two_sigma2;   // 1 / (2 sigma^2)
    float r_t2;
    void* cells;
    int dtype;
    const uint2* dir;       // column-sparse: the column directory (dense: null)
};

void launch_fill_u32(unsigned* p, size_t n, unsigned v, cudaStream_t s);
void launch_splat(const SplatArgs& a, cudaStream_t s);
void launch_pack(const PackArgs& a, cudaStream_t s);
void launch_unpack(const void* cells, const uint2* dir, int dtype, int nx, int ny, int nz, float* out, cudaStream_t s);
void launch_records(const void* cells, const uint2* dir, int dtype, int nx, int ny, int nz, size_t c0, size_t n,
                    float* out, cudaStream_t s);
// column-sparse tables: per column (zlo | count << 16) of its nonzero run, from the squared distances
void launch_col_range(const unsigned* d2, int nx, int ny, int nz, float inv_two_sigma2, float r_t2, uint32_t* out,
                      cudaStream_t s);

// ------------------------------------------------------------------ filter
struct ScanPackArgs {
    const float* xyz;       // n x 3
    int n;
    float4* out;
};

struct PredictArgs {
    float* pose;            // [12][ld], in/out
    size_t ld;
    int P;
    float dT[12];
    float cov[36];
    const float* z;         // P x 6 or null
    uint64_t seed;
    uint32_t frame;
};

struct SelectArgs {
    const float* pose;
    const float* kf;        // [K][12][ld]
    size_t ld;
    int P, K, k_nb;
    int* nbr;               // [k_nb][ld]
    int* nbr_out;           // P x k_nb (row-major) or null
};

struct PassArgs {
    const float* pose;
    const float* kf;
    const int* nbr;
    const TableDesc* tables;
    const float4* scan;
    const float4* scov;     // GICP: scan point normals (n, 0); covariance I - cov_w n n^T
    float cov_w, cov_eps;   // GICP: 1 - eps and eps of the plane regularisation
    float tau;              // GICP: cap of a term's e^T Omega e
    int model;              // 0 voxel likelihood field, 1 GICP
    float* part;            // [groups][nacc][ld]
    size_t ld;
    int P, N, k_nb;
    int ntiles, groups, chunk_len;   // groups: chunk groups (kPassCW chunks each)
    float eps;
    int want_ll;            // gradient pass: also accumulate the log-likelihood (the moves do not need it)
    int sparse;             // the context's tables are column-sparse (TableDesc::dir)
    const int* perm;        // optional order of the particles over the lanes (null: lane tile*32 + l is particle tile*32 + l)
};

struct FinishArgs {
    const float* part;
    float* pose;            // moved in place when do_move
    size_t ld;
    int P, groups;
    int do_move;
    float sigma, lambda, theta_max, t_max, w_min;
    float* out_ll;          // P
    float* out_g;           // P x 6
    float* out_mom;         // P x 10
    double* logw;           // value pass: logw += ll when non-null
    // keyframe pose propagation (Eq. 8-10) and the loop condition (moves only)
    float* kf;              // [K][12][ld]
    const int* nbr;         // [k_nb][ld]
    const float* kf_path;   // K odometry path lengths
    float path_now;
    int K, k_nb, propagate, loop_recent;
    int model;              // 0 voxel likelihood field, 1 GICP
};

// Differentiable log-likelihood: poses T0 exp(xi) and the chain rule through Jr(xi).
void launch_perturb(const float* pose0, const float* xi, int P, size_t ld, float* dst, cudaStream_t s);
void launch_chain(const float* xi, const float* g, const float* grad_ll, int P, float* grad_xi, cudaStream_t s);

void launch_scan_pack(const float* xyz, int n, float4* out, cudaStream_t s);
void launch_aos_to_soa(const float* aos, int P, int C, float* soa, size_t ld, cudaStream_t s);
void launch_soa_to_aos(const float* soa, size_t ld, int P, int C, float* aos, cudaStream_t s);
void launch_predict(const PredictArgs& a, cudaStream_t s);
void launch_select(const SelectArgs& a, cudaStream_t s);
void launch_pass(const PassArgs& a, int dtype, bool grad, cudaStream_t s);
void launch_gicp_pass(const PassArgs& a, bool grad, cudaStream_t s);

// GICP keyframe maps and scan covariances (k_gicp.cu).
struct KnnCovArgs {
    const float4* pts;      // n points (x, y, z, -)
    int n, k;               // k nearest (the point itself included), k <= kKnnMax
    double eps;             // plane regularisation: eigenvalues (eps, 1, 1)
    double* cov64;          // optional n x 6 doubles (xx xy xz yy yz zz)
    float4* nrm32;          // optional unit normal per point (n, 0): covariance I - (1 - eps) n n^T
};
constexpr int kKnnMax = 32;
void launch_knn_cov(const KnnCovArgs& a, cudaStream_t s);
struct VoxelArgs {
    const float4* pts;
    const double* cov;      // n x 6
    int n;
    double ox, oy, oz, h;
    int nx, ny, nz;
    double* sums;           // voxels x 10: sum p (3), count, sum cov (6)
    float4* rec;            // voxels x 3 float4: mean + valid | xx xy xz yy | yz zz 0 0
};
void launch_voxel_accum(const VoxelArgs& a, cudaStream_t s);
void launch_voxel_final(const VoxelArgs& a, cudaStream_t s);
int grid_knn_cov(int n);

// Keyframe insertion by overlap (k_keyframe.cu).
struct BBoxArgs {
    const float4* pts;
    int n;
    int* mm;                // 6 ints: order-preserving int images of min x, y, z and max x, y, z
};
struct OccArgs {
    const float4* pts;
    int n;
    double ox, oy, oz, h;
    int nx, ny, nz;
    unsigned char* occ;     // [nz][ny][nx], 1 where a point falls
};
struct OverlapArgs {
    const float4* scan;
    int n;
    double T[12];           // scan frame -> keyframe frame (odometry), row-major 3 x 4
    const unsigned char* occ;
    double ox, oy, oz, h;
    int nx, ny, nz;
    unsigned* count;        // += scan points over occupied voxels
};
void launch_bbox(const BBoxArgs& a, cudaStream_t s);
void launch_occ_fill(const OccArgs& a, cudaStream_t s);
void launch_overlap(const OverlapArgs& a, cudaStream_t s);
void launch_finish(const FinishArgs& a, bool grad, cudaStream_t s);

// ------------------------------------------------------------------ weights / resampling
struct WeighResult {
    double M;           // max log-weight
    double logS;        // log sum exp(logw - M)
    double ess;         // S^2 / S2
    double max_w;
    double ll_max;      // max of the frame log-likelihoods (WeighArgs::llm), -inf without
    int argmax;
    int nonfinite;      // 1 if every log-weight was -inf or NaN
    int do_resample;    // policy decision
    int pruned;         // dead particles refilled (pruning policy)
    float est[12];      // pose of argmax (before resampling)
};

struct WeighArgs {
    double* logw;       // in/out
    const float* ll;    // added to logw first when non-null
    int P;
    int policy;         // 0 always, 1 ESS < P/2, 2 never, 3 prune
    const float* llm;   // frame log-likelihoods whose max goes to res->ll_max, or null
    double* part;       // kWeighPart doubles per block
    unsigned* counter;  // zero between launches
    WeighResult* res;
    const float* pose;  // current poses (for the estimate)
    size_t ld;
};

struct ScanArgs {
    const double* logw;     // weights from log-weights (when w is null)
    const double* w;        // given normalised weights, or null
    const WeighResult* res; // M, logS (when w is null)
    double* w_out;          // optional normalised weights
    int P;
    unsigned long long* cl;     // block-local inclusive prefix of q
    unsigned long long* btot;   // per-block totals -> exclusive offsets
};

struct TotalsArgs {
    unsigned long long* btot;   // block totals -> exclusive offsets, grand total at [nblocks]
    int nblocks;
};

struct SearchArgs {
    const unsigned long long* cl;
    const unsigned long long* boff;   // exclusive block offsets, then total at [nblocks]
    int nblocks;
    int P;
    double u;               // systematic offset when u_from_philox == 0
    int u_from_philox;      // 1: u = 53-bit Philox draw for (seed, frame)
    uint64_t seed;
    uint32_t frame;
    const WeighResult* res; // do_resample flag (identity when 0); may be null
    int* anc;
};

struct GatherArgs {
    const float* pose_src;
    float* pose_dst;
    const float* kf_src;
    float* kf_dst;
    size_t ld;
    int P, K;
    const int* anc;
    double* logw;
    const WeighResult* res;   // null: resampled unconditionally
};

constexpr int kScanBlock = 1024;
constexpr int kWeighPart = 5;   // doubles per weigh block partial (M, S, S2, argmax, ll max)

// Dead-particle pruning (Sec. III-F): mark + block scans, scans of the block
// totals, refill of the dead slots, weight split. State is refilled in place.
struct PruneArgs {
    double* logw;             // in: log-weights (x = logw - M - logS); out: new log-weights
    const double* w;          // given normalised weights, or null (w = exp(x))
    double* w_out;            // optional normalised weights
    const float* ll;          // frame log-likelihoods (likelihood criterion), or null
    WeighResult* res;         // M, logS, argmax, ll_max, nonfinite in; pruned out
    float* pose;              // current poses [12][ld] (null: no state refill)
    float* kf;                // keyframe poses [K][12][ld]
    size_t ld;
    int P, K;
    int nblocks;              // scan blocks of kScanBlock particles
    unsigned long long* cl;   // block-local inclusive prefix of q
    unsigned long long* btot; // q block totals -> exclusive offsets, total at [nblocks]
    unsigned long long* dtot; // dead counts per block -> exclusive offsets, total at [nblocks]
    int* anc;                 // i for survivors, ancestor for dead slots
    double prune_w;           // posterior threshold
    double ll_cut;            // log likelihood-ratio threshold (-inf: off)
    double u;                 // systematic offset when u_from_philox == 0
    int u_from_philox;
    uint32_t frame;
    uint64_t seed;
};

void launch_weigh(const WeighArgs& a, int nblocks, cudaStream_t s);
constexpr int kWeighMaxBlocks = 148 * 4;   // CTA partials of the weight reduction (scratch bound)
int weigh_blocks(int P);
void launch_resample_scan(const ScanArgs& a, cudaStream_t s);
void launch_scan_totals(unsigned long long* btot, int nblocks, cudaStream_t s);
void launch_resample_search(const SearchArgs& a, cudaStream_t s);
void launch_gather(const GatherArgs& a, cudaStream_t s);
void launch_normalize(double* logw, int P, const WeighResult* res, double* w_out, int* anc, cudaStream_t s);
void launch_prune_mark(const PruneArgs& a, cudaStream_t s);
void launch_prune_totals(const PruneArgs& a, cudaStream_t s);
void launch_prune_spawn(const PruneArgs& a, cudaStream_t s);
void launch_prune_reweigh(const PruneArgs& a, cudaStream_t s);

// ------------------------------------------------------------------ batched (serving) launches
// One launch covers the work of up to kMaxSlots sessions: session s owns the
// virtual blocks [offset[s], offset[s] + vgrid[s]) of a persistent grid that
// walks them in order; each virtual block runs the same body as the
// single-session kernel with blockIdx / gridDim replaced by (vb, vgrid[s]).
constexpr int kMaxSlots = 32;

// Persistent-grid walk over a BatchList: CTA-sized items, item -> (session s,
// virtual block vb of vgrid[s]); every thread reaches the barrier after each item.
#define GMCS_BATCH_LOOP(L, CALL)                                               \
    for (int item = blockIdx.x; item < (L)->total; item += gridDim.x) {        \
        int s = 0;                                                             \
        while (s + 1 < (L)->count && (L)->offset[s + 1] <= item) ++s;          \
        const int vb = item - (L)->offset[s], vg = (L)->vgrid[s];              \
        (void)vg;                                                              \
        CALL;                                                                  \
        __syncthreads();                                                       \
    }

template <typename A>
struct BatchList {
    int count;                 // sessions in this launch
    int total;                 // sum of vgrid
    int vgrid[kMaxSlots];
    int offset[kMaxSlots];     // exclusive prefix of vgrid
    A args[kMaxSlots];
};

void launch_scan_pack_b(const BatchList<ScanPackArgs>* L, cudaStream_t s);
void launch_predict_b(const BatchList<PredictArgs>* L, cudaStream_t s);
void launch_select_b(const BatchList<SelectArgs>* L, cudaStream_t s);
void launch_pass3_b(const BatchList<PassArgs>* L, int dtype, bool grad, bool sparse, cudaStream_t s);
// a locality order of P particles (k_order.cu): Morton buckets of their translations
size_t order_scratch_words(int P);
void launch_locality_order(const float* pose, size_t ld, int P, uint32_t* scratch, int* perm, cudaStream_t s);
void launch_finish_b(const BatchList<FinishArgs>* L, bool grad, bool gicp, cudaStream_t s);
void launch_weigh_b(const BatchList<WeighArgs>* L, cudaStream_t s);
void launch_resample_scan_b(const BatchList<ScanArgs>* L, cudaStream_t s);
void launch_scan_totals_b(const BatchList<TotalsArgs>* L, cudaStream_t s);
void launch_resample_search_b(const BatchList<SearchArgs>* L, cudaStream_t s);
void launch_gather_b(const BatchList<GatherArgs>* L, cudaStream_t s);
void launch_prune_mark_b(const BatchList<PruneArgs>* L, cudaStream_t s);
void launch_prune_totals_b(const BatchList<PruneArgs>* L, cudaStream_t s);
void launch_prune_spawn_b(const BatchList<PruneArgs>* L, cudaStream_t s);
void launch_prune_reweigh_b(const BatchList<PruneArgs>* L, cudaStream_t s);
void launch_knn_cov_b(const BatchList<KnnCovArgs>* L, int k, cudaStream_t s);
void launch_gicp_b(const BatchList<PassArgs>* L, bool grad, cudaStream_t s);
void prepare_gicp_batched();
// Size every persistent grid (occupancy queries) before a graph capture records the launches.
void prepare_filter_batched();
void prepare_weights_batched();

// Virtual grid sizes of the single-session launches (the batched launches use the same).
int grid_scan_pack(int n);
int grid_per_particle(int P);          // 128-thread blocks
int grid_pass(const PassArgs& a);
int grid_resample_scan(int P);
int grid_resample_search(int P);
int grid_gather(const GatherArgs& a);
int grid_prune_slots(int P);           // spawn / reweigh: 256-thread blocks over the slots

}  // namespace gmcs
