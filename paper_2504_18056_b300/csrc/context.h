// context.h -- the filter context behind the C ABI (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/gmcs.h"
#include "kernels.h"

namespace gmcs {

enum Kind { K_PREDICT, K_SELECT, K_PASS_GRAD, K_PASS_VALUE, K_FINISH, K_WEIGH, K_RESAMPLE, K_GATHER, K_TABLE, K_MISC, K_COUNT };

struct HostTable {
    void* cells = nullptr;           // the allocation: [column directory][cell records] (field) or voxel records (GICP)
    size_t bytes = 0;                // allocation size
    size_t dir_bytes = 0;            // column-sparse field tables: directory bytes (256-byte aligned); dense: 0
    int layout = 0;                  // GMCS_LAYOUT_*
    gmcs_grid grid;
    int dtype = 0;
    unsigned char* occ = nullptr;   // occupancy lattice for the overlap rate (Sec. III-E)
    gmcs_grid occ_grid;
    size_t occ_bytes = 0;
};

// First cell record and column directory of a table (dense: no directory).
inline void* table_records(const HostTable& t) { return static_cast<char*>(t.cells) + t.dir_bytes; }
inline const uint2* table_dir(const HostTable& t) {
    return t.dir_bytes ? static_cast<const uint2*>(t.cells) : nullptr;
}

struct EvPair {
    int kind;
    cudaEvent_t a, b;
};

}  // namespace gmcs

struct gmcs_ctx {
    gmcs_config cfg;
    int device = 0;
    cudaStream_t stream = nullptr;
    int Pmax = 0, Kmax = 0, Nmax = 0;
    size_t ld = 0;
    int P = 0, K = 0;
    uint32_t frame = 0;
    uint64_t version = 0;            // bumped by every call that changes poses, neighbours or keyframes
    int* perm = nullptr;             // locality order of the particles (differentiable log-likelihood)
    uint32_t* order_scratch = nullptr;
    uint64_t perm_version = ~0ull;   // state version the order was computed for
    int nbr_K = 0;                    // keyframes when the neighbours were last selected (0: never)
    bool have_particles = false;
    int cur = 0;
    float* pose[2] = {nullptr, nullptr};
    float* kf[2] = {nullptr, nullptr};
    double* logw = nullptr;
    double* w = nullptr;             // normalised weights of the last frame
    float* gbuf = nullptr;           // P x 6 gradients (differentiable log-likelihood)
    float* ll = nullptr;
    int* nbr = nullptr;
    float* part = nullptr;
    size_t part_floats = 0;
    float4* scan = nullptr;
    float4* scov = nullptr;          // GICP: scan point normals (plane-regularised covariances)
    float* stage = nullptr;          // N x 3 points / P x 6 noise staging
    size_t stage_floats = 0;
    double* wpart = nullptr;
    unsigned* counter = nullptr;
    gmcs::WeighResult* d_res = nullptr;
    gmcs::WeighResult* h_res = nullptr;    // pinned
    unsigned long long* cl = nullptr;
    unsigned long long* btot = nullptr;
    unsigned long long* dtot = nullptr;   // pruning: dead counts per scan block
    int* anc = nullptr;
    gmcs::TableDesc* d_tables = nullptr;
    std::vector<gmcs::HostTable> tables;
    std::vector<double> kf_path;     // odometry path length at each keyframe
    double path_now = 0.0;           // and at the current frame
    float* d_kf_path = nullptr;
    double odo[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};   // odometry pose of the frame in the last keyframe's frame
    int* d_mm = nullptr;             // bounding-box scratch (6 ints)
    unsigned* d_ovl = nullptr;       // overlap hit count of the frame
    unsigned* h_ovl = nullptr;       // pinned copy
    bool ovl_valid = false;
    int last_N = 0;
    int last_inserted = 0;
    unsigned* d2 = nullptr;
    size_t d2_cap = 0;
    size_t dev_bytes = 0;
    // stats
    uint64_t launches = 0, frames = 0;
    uint64_t kind_launches[gmcs::K_COUNT] = {0};
    double kind_ms[gmcs::K_COUNT] = {0};
    bool profiling = false;
    std::vector<gmcs::EvPair> pending;
    std::vector<cudaEvent_t> free_events;
    gmcs_step_out last{};
    bool last_valid = false;
};

namespace gmcs {

// Argument records of one session's kernels, built exactly as the single-session
// frame driver builds them (gmcs.cu); the serving path batches them.
int cuda_status(cudaError_t e);
bool config_valid(const gmcs_config* c);   // every field within the range the library accepts
size_t ctx_device_bytes(int max_particles, int max_keyframes, int max_points);
void pass_args(gmcs_ctx* c, int N, bool grad, bool move, float* out_ll, float* out_g, float* out_mom, double* logw,
               const float* pose_override, PassArgs* pa, FinishArgs* fa);
PredictArgs predict_args(gmcs_ctx* c, const double dT[12], const double cov[36], const float* z, uint32_t frame);
SelectArgs select_args(gmcs_ctx* c, int* nbr_out);
WeighArgs weigh_args(gmcs_ctx* c, const float* ll, WeighResult* res);
void resample_args(gmcs_ctx* c, int P, const double* w, const WeighResult* res, double* w_out, double u,
                   int u_from_philox, uint32_t frame, int* anc, ScanArgs* sa, TotalsArgs* ta, SearchArgs* se);
GatherArgs gather_args(gmcs_ctx* c, const WeighResult* res);
PruneArgs prune_args(gmcs_ctx* c, int P, WeighResult* res, const double* w, const float* ll, double u,
                     int u_from_philox, uint32_t frame, bool refill);
void fill_out(const WeighResult& r, uint32_t frame, gmcs_step_out* o);
void pass_shape(int P, int N, int* ntiles, int* groups, int* chunk_len, int max_groups = kMaxGroups);

}  // namespace gmcs
