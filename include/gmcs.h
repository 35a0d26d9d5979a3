/*
 * gmcs.h -- C ABI of the B300 (sm_103a) per-frame particle update of
 * gradient-guided Monte Carlo SLAM (Nakao et al., "Range-based 6-DoF Monte
 * Carlo SLAM with Gradient-guided Particle Filter on GPU", arXiv 2504.18056).
 *
 * The problem statement of Sec. III-A: estimate the sensor pose T_t and the map
 * from range scans and odometry, with every particle x_t^i holding its current
 * pose T_t^i plus its own copy T_k^i of every keyframe pose, while keyframe
 * point clouds are stored once and shared by all particles.
 *
 * The map of each keyframe is a voxel likelihood field: on a lattice of edge h,
 * vertex value exp(-d^2 / 2 sigma^2) with d the distance to the nearest
 * keyframe point (0 beyond r_t), read by trilinear interpolation. This replaces
 * the GICP distribution-to-distribution metric of Eq. 2-4 on the hot path.
 *
 * Conventions (all entry points)
 *   - Return GMCS_OK (0) or a negative GMCS_E_* code; nothing is thrown across
 *     the ABI; gmcs_strerror() names the code. After GMCS_E_INVALID or
 *     GMCS_E_CAPACITY the context is unchanged and usable. GMCS_E_CUDA means a
 *     CUDA call failed and the context should be destroyed.
 *   - Poses at the boundary are 12 floats (or doubles where stated), row-major
 *     3x4 [R | t], mapping sensor-frame points into the frame of reference:
 *     x = R p + t. Arrays of poses are P x 12 (particle-major).
 *   - Tangent vectors are xi = [omega(3); v(3)], rotation first; poses are
 *     perturbed on the right, T exp(xi) (Eq. 1, Eq. 7, Eq. 10).
 *   - Pointer arguments marked "host or device" are classified with
 *     cudaPointerGetAttributes; device pointers must belong to the context's
 *     device. The caller keeps ownership of every buffer it passes; inputs are
 *     consumed in stream order on the context's stream (a host input is copied
 *     before the call returns). The library owns all state it allocates.
 *   - All GPU work is enqueued on the stream given to gmcs_create. Calls that
 *     return results to host memory synchronise that stream.
 *   - One context is not thread-safe; distinct contexts are independent.
 */
#ifndef GMCS_H
#define GMCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GMCS_OK 0
#define GMCS_E_INVALID (-1)   /* bad argument, size or pointer */
#define GMCS_E_OOM (-2)       /* device or pinned allocation failed */
#define GMCS_E_CUDA (-3)      /* a CUDA runtime call failed */
#define GMCS_E_CAPACITY (-4)  /* more particles / keyframes / points than the context holds */
#define GMCS_E_STATE (-5)     /* call out of order (e.g. step before particles exist) */
#define GMCS_E_NONFINITE (-6) /* weights degenerated (all log-weights -inf or NaN); reset to uniform */
#define GMCS_E_BUDGET (-7)    /* serving: the session does not fit the memory budget or the session limit */
#define GMCS_E_IO (-8)        /* checkpoint file cannot be written, read or is not a checkpoint */
#define GMCS_PENDING 1        /* serving: the frame has not completed yet */

#define GMCS_LAYOUT_DENSE 0     /* one record per lattice cell */
#define GMCS_LAYOUT_COLUMNS 1   /* per (x, y) column only the run of cells whose polynomial is not zero */
#define GMCS_TABLE_F32 0
#define GMCS_TABLE_BF16 1
#define GMCS_TABLE_F16 2

#define GMCS_RESAMPLE_ALWAYS 0
#define GMCS_RESAMPLE_ESS_HALF 1
#define GMCS_RESAMPLE_NEVER 2
#define GMCS_RESAMPLE_PRUNE 3 /* dead-particle pruning (Sec. III-F): refill only the dead slots */

#define GMCS_MAX_NB 8         /* upper bound on k_nb */

#define GMCS_MODEL_FIELD 0    /* voxel likelihood field exp(-d^2 / 2 sigma^2), trilinear */
#define GMCS_MODEL_GICP 1     /* GICP distribution-to-distribution terms on voxel maps (Eq. 2-6) */
#define GMCS_KNN_MAX 32       /* upper bound on knn */

typedef struct {
    float sigma;       /* field width (m): vertex value exp(-d^2 / 2 sigma^2) */
    float r_t;         /* truncation radius (m): value 0 where d > r_t */
    float eps;         /* likelihood floor: per-lookup log-likelihood log(L + eps) */
    float lambda;      /* Levenberg-Marquardt factor: H_ii *= (1 + lambda) */
    float theta_max;   /* rad, clamp on |psi_omega| per move */
    float t_max;       /* m, clamp on |psi_v| per move */
    float w_min;       /* no move when the contact weight W = sum L/(L+eps) < w_min */
    int k_nb;          /* neighbour keyframes per particle (Sec. III-C: three) */
    int steps;         /* gradient-guided moves per frame */
    int table_dtype;   /* GMCS_TABLE_* storage type of the likelihood tables */
    int resample;      /* GMCS_RESAMPLE_* policy */
    int propagate;     /* 1: after every move, propagate psi to the particle's keyframe poses
                          (Eq. 8-10, see gmcs_set_path); 0: off */
    int loop_recent;   /* > 0: a particle moves only when its oldest neighbour keyframe is not
                          among the loop_recent newest keyframes (the loop condition of
                          Sec. III-C2); 0: every particle moves every frame */
    float prune_w;     /* GMCS_RESAMPLE_PRUNE: a particle whose normalised weight is below
                          prune_w is dead (the posterior criterion of Sec. III-F; 1e-8) */
    float prune_lr;    /* GMCS_RESAMPLE_PRUNE: a particle whose frame likelihood is below
                          prune_lr times the best particle's is dead (the likelihood criterion
                          of Sec. III-F, relative to the frame's best; 1e-16); 0: off */
    int model;         /* GMCS_MODEL_* likelihood of the context (its keyframes' map type) */
    int knn;           /* GICP: neighbours per point covariance (the point included; 10) */
    float cov_eps;     /* GICP: plane regularisation, covariance eigenvalues (cov_eps, 1, 1) */
    float gicp_tau;    /* GICP: cap of a term's e^T Omega e; points without a voxel or with
                          e^T Omega e >= gicp_tau add -gicp_tau and no gradient (20) */
    float kf_overlap;  /* > 0: gmcs_step inserts the frame as a keyframe when its overlap rate
                          with the last keyframe falls below this (Sec. III-E: 0.7); 0: off */
    float kf_voxel;    /* voxel edge (m) of the keyframes' occupancy lattices (1.0) */
    float kf_h;        /* lattice step (field) or voxel edge (GICP) of inserted keyframes (0.2) */
    int table_layout;  /* GMCS_LAYOUT_* of the field tables: dense lattice, or column-sparse */
    uint64_t seed;     /* key of the Philox4x32-10 draws (motion noise, resampling offset) */
} gmcs_config;

/* Lattice of one keyframe table, in the keyframe's own frame: vertex (ix,iy,iz)
 * sits at origin + h*(ix,iy,iz), 0 <= ix < n[0] etc. At least 2 and at most 2^22
 * vertices per axis. */
typedef struct {
    double origin[3];
    double h;
    int n[3];
} gmcs_grid;

typedef struct {
    double estimate[12];  /* current pose of the largest-weight particle (Sec. IV-A), before resampling */
    double ess;           /* effective sample size 1 / sum w^2 of the normalised weights */
    double max_w;         /* largest normalised weight */
    double log_norm;      /* M + log S of the log-sum-exp normalisation */
    int argmax;           /* its index (lowest index on ties) */
    int resampled;        /* 1 if systematic resampling ran this frame */
    uint32_t frame;       /* frame counter used for this frame's draws */
    int status;           /* GMCS_OK or GMCS_E_NONFINITE */
    int pruned;           /* GMCS_RESAMPLE_PRUNE: dead particles refilled this frame */
    int kf_inserted;      /* 1 if the frame was inserted as a keyframe (cfg.kf_overlap) */
    double overlap;       /* overlap rate with the last keyframe (cfg.kf_overlap > 0), else -1 */
} gmcs_step_out;

typedef struct {
    uint64_t launches;        /* kernels launched by this context since creation */
    uint64_t frames;          /* gmcs_step calls completed */
    int profiling;            /* 1 while per-kernel event timing is enabled */
    int n_kinds;              /* entries used below */
    const char* kind[16];     /* kernel family names */
    uint64_t kind_launches[16];
    double kind_ms[16];       /* summed event time per family (profiling only) */
} gmcs_stats;

typedef struct gmcs_ctx gmcs_ctx;

/* Defaults: sigma 0.2 m, r_t 1.0 m, eps 1e-3, lambda 1e-3, theta_max 2 deg,
 * t_max 0.1 m, w_min 1e-6, k_nb 3, steps 3, FP32 tables, resample always,
 * no propagation, no loop condition, prune_w 1e-8, prune_lr 1e-16, voxel field
 * model (GICP settings knn 10, cov_eps 1e-3, gicp_tau 20), no keyframe insertion
 * (kf_voxel 1.0, kf_h 0.2), seed 0. */
void gmcs_config_default(gmcs_config* cfg);

/*
 * Create a context on the current CUDA device, holding up to max_particles
 * particles, max_keyframes keyframes and scans of up to max_points points.
 * cuda_stream is a cudaStream_t (NULL = legacy default stream). Allocates all
 * per-particle device state up front: poses and keyframe poses double-buffered
 * (2 x 48 B x (1 + max_keyframes) per particle) plus per-frame scratch.
 * Errors: GMCS_E_INVALID (sizes <= 0, k_nb outside 1..GMCS_MAX_NB, bad config),
 * GMCS_E_OOM.
 */
int gmcs_create(const gmcs_config* cfg, int max_particles, int max_keyframes, int max_points,
                void* cuda_stream, gmcs_ctx** out);

/* Free everything the context owns (synchronises its stream). NULL is a no-op. */
int gmcs_destroy(gmcs_ctx* ctx);

/*
 * Set the particle set: P current poses (P x 12 floats, host or device) and
 * optional log-weights (P doubles, host or device; NULL = uniform -log P).
 * Resets the frame counter to 0 and drops nothing else (keyframes stay).
 * Errors: GMCS_E_INVALID, GMCS_E_CAPACITY (P > max_particles).
 */
int gmcs_init_particles(gmcs_ctx* ctx, const float* poses, int P, const double* logw);

/*
 * Insert a keyframe (Sec. III-A: shared cloud P_k, per-particle pose T_k^i).
 * pts: n points (n x 3 floats, host or device) in the keyframe's own frame.
 * grid: the table lattice in that frame. The library builds the table on the
 * device (K8: splat of d^2 within r_t, then exp) and stores one 32-byte
 * (FP32) or 16-byte (BF16/FP16) record per lattice cell, in cfg.table_dtype,
 * holding the 8 coefficients of the cell's trilinear polynomial (differences of
 * the float corner values): FP32 as computed; FP16 rounded to nearest; BF16 as
 * four 32-bit words, each holding one coefficient as a bfloat16 value (rounded
 * to nearest) in its low half and another as the word itself read as an FP32
 * number (the word with that low half nearest to the coefficient: within half a
 * bfloat16 ulp). gmcs_get_records returns the stored values.
 * GICP model: grid is the voxel lattice (n = voxels per axis, voxel (ix,iy,iz)
 * covering origin + h [ix, ix+1) x ...); the library computes every point's
 * plane-regularised covariance from its cfg.knn nearest keyframe points (FP64)
 * and stores per voxel the mean of its points and of their covariances (48 B,
 * FP32). Points outside the lattice are dropped.
 * kf_poses: P x 12 floats (host or device), the keyframe pose held by each
 * particle, or NULL to copy every particle's current pose (the paper's
 * insertion of the current frame as a keyframe). Needs particles to exist.
 * *kf_id receives the keyframe index (0, 1, ...).
 * Errors: GMCS_E_INVALID, GMCS_E_CAPACITY (too many keyframes), GMCS_E_STATE,
 * GMCS_E_OOM (table allocation).
 */
int gmcs_add_keyframe(gmcs_ctx* ctx, const float* pts, int n, const gmcs_grid* grid,
                      const float* kf_poses, int* kf_id);

/*
 * One frame of the hot path, all on the device:
 *   prediction (Eq. 1) with Philox4x32-10 noise of covariance cov,
 *   neighbour keyframes by translation distance (Sec. III-C1), frozen for the frame,
 *   cfg.steps x [scan transform, table lookup, log-likelihood, se(3) gradient and
 *               Gauss-Newton moments per particle, damped move (Eq. 5-7)],
 *   value pass at the moved poses, log-weight update (Eq. 11) with log-sum-exp
 *   normalisation in FP64, argmax estimate,
 *   systematic resampling per cfg.resample (FP64 offsets on 2^-52-quantised
 *   weights, exact integer prefix sums), and the gather of all particle state;
 *   under GMCS_RESAMPLE_PRUNE instead only the dead slots are refilled in place
 *   from the survivors (as gmcs_prune, with the value-pass log-likelihoods).
 * scan: N points (N x 3 floats, host or device) in the sensor frame; a point with
 * a non-finite coordinate is taken as a point far from every map (all its
 * lookups miss), which leaves the normalised weights and the moves unchanged.
 * delta_T: odometry increment (T^o_{t-1})^-1 T^o_t as 12 doubles (host).
 * cov: 6 x 6 motion covariance in the tangent space (36 doubles, host, row-major).
 * u_override: NULL, or a host double in [0,1) used as the systematic offset.
 * out: NULL (asynchronous: nothing is read back; see gmcs_last_result), or a
 * host struct filled after synchronising the stream.
 * Keyframe insertion (Sec. III-E, cfg.kf_overlap > 0): the scan is moved into
 * the last keyframe's frame by the odometry accumulated since that keyframe and
 * its overlap rate (gmcs_overlap) is computed on the device with the frame; with
 * out != NULL, a rate below cfg.kf_overlap inserts the scan as a new keyframe
 * (as gmcs_add_keyframe with kf_poses = NULL: every particle's pose after this
 * frame; lattice step cfg.kf_h over the scan's bounding box plus r_t, or GICP
 * voxels of edge cfg.kf_h) before the call returns, used from the next frame on.
 * The asynchronous form reports the rate through gmcs_last_result only.
 * Errors: GMCS_E_INVALID, GMCS_E_CAPACITY (N > max_points), GMCS_E_STATE (no
 * particles or no keyframes), GMCS_E_CUDA.
 */
int gmcs_step(gmcs_ctx* ctx, const float* scan, int N, const double delta_T[12], const double cov[36],
              const double* u_override, gmcs_step_out* out);

/*
 * Odometry path lengths for keyframe pose propagation (Eq. 9): `now` is the
 * travelled distance at the current frame; kf_path (K doubles, host, or NULL)
 * that at each keyframe's frame. gmcs_add_keyframe records the current value for
 * the new keyframe and gmcs_step adds |t(delta_T)| before its moves. With o the
 * particle's oldest neighbour keyframe, keyframe k > o moves by exp(r_k psi),
 * r_k = (D_k - D_o) / (now - D_o), clamped to [0, 1]; nothing moves if now <= D_o.
 */
int gmcs_set_path(gmcs_ctx* ctx, double now, const double* kf_path);

/* Result of the last gmcs_step (synchronises the stream). */
int gmcs_last_result(gmcs_ctx* ctx, gmcs_step_out* out);

/* ---- stage entry points (each one row of the hot path, on the resident state) */

/* Eq. 1 on all particles. z: NULL (Philox draws for frame `frame`) or P x 6
 * standard normals (host or device floats). Does not advance the frame counter. */
int gmcs_predict(gmcs_ctx* ctx, const double delta_T[12], const double cov[36], const float* z, uint32_t frame);

/* Neighbour keyframes of every particle for its current pose: the k_nb smallest
 * squared distances |t_k^i - t_t^i|^2 (float, formed as (dx*dx + dy*dy) + dz*dz
 * without fused multiply-add), ties to the lower index. nbr_out: NULL or P x k_nb
 * ints (host or device) receiving the indices (-1 for unused slots). */
int gmcs_select(gmcs_ctx* ctx, int* nbr_out);

/*
 * Evaluate the current particles against the scan with the current neighbour
 * sets (gmcs_select or the last step): per particle
 *   ll  = sum_{j, k} log(L_jk + eps)                       (P floats)
 *   g   = d ll / d xi for T_t exp(xi) at xi = 0             (P x 6 floats)
 *   mom = [W, Sx, Sy, Sz, Qxx, Qxy, Qxz, Qyy, Qyz, Qzz], w = L/(L+eps),
 *         W = sum w, S = sum w p, Q = sum w p p^T            (P x 10 floats)
 * GICP model (Eq. 3-6): ll = sum_{j,k} -min(e^T Omega e, gicp_tau) (gicp_tau for
 * points without a voxel), g = 2 b with b = sum J^T Omega e over the inliers
 * (the gradient of ll where Omega does not move with the pose), and mom = the
 * upper triangle of H = sum J^T Omega J, row-major, then the number of inlier
 * lookups (P x 22 floats).
 * Any output may be NULL; outputs are host or device (host: synchronises).
 */
int gmcs_eval(gmcs_ctx* ctx, const float* scan, int N, float* ll, float* g, float* mom);
/* gmcs_eval, gmcs_move, gmcs_loglik and gmcs_loglik_backward return GMCS_E_STATE
 * until the neighbour sets have been selected (gmcs_select or gmcs_step) since the
 * context was created or loaded, and while the context has no particles or no
 * keyframes. */

/* One gradient-guided move of every particle (eval with gradient, then Eq. 5-7
 * with H = sigma^-2 sum w B^T B assembled from the moments). */
int gmcs_move(gmcs_ctx* ctx, const float* scan, int N);

/*
 * Differentiable scan log-likelihood at perturbed poses T_i = T0_i exp(xi_i), T0 the
 * current particle poses and xi P x 6 floats (host or device), with the neighbour
 * keyframes of the last gmcs_select / gmcs_step held fixed:
 *   gmcs_loglik:          ll_i = sum_jk log(L + eps) at T_i            (P floats out)
 *   gmcs_loglik_backward: grad_xi_i = grad_ll_i * d ll_i / d xi_i       (P x 6 floats out)
 *                         = grad_ll_i * Jr(xi_i)^T g_i, g_i the right-perturbation
 *                         gradient at T_i (the lookup pass with gradient) and Jr the
 *                         right Jacobian of SE(3).
 * The scan is re-read in both calls; particle state is not modified. The trilinear
 * field is continuous but its gradient jumps across cell faces; the value is the
 * derivative of the cell polynomials that contain the points at T_i.
 * Both calls run their lookup pass with the particles in a locality order (a
 * counting sort of their current poses -- translation and rotation -- into Morton
 * buckets, kept until the state changes; gmcs_state_version): a set the caller
 * spread or perturbed reads
 * more of the same cells per warp. Each particle is still computed alone, so the
 * results do not depend on the order. The first call allocates the order's
 * scratch (about 4 MB plus 8 bytes per particle).
 */
int gmcs_loglik(gmcs_ctx* ctx, const float* xi, const float* scan, int N, float* ll);
int gmcs_loglik_backward(gmcs_ctx* ctx, const float* xi, const float* scan, int N, const float* grad_ll,
                         float* grad_xi);

/*
 * Log-sum-exp weighting (Eq. 11): logw += ll (ll: P floats, host or device),
 * then w = exp(logw - M - log S) in FP64. w_out: NULL or P doubles (host or
 * device). res: NULL or host struct receiving ess, max_w, argmax, log_norm and
 * the argmax particle's pose. Leaves logw unnormalised (logw + ll).
 */
int gmcs_weigh(gmcs_ctx* ctx, const float* ll, double* w_out, gmcs_step_out* res);

/*
 * Systematic resampling of arbitrary weights (a stand-alone hook on the same
 * kernels the step uses): w (P doubles, host or device, normalised), offset u
 * in [0,1), ancestors written to anc (P ints, host or device):
 *   q_i = rint(w_i 2^52), C_i = q_0 + ... + q_i (exact), S = C_{P-1},
 *   a_m = min{ i : C_i > ((u + m) / P) * S } (IEEE double, no contraction),
 *   clamped to P - 1.
 * P may exceed max_particles only up to the context's scratch (same bound).
 */
int gmcs_resample(gmcs_ctx* ctx, const double* w, int P, double u, int* anc);

/*
 * Dead-particle pruning (Sec. III-F) of arbitrary weights, on the kernels the
 * step runs under GMCS_RESAMPLE_PRUNE; the context's particles are not touched.
 *   x       P normalised log-weights (doubles)
 *   w       P normalised weights, w = exp(x) as the caller computed it (doubles)
 *   ll      P frame log-likelihoods (floats) for the likelihood criterion, or NULL
 *   argmax  index of the largest weight: never pruned
 *   u       systematic offset in [0, 1)
 * Particle i != argmax is dead when w_i is not >= cfg.prune_w, or, with ll and
 * cfg.prune_lr > 0, when ll_i - max_j ll_j is not >= log(prune_lr). With the
 * survivors' weights quantised to q_i = rint(w_i 2^52) (q = 0 when dead),
 * C_i = q_0 + ... + q_i and S = C_{P-1}, the r-th dead slot (index order,
 * r = 0..D-1) takes ancestor a_r = min{ i : C_i > min(((u + r) / D) * S, S - 1) }.
 * Outputs (host or device): anc (P ints: i for survivors, a_r for dead slots),
 * logw (P doubles: x_a - log1p(c_a) for a survivor a with c_a copies and for
 * each of its copies, x_i for survivors without copies), n_dead (host int, may
 * be NULL) = D. All arrays may be host or device memory.
 */
int gmcs_prune(gmcs_ctx* ctx, const double* x, const double* w, const float* ll, int P, int argmax, double u,
               int* anc, double* logw, int* n_dead);

/*
 * The paper has no counterpart of this call: it is systematic resampling, with
 * the same definition and kernels as gmcs_resample, for callers that cannot
 * allocate device memory -- code running under a memory manager that owns the
 * whole device budget, or a real-time loop that cannot afford cudaMalloc's
 * implicit device synchronisation and unbounded latency. It needs no context
 * and allocates nothing: its prefix-sum scratch is a file-scope __device__ array
 * of GMCS_NOALLOC_MAX_P + 257 eight-byte words (about 2.1 MB) that every device
 * which loads the library holds until the process exits.
 *   w    P normalised weights, device doubles (host pointers: GMCS_E_INVALID)
 *   u    systematic offset in [0, 1)
 *   anc  P device ints receiving the ancestors
 *   cuda_stream  stream the work is enqueued on (NULL: legacy default stream);
 *        the call returns without synchronising it
 * P > GMCS_NOALLOC_MAX_P returns GMCS_E_CAPACITY. The first call on a device
 * looks up the array's device address with that device current
 * (cudaGetSymbolAddress); make that first call before any stream capture. The
 * address is kept per device and context: the first call after a
 * cudaDeviceReset (a new context) looks it up again.
 * Every call shares the one array and leaves its contents behind (each call
 * writes all the scratch it reads): calls whose work can overlap on the GPU --
 * on different streams or from different threads -- race on it and must be
 * serialised by the caller.
 */
#define GMCS_NOALLOC_MAX_P 262144
int gmcs_resample_noalloc(const double* w, int P, double u, int* anc, void* cuda_stream);

/* ---- state access */

/* Overlap rate (Sec. III-E) of a scan (N x 3 floats, host or device) with the
 * last keyframe: the share of its points that, moved by T_rel (12 host doubles,
 * the scan's frame in the keyframe's frame), fall into an occupied voxel of the
 * keyframe's occupancy lattice (edge cfg.kf_voxel; per axis from floor(min/h) - 1
 * to floor(max/h) + 1 voxels of the keyframe points). The transform is taken in
 * FP64 with separately rounded products and sums, the voxel is floor((x - o)/h).
 * Errors: GMCS_E_STATE without keyframes. */
int gmcs_overlap(gmcs_ctx* ctx, const float* scan, int N, const double T_rel[12], double* rate);

/*
 * Checkpoint / resume of a session. gmcs_save writes the context's state to a
 * file: particles (current poses, log-weights), every keyframe's table as stored,
 * its occupancy lattice, path length and per-particle poses, and the frame
 * counter, odometry path, odometry since the last keyframe and the config.
 * gmcs_load restores it into a context that holds no keyframes yet and whose
 * capacities are at least the saved counts; the context's config becomes the
 * saved one, and the frames that follow are bit-identical to those the saved
 * context would have computed.
 * gmcs_load checks the whole file on the host before it touches the device:
 * a config the library would not accept, a table whose storage type does not
 * match the config, or any size that disagrees with the lattice it belongs to or
 * with the file's length returns GMCS_E_IO. If the load fails after it began to
 * restore (device error, out of memory), the context is left empty -- no
 * particles, no keyframes -- and can be loaded into again.
 * Errors: GMCS_E_IO (file unreadable, not a checkpoint, inconsistent, or written
 * by another format version: version 3 stores 16-bit field tables as coefficient
 * records), GMCS_E_STATE (save without particles, load
 * into a context with keyframes), GMCS_E_CAPACITY (nothing restored), GMCS_E_OOM.
 */
int gmcs_save(gmcs_ctx* ctx, const char* path);
int gmcs_load(gmcs_ctx* ctx, const char* path);

/* Check a checkpoint file on the host alone (no device, no context) as gmcs_load
 * does, and return its config, particle and keyframe counts and frame counter
 * (any output pointer may be NULL). Errors: GMCS_E_INVALID, GMCS_E_IO. */
int gmcs_checkpoint_info(const char* path, gmcs_config* cfg, int* P, int* K, uint32_t* frame);

/* Copy current poses (P x 12 floats) and/or log-weights (P doubles) out; NULL skips. */
int gmcs_get_particles(gmcs_ctx* ctx, float* poses, double* logw);
/* Copy particle keyframe poses of keyframe k (P x 12 floats). */
int gmcs_get_kf_poses(gmcs_ctx* ctx, int k, float* poses);
/* Overwrite keyframe k's per-particle poses (P x 12 floats, host or device). */
int gmcs_set_kf_poses(gmcs_ctx* ctx, int k, const float* poses);
/*
 * Per-particle diagnostics of the last gmcs_step (any pointer may be NULL; host
 * or device): ll = value-pass log-likelihood (P floats), w = normalised weights
 * before resampling (P doubles), anc = ancestors (P ints; identity when the
 * frame did not resample), nbr = neighbour keyframes (P x k_nb ints).
 */
int gmcs_get_frame_diag(gmcs_ctx* ctx, float* ll, double* w, int* anc, int* nbr);
/* GICP point covariances of a cloud, as the context computes them for scans and
 * keyframes: for each of the n points (n x 3 floats, host or device) the
 * cfg.knn nearest points of the cloud (the point included; squared distances
 * in float as ((dx*dx + dy*dy) + dz*dz), ties to the lower index), their FP64
 * covariance (1/k), plane-regularised to eigenvalues (cfg.cov_eps, 1, 1).
 * cov: n x 6 doubles (xx xy xz yy yz zz), host or device. Any model. */
int gmcs_point_covariances(gmcs_ctx* ctx, const float* pts, int n, double* cov);

/* Copy table k as float vertex values [n2][n1][n0], read back from its cell
 * records: vertex i is the corner of cell min(i, n-2) whose value is the sum of
 * the cell's stored coefficients (in double, rounded once). With FP32 records
 * that is within a few float roundings of the value the table was built from.
 * GICP model: the voxel records, 12 floats per voxel [n2][n1][n0]: mean (3),
 * 1 or 0 (voxel holds points), covariance xx xy xz yy yz zz, 0, 0. */
int gmcs_get_table(gmcs_ctx* ctx, int k, float* vals);

/* A counter of the context's state: every call that can change the particles'
 * current or keyframe poses, the neighbour sets or the keyframes (gmcs_init_particles,
 * gmcs_add_keyframe, gmcs_step, gmcs_predict, gmcs_select, gmcs_move,
 * gmcs_set_kf_poses, gmcs_load, a served frame) increases it. A caller that keeps
 * results derived from that state (the autograd wrapper's saved forward) compares
 * it to detect a change. */
int gmcs_state_version(gmcs_ctx* ctx, uint64_t* version);

/* Copy the stored trilinear coefficients of cells [c0, c0 + n) of field table k
 * (cells numbered x fastest, (n0-1) x (n1-1) x (n2-1) of them): 8 floats per cell,
 * c0..c7 of L = c0 + c1 x + c2 y + c3 z + c4 xy + c5 xz + c6 yz + c7 xyz in the
 * in-cell fraction (x, y, z) in [0, 1)^3, exactly the values the lookups use
 * (16-bit records decoded). coef: n x 8 floats, host or device.
 * Errors: GMCS_E_INVALID for a GICP map or a range past the last cell. */
int gmcs_get_records(gmcs_ctx* ctx, int k, uint64_t c0, uint64_t n, float* coef);
/* Current sizes. Any pointer may be NULL. */
int gmcs_get_sizes(gmcs_ctx* ctx, int* P, int* K, uint32_t* frame);

/* Per-kernel CUDA-event timing (on the context stream) on/off; counters. */
int gmcs_set_profiling(gmcs_ctx* ctx, int on);
int gmcs_get_stats(gmcs_ctx* ctx, gmcs_stats* out);
int gmcs_reset_stats(gmcs_ctx* ctx);

/* Bytes of device memory the context holds (state, scratch and tables). */
int gmcs_device_bytes(gmcs_ctx* ctx, uint64_t* bytes);

/* ---- serving: continuous batching of frames from many sessions
 *
 * A server holds filter sessions whose state stays on the device (each is a
 * gmcs_ctx created with the server's config, its own seed, and capacities given
 * at open). Frames submitted to any session are queued; the server repeatedly
 * takes, for up to 32 sessions that have a queued frame and none on the GPU,
 * their oldest frames and runs all of them as one tick: a CUDA graph (captured
 * once at creation) that uploads the tick's argument records and replays one
 * persistent launch per kernel of the frame, each walking a work list over the
 * sessions' blocks. Two ticks can be in flight on disjoint sessions (two
 * streams), so frames arriving during a tick start without waiting for it.
 * Every session's frame is computed exactly as gmcs_step computes it (same
 * kernels, same block decomposition), so its result does not depend on which
 * other sessions share its ticks.
 */
typedef struct gmcs_server gmcs_server;

typedef struct {
    uint64_t frames;              /* completed frames */
    uint64_t ticks;               /* graph launches */
    int sessions;                 /* open sessions */
    int pad;
    uint64_t used_bytes, budget_bytes;
    double evals;                 /* particle x point likelihood+gradient evaluations (P * N * steps) */
    double span_s;                /* first submission to last completion */
    double busy_s;                /* time with at least one tick on the GPU (graph start to end) */
    double mean_sessions_per_tick;
    double latency_p50_s, latency_p99_s, latency_max_s, latency_mean_s;   /* submission to completion */
} gmcs_server_stats;

/* cfg: shared by all sessions (k_nb must be 3); budget_bytes: device memory the
 * sessions may hold; max_sessions: open-session limit. Errors: GMCS_E_INVALID,
 * GMCS_E_OOM, GMCS_E_CUDA. */
int gmcs_server_create(const gmcs_config* cfg, uint64_t budget_bytes, int max_sessions, gmcs_server** out);
int gmcs_server_destroy(gmcs_server* srv);
/* Run the scheduler on a background thread (start) or not (stop); without it,
 * gmcs_server_pump / gmcs_server_poll / gmcs_server_drain advance the work. */
int gmcs_server_start(gmcs_server* srv);
int gmcs_server_stop(gmcs_server* srv);
int gmcs_server_pump(gmcs_server* srv);
/* Ticks allowed on the GPU at once: 2 (default; a tick starts while another runs)
 * or 1 (one after another). */
int gmcs_server_set_inflight(gmcs_server* srv, int ticks);
/* Work cap of a tick, in evaluations (particles x points x cfg.steps): a tick
 * takes the oldest pending frame, then further frames, oldest first, only while
 * its total stays within max_evals, so that a frame is not held until a much
 * larger one in the same tick finishes; the rest go to the next tick, which runs
 * beside it. 0 lifts the cap (every ready session joins the tick). Default 4e8
 * (about 4 ms of lookups). Errors: GMCS_E_INVALID. */
int gmcs_server_set_tick_work(gmcs_server* srv, double max_evals);
/* Admission: open a session if its context (capacities) plus table_bytes fit the
 * remaining budget, else GMCS_E_BUDGET (retry after another session closes).
 * Then fill it through its context (gmcs_server_context: gmcs_init_particles,
 * gmcs_add_keyframe, gmcs_set_path; at least 3 keyframes) and call
 * gmcs_server_ready, which charges the session's actual device bytes. The
 * context may be read (gmcs_get_particles, ...) only while the session has no
 * frame in flight (after gmcs_server_poll reports its frames or after drain). */
int gmcs_server_open(gmcs_server* srv, int max_particles, int max_keyframes, int max_points, uint64_t table_bytes,
                     uint64_t seed, int* sid);
int gmcs_server_context(gmcs_server* srv, int sid, gmcs_ctx** ctx);
int gmcs_server_ready(gmcs_server* srv, int sid);
/* Queue one frame (scan: N x 3 host floats, copied into the session's pinned ring
 * before return; delta_T, cov as in gmcs_step). At most 64 frames per session may
 * be queued (GMCS_E_CAPACITY beyond). *ticket identifies the frame. */
int gmcs_server_submit(gmcs_server* srv, int sid, const float* scan, int N, const double delta_T[12],
                       const double cov[36], uint64_t* ticket);
/* GMCS_PENDING until the frame completes; then GMCS_OK (once) with its result and
 * latency (submission to completion, seconds). */
int gmcs_server_poll(gmcs_server* srv, uint64_t ticket, gmcs_step_out* out, double* latency_s);
/* Wait until every queued frame has completed. */
int gmcs_server_drain(gmcs_server* srv);
/* Close a session: queued frames are dropped (their tickets report GMCS_E_STATE),
 * a frame on the GPU is waited for, and the session's memory returns to the budget. */
int gmcs_server_close(gmcs_server* srv, int sid);
int gmcs_server_get_stats(gmcs_server* srv, gmcs_server_stats* out);
int gmcs_server_reset_stats(gmcs_server* srv);

const char* gmcs_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* GMCS_H */
