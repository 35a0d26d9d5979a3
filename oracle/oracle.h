/*
 * oracle.h -- plain, slow FP64 reference of the per-frame particle update of
 * "Range-based 6-DoF Monte Carlo SLAM with Gradient-guided Particle Filter on
 * GPU" (Nakao et al., arXiv 2504.18056).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline / reference arm may load this library. The CUDA product path
 * shares no code with it and never calls it.
 *
 * Conventions
 *   pose    12 doubles, row-major 3x4 [R | t]; x_world = R p + t.
 *   xi      se(3) tangent vector [omega(3); v(3)], rotation first; a pose is
 *           perturbed on the right, T exp(xi), as in Eq. 1, Eq. 7 and Eq. 10.
 *   grid    lattice vertices at origin + h*(ix, iy, iz), 0 <= i? < n?, values
 *           stored [iz][iy][ix] (x fastest).
 *   scan    float triples (the sensor's own precision) widened to double.
 *
 * Parity status of each function is stated beside it; the pins live in the
 * test-suite (tests/test_oracle_*.py).
 */
#ifndef GMCS_ORACLE_H
#define GMCS_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double origin[3];
    double h;
    int n[3];
    int coef;   /* 0: vals holds vertex values [n2][n1][n0]; 1: vals holds per-cell
                   trilinear coefficients c0..c7 [n2-1][n1-1][n0-1][8] (below) */
} ora_grid;

/* ---- SE(3) (closed forms: Rodrigues + left Jacobian; Taylor below 1e-4 rad) */
void ora_pose_mul(const double A[12], const double B[12], double C[12]);
void ora_pose_inv(const double A[12], double B[12]);
void ora_se3_exp(const double xi[6], double T[12]);
void ora_se3_log(const double T[12], double xi[6]);
/* Right Jacobian: exp(xi + d) = exp(xi) exp(Jr d) to first order (6 x 6, row-major). */
void ora_se3_jr(const double xi[6], double J[36]);

/* ---- Philox4x32-10 (Salmon et al., SC'11) and the draws built on it */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Six standard normals for particle i at frame t: Box-Muller on uniforms
 * (k + 1/2) 2^-23 built from the top 23 bits of two Philox blocks with
 * counters (i, t, 0|1, 'NORM'). */
void ora_normal6(uint64_t seed, uint32_t i, uint32_t t, double z[6]);
/* Systematic-resampling offset u in [0,1) for frame t (53-bit uniform). */
double ora_systematic_u(uint64_t seed, uint32_t t);

/* ---- likelihood tables (Sec. III-C1 replaced by a voxel likelihood field) */
/* vals[v] = exp(-d^2 / 2 sigma^2) if d <= r_t else 0, d = distance from vertex v
 * to the nearest point. Points are visited one by one and every vertex within
 * r_t of the point is relaxed. */
void ora_build_table(const float* pts, int n, const ora_grid* g, double sigma, double r_t, double* vals);
/* Same value, with the minimum taken over all points for every vertex. */
void ora_build_table_brute(const float* pts, int n, const ora_grid* g, double sigma, double r_t, double* vals);
/* Round to bfloat16 (dtype 1) or IEEE half (dtype 2), nearest-even, widened back. */
void ora_quantize(const double* in, size_t n, int dtype, double* out);

/* Trilinear value and gradient (w.r.t. lattice coordinate u) of cell c at u.
 * Vertex tables: the interpolation of the cell's 8 corner values. Coefficient
 * tables (g->coef): with f = u - c, the polynomial
 *   L = c0 + c1 fx + c2 fy + c3 fz + c4 fx fy + c5 fx fz + c6 fy fz + c7 fx fy fz
 * of the cell's stored coefficients and its derivative.
 * Returns 1 if c is inside the table, else 0 (value and gradient set to 0). */
int ora_cell_eval(const double* vals, const ora_grid* g, const int c[3], const double u[3],
                  double* L, double dLdu[3]);

/* ---- per-particle evaluation (form of Eq. 2-3 and Eq. 6 on the voxel field) */
typedef struct {
    double eps;          /* likelihood floor: l = log(L + eps) */
    double face_delta;   /* cells; lookups closer than this to a cell face add slack */
} ora_eval_params;

/*
 * One particle: current pose Tt, n_nb neighbour keyframes with this particle's
 * keyframe poses Tk[s] (12 each), their tables and grids, N scan points.
 * Outputs (any may be NULL):
 *   ll      sum over points and neighbours of log(L + eps)
 *   g       d ll / d xi at xi = 0 for Tt exp(xi)  (6)
 *   mom     [W, Sx, Sy, Sz, Qxx, Qxy, Qxz, Qyy, Qyz, Qzz] with weight w = L/(L+eps):
 *           W = sum w, S = sum w p, Q = sum w p p^T (p in the sensor frame)
 *   slack   sum over lookups within face_delta of a face of the norm of the
 *           change in that lookup's d l / d xi when the neighbouring cell is used
 *   gabs    sum over lookups of the norm of that lookup's d l / d xi
 *   cells   if frozen == 0 and cells != NULL: the cell used per (s, j) is written
 *           (3 ints, -1 -1 -1 when outside); if frozen == 1 those cells are used
 *           instead of floor(u), their polynomial extended past the faces.
 */
void ora_eval_particle(const double Tt[12], int n_nb, const double* Tk, const double* const* tables,
                       const ora_grid* grids, const float* scan, int N, const ora_eval_params* prm,
                       double* ll, double g[6], double mom[10], double* slack, double* gabs,
                       int* cells, int frozen);

/* Gauss-Newton matrix from the moments (Eq. 6 on the field, sigma^-2 sum w B^T B). */
void ora_h_from_moments(const double mom[10], double sigma, double H[36]);
/* Same matrix, summed explicitly from points and weights. */
void ora_h_explicit(const float* scan, int N, const double* w, double sigma, double H[36]);

typedef struct {
    double sigma;       /* field width (m) */
    double lambda;      /* Levenberg-Marquardt factor on diag(H) */
    double theta_max;   /* rad, clamp on |psi_omega| */
    double t_max;       /* m, clamp on |psi_v| */
    double w_min;       /* no move when W < w_min */
} ora_move_params;

/* Eq. 5-7: psi = (H + lambda diag H)^-1 g, clamped, Tout = Tt exp(psi). */
void ora_move(const double Tt[12], const double g[6], const double mom[10], const ora_move_params* mp,
              double Tout[12], double psi[6]);

/* Eq. 5-7 with a given Gauss-Newton matrix: psi = (H + lambda diag H)^-1 b,
 * clamped, Tout = Tt exp(psi) (no move when the damped H is not positive definite). */
void ora_move_h(const double Tt[12], const double b[6], const double H[36], const ora_move_params* mp,
                double Tout[12], double psi[6]);

/* ---- GICP distribution-to-distribution likelihood (Eq. 2-6) on voxel maps.
 * A map is a dense lattice of n[0] x n[1] x n[2] voxels of edge h from origin
 * (voxel (ix,iy,iz) covers origin + h [ix, ix+1) x [iy, iy+1) x [iz, iz+1)),
 * 10 doubles each, x fastest: mean (3), point count (1), covariance (6: xx xy
 * xz yy yz zz); a voxel with count 0 has no distribution. scov: N x 6 scan point
 * covariances. Every (neighbour s, scan point mu_j) pair adds one term. When the
 * transformed point lies in a non-empty voxel,
 *   e = mu' - kT_t mu_j, Omega = (Sigma' + R Sigma_j R^T)^-1,  d2 = e^T Omega e,
 * and d2 < tau (an inlier):
 *   ll += -d2,  J = d(kT_t exp(xi) mu_j)/d xi = R [-[mu_j]x | I],
 *   b += J^T Omega e,  H += J^T Omega J;
 * otherwise (no voxel, empty voxel, or d2 >= tau) ll += -tau and nothing else
 * (the step psi = H^-1 b ascends ll). slack[3]: summed over lookups whose
 * coordinate lies within face_delta voxels of a face, |change| of the term's
 * ll, b (norm) and H (Frobenius) when the voxel across that face is used; and
 * over lookups with |d2 - tau| < gate_delta tau, |d2 - tau| and the norms of
 * the term's b and H (the cap decides them at the rounding level).
 * nvalid: inlier lookups. Any output may be NULL. */
void ora_gicp_eval_particle(const double Tt[12], int n_nb, const double* Tk, const double* const* maps,
                            const ora_grid* grids, const float* scan, const double* scov, int N, double tau,
                            double face_delta, double gate_delta, double* ll, double b[6], double H[36],
                            double slack[3], int* nvalid);

/* ---- keyframe pose propagation, Eq. 8-10: with o the oldest (lowest-index)
 * neighbour keyframe, every keyframe k > o moves by T_k exp(r_k psi),
 * r_k = (D_k - D_o) / (Dt - D_o), D the odometry path length at each keyframe
 * and Dt at the current frame (Eq. 9 summed along the odometry trajectory).
 * kf_i: this particle's K keyframe poses (K x 12, in/out). No change when
 * Dt - D_o <= 0. */
void ora_propagate(const double psi[6], const int* nbr, int k_nb, int K, const double* D, double Dt, double* kf_i);
/* Loop condition of Sec. III-C2: 1 if the particle's oldest neighbour keyframe is
 * not among the `recent` newest keyframes (recent = 0: always 1). */
int ora_loop(const int* nbr, int k_nb, int K, int recent);

/* ---- neighbour keyframes: the k_nb smallest |t_k - t_t| (ties -> lower k).
 * The squared distances are formed in float with a fixed order of operations,
 * the precision the GPU takes this decision in. */
void ora_select_nbrs(const double Tt[12], const double* kf_t /* K x 3 */, int K, int k_nb, int* idx);

/* ---- prediction, Eq. 1: Tout = T dT exp(L z), L = chol(cov) (lower). */
void ora_predict(const double T[12], const double dT[12], const double cov[36], const double z[6],
                 double Tout[12]);

/* ---- importance weighting, Eq. 11, normalised by log-sum-exp. */
void ora_lse(const double* logw, const double* ll, int P, double* logw_out, double* w,
             double* M, double* logS, int* argmax, double* ess);

/* ---- systematic resampling on weights quantised to the 2^-52 grid. */
void ora_resample(const double* w, int P, double u, int* anc);

/* ---- dead-particle pruning (Sec. III-F) as a resampling policy.
 * Particle i (i != argmax, the largest weight, which always survives) is dead
 * when its normalised weight is not >= prune_w (the posterior criterion; NaN is
 * dead), or, when ll is given and ll_cut > -inf, when ll_i - max_j ll_j is not
 * >= ll_cut (the likelihood criterion, relative to the frame's best particle;
 * ll_cut = log of the likelihood ratio). The D dead slots, taken in index order
 * r = 0..D-1, are refilled by systematic sampling over the survivors' weights
 * quantised as q_i = rint(w_i 2^52) (q = 0 for dead slots), C_i = q_0+...+q_i,
 * S = C_{P-1}:
 *     tau_r = min(((u + r) / D) * S, S - 1),   a_r = min{ i : C_i > tau_r }.
 * A survivor a drawn c_a times shares its weight with its copies: the survivor
 * and each copy get x_a - log1p(c_a), x the normalised log-weights; survivors
 * with no copy keep x. anc: i for survivors, a_r for the r-th dead slot.
 * Returns D. */
int ora_prune(const double* x, const double* w, const double* ll, int P, int argmax, double prune_w,
              double ll_cut, double u, int* anc, double* logw_out);

/* ---- keyframe insertion by overlap (Sec. III-E).
 * Occupancy lattice of a cloud at voxel edge h: per axis lo = floor(min / h) - 1,
 * hi = floor(max / h) + 1 (min, max over the points, FP64), origin = lo h,
 * n = hi - lo + 1 voxels, so every point lies at least one voxel inside.
 * ora_occupancy_grid fills g; ora_overlap returns the fraction of the n scan
 * points that, moved by T_rel (the current frame in the last keyframe's frame,
 * from odometry), fall into a voxel of g holding at least one keyframe point.
 * Every product and sum is rounded separately (FP64), the voxel is
 * floor((x - origin) / h). */
void ora_occupancy_grid(const float* pts, int n, double h, ora_grid* g);
double ora_overlap(const float* kf_pts, int nk, const ora_grid* g, const float* scan, int n, const double T_rel[12]);

/* ---- whole frame over a particle set (the hot path, all steps in order). */
typedef struct {
    double sigma, eps, lambda, theta_max, t_max, w_min, face_delta;
    int k_nb, steps;
    int resample;        /* 0 always, 1 when ESS < P/2, 2 never, 3 prune dead particles */
    int propagate;       /* 1: keyframe pose propagation after every move (Eq. 8-10) */
    int loop_recent;     /* > 0: move only particles whose oldest neighbour is not among the newest loop_recent */
    int model;           /* 0 voxel likelihood field, 1 GICP (tables are voxel maps, scov required) */
    double gicp_tau;     /* model 1: cap of a term's e^T Omega e (outliers and points without a voxel) */
    double prune_w;      /* resample 3: posterior threshold */
    double ll_cut;       /* resample 3: log likelihood-ratio threshold (-inf: off) */
    uint64_t seed;
} ora_step_params;

typedef struct {
    double estimate[12];
    double ess, max_w;
    int argmax, resampled;
    int pruned, pad;
} ora_step_out;

/*
 * tables    K likelihood tables (model 0) or K GICP voxel maps (model 1), with grids
 * scov      model 1: N x 6 scan point covariances (else may be NULL)
 * poses     P x 12 current poses (in/out)
 * kf_poses  K x P x 12 per-particle keyframe poses (in/out; gathered on resample)
 * logw      P log-weights (in/out)
 * frame     frame counter for the counter-based draws
 * z         optional P x 6 standard normals (NULL -> Philox draws)
 * u         optional systematic offset (NULL -> Philox draw)
 * kf_path   K odometry path lengths of the keyframes, path_now that of this frame
 *           (used when sp->propagate; may be NULL otherwise)
 * ll_out, w_out, anc_out, nbr_out   optional diagnostics (P, P, P, P x k_nb)
 */
void ora_step(int P, int K, double* poses, double* kf_poses, double* logw,
              const double* const* tables, const ora_grid* grids,
              const float* scan, const double* scov, int N, const double dT[12], const double cov[36],
              uint32_t frame, const double* z, const double* u, const ora_step_params* sp,
              const double* kf_path, double path_now,
              ora_step_out* out, double* ll_out, double* w_out, int* anc_out, int* nbr_out);

#ifdef __cplusplus
}
#endif
#endif
