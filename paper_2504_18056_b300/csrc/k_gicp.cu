// k_gicp.cu -- the GICP distribution-to-distribution likelihood (Eq. 2-6).
//
// Each point carries a Gaussian: its k nearest points of the same cloud give a
// covariance, plane-regularised as in generalised ICP (eigenvalues replaced by
// (eps, 1, 1), so only the direction of the smallest eigenvalue -- the surface
// normal n -- survives: Sigma = I - (1 - eps) n n^T). A keyframe is a dense
// voxel map: per voxel the mean of its points and the mean of their
// covariances (the voxel-based correspondence of Sec. III-C1: a transformed
// scan point corresponds to the voxel it falls in).
//
// The lookup pass works in each neighbour keyframe's frame. With kT_t = [R | t],
// the rotated point x' = R mu and x = x' + t,
//   e = mu' - x,  Omega = (Sigma' + R Sigma_j R^T)^-1,  d2 = e^T Omega e  (Eq. 3-4),
// where the scan covariance is plane-regularised, Sigma_j = I - (1 - eps) n n^T,
// so R Sigma_j R^T = I - (1 - eps) m m^T with m = R n (a rank-one update, no
// 3x3 rotation of a matrix per lookup). The right perturbation of the current
// pose moves x by R (omega x mu + v) = [-[x']x | I] diag(R, R) xi (R [mu]x = [R mu]x R),
// so the Gauss-Newton terms of Eq. 5-6 are accumulated per keyframe as
//   b_k += [x' x q; q],  q = Omega e,
//   H_k += [[-[x']x Omega [x']x, [x']x Omega], [.., Omega]]
// and rotated once per (particle, keyframe): b += diag(R, R)^T b_k,
// H += diag(R, R)^T H_k diag(R, R).
// Every (point, neighbour) pair adds one term to the log-likelihood: -d2 for an
// inlier (d2 < tau), -tau when the voxel is empty, outside the map, or d2 >= tau.
#include <math.h>

#include "kernels.h"
#include "pass.cuh"

namespace gmcs {

// ------------------------------------------------------------------ covariances

// One Jacobi rotation zeroing a_pq of a symmetric 3x3 matrix (a_rp, a_rq the
// entries coupling the third index r), accumulated into the eigenvector
// columns vp, vq (Golub & Van Loan, the symmetric Schur decomposition of the
// 2x2 block). Scalars, so that everything stays in registers.
__device__ __forceinline__ void jacobi_rot(double& app, double& aqq, double& apq, double& arp, double& arq,
                                           double& vp0, double& vp1, double& vp2, double& vq0, double& vq1,
                                           double& vq2) {
    if (apq == 0.0) return;
    const double theta = (aqq - app) / (2.0 * apq);
    const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
    const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
    const double rp = arp, rq = arq;
    arp = c * rp - s * rq;
    arq = s * rp + c * rq;
    app -= t * apq;
    aqq += t * apq;
    apq = 0.0;
    double x = vp0, y = vq0;
    vp0 = c * x - s * y; vq0 = s * x + c * y;
    x = vp1; y = vq1;
    vp1 = c * x - s * y; vq1 = s * x + c * y;
    x = vp2; y = vq2;
    vp2 = c * x - s * y; vq2 = s * x + c * y;
}

// Unit eigenvector of the smallest eigenvalue (lowest index on ties) of the
// symmetric matrix [[a00 a01 a02] [a01 a11 a12] [a02 a12 a22]] by cyclic Jacobi.
__device__ __forceinline__ void sym3_min_eigvec(double a00, double a01, double a02, double a11, double a12,
                                                double a22, double n[3]) {
    // V columns: (v00 v10 v20), (v01 v11 v21), (v02 v12 v22)
    double v00 = 1.0, v01 = 0.0, v02 = 0.0, v10 = 0.0, v11 = 1.0, v12 = 0.0, v20 = 0.0, v21 = 0.0, v22 = 1.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        const double off = a01 * a01 + a02 * a02 + a12 * a12;
        const double dia = a00 * a00 + a11 * a11 + a22 * a22;
        if (!(off > 1e-36 * dia)) break;
        jacobi_rot(a00, a11, a01, a02, a12, v00, v10, v20, v01, v11, v21);   // (p,q,r) = (0,1,2)
        jacobi_rot(a00, a22, a02, a01, a12, v00, v10, v20, v02, v12, v22);   // (0,2,1)
        jacobi_rot(a11, a22, a12, a01, a02, v01, v11, v21, v02, v12, v22);   // (1,2,0)
    }
    int m = 0;
    double lm = a00;
    if (a11 < lm) { m = 1; lm = a11; }
    if (a22 < lm) m = 2;
    n[0] = m == 0 ? v00 : (m == 1 ? v01 : v02);
    n[1] = m == 0 ? v10 : (m == 1 ? v11 : v12);
    n[2] = m == 0 ? v20 : (m == 1 ? v21 : v22);
}

// One warp per point. The cloud streams through shared memory in tiles; lane l
// takes the candidates of index l mod 32 and keeps its k best sorted by squared
// distance, formed in float as ((dx*dx + dy*dy) + dz*dz) with separate
// round-to-nearest operations (a candidate enters only when strictly closer, so
// equal distances stay in index order). The warp then merges the 32 lists by k
// rounds of a shuffle arg-min on (distance, index): the k nearest points of the
// cloud with ties to the lower index. Lane 0 takes their FP64 covariance (1/k)
// and the plane regularisation.
template <int KM>
__device__ __forceinline__ void knn_cov_body(const KnnCovArgs& a, int vb) {
    constexpr int kTile = 1024;
    __shared__ float4 tile[kTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = vb * (blockDim.x >> 5) + warp;
    const bool act = i < a.n;
    const float4 p = act ? a.pts[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int k = min(a.k, a.n);
    float bd[KM];
    int bi[KM];
#pragma unroll
    for (int s = 0; s < KM; ++s) { bd[s] = __int_as_float(0x7f800000); bi[s] = 0x7fffffff; }
    float worst = __int_as_float(0x7f800000);
    for (int base = 0; base < a.n; base += kTile) {
        const int m = min(kTile, a.n - base);
        for (int t = threadIdx.x; t < m; t += blockDim.x) tile[t] = a.pts[base + t];
        __syncthreads();
        if (act) {
            for (int t = lane; t < m; t += 32) {
                const float4 q = tile[t];
                const float dx = __fsub_rn(q.x, p.x), dy = __fsub_rn(q.y, p.y), dz = __fsub_rn(q.z, p.z);
                const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                if (d2 < worst) {
                    bool done = false;
#pragma unroll
                    for (int s = KM - 1; s >= 0; --s) {
                        if (s < k && !done) {
                            if (s > 0 && bd[s - 1] > d2) {
                                bd[s] = bd[s - 1];
                                bi[s] = bi[s - 1];
                            } else {
                                bd[s] = d2;
                                bi[s] = base + t;
                                done = true;
                            }
                        }
                    }
#pragma unroll
                    for (int s = 0; s < KM; ++s)
                        if (s == k - 1) worst = bd[s];
                }
            }
        }
        __syncthreads();
    }
    if (!act || k <= 0) return;                 // warp-uniform: one point per warp
    int nb[KM];
#pragma unroll
    for (int r = 0; r < KM; ++r) {
        nb[r] = 0;
        if (r < k) {
            float d = bd[0];
            int j = bi[0];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float od = __shfl_xor_sync(0xffffffffu, d, off);
                const int oj = __shfl_xor_sync(0xffffffffu, j, off);
                if (od < d || (od == d && oj < j)) { d = od; j = oj; }
            }
            nb[r] = j;
            if (bi[0] == j) {                   // the owner pops its head
#pragma unroll
                for (int s = 0; s < KM - 1; ++s) { bd[s] = bd[s + 1]; bi[s] = bi[s + 1]; }
                bd[KM - 1] = __int_as_float(0x7f800000);
                bi[KM - 1] = 0x7fffffff;
            }
        }
    }
    if (lane != 0) return;
    double mx = 0.0, my = 0.0, mz = 0.0;
#pragma unroll
    for (int s = 0; s < KM; ++s) {
        if (s < k) {
            const float4 q = a.pts[nb[s]];
            mx += (double)q.x;
            my += (double)q.y;
            mz += (double)q.z;
        }
    }
    mx /= (double)k;
    my /= (double)k;
    mz /= (double)k;
    double c00 = 0.0, c01 = 0.0, c02 = 0.0, c11 = 0.0, c12 = 0.0, c22 = 0.0;
#pragma unroll
    for (int s = 0; s < KM; ++s) {
        if (s < k) {
            const float4 q = a.pts[nb[s]];
            const double dx = (double)q.x - mx, dy = (double)q.y - my, dz = (double)q.z - mz;
            c00 += dx * dx; c01 += dx * dy; c02 += dx * dz;
            c11 += dy * dy; c12 += dy * dz; c22 += dz * dz;
        }
    }
    const double ik = 1.0 / (double)k;
    double n[3];
    sym3_min_eigvec(c00 * ik, c01 * ik, c02 * ik, c11 * ik, c12 * ik, c22 * ik, n);
    const double w = 1.0 - a.eps;
    const double sxx = 1.0 - w * n[0] * n[0], sxy = -w * n[0] * n[1], sxz = -w * n[0] * n[2];
    const double syy = 1.0 - w * n[1] * n[1], syz = -w * n[1] * n[2], szz = 1.0 - w * n[2] * n[2];
    if (a.cov64) {
        double* o = a.cov64 + 6 * (size_t)i;
        o[0] = sxx; o[1] = sxy; o[2] = sxz; o[3] = syy; o[4] = syz; o[5] = szz;
    }
    if (a.nrm32) a.nrm32[i] = make_float4((float)n[0], (float)n[1], (float)n[2], 0.f);
}

template <int KM>
__global__ void __launch_bounds__(128) k_knn_cov(KnnCovArgs a) {
    knn_cov_body<KM>(a, blockIdx.x);
}

template <int KM>
__global__ void __launch_bounds__(128) k_knn_cov_b(const BatchList<KnnCovArgs>* L) {
    GMCS_BATCH_LOOP(L, const KnnCovArgs a = L->args[s]; knn_cov_body<KM>(a, vb));
}

// ------------------------------------------------------------------ voxel maps

__global__ void k_voxel_accum(VoxelArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float4 p = a.pts[i];
    const double px = (double)p.x, py = (double)p.y, pz = (double)p.z;
    const double fx = floor((px - a.ox) / a.h), fy = floor((py - a.oy) / a.h), fz = floor((pz - a.oz) / a.h);
    if (!(fx >= 0.0 && fx < (double)a.nx && fy >= 0.0 && fy < (double)a.ny && fz >= 0.0 && fz < (double)a.nz))
        return;
    const size_t v = ((size_t)fz * a.ny + (size_t)fy) * a.nx + (size_t)fx;
    double* s = a.sums + 10 * v;
    atomicAdd(s + 0, px);
    atomicAdd(s + 1, py);
    atomicAdd(s + 2, pz);
    atomicAdd(s + 3, 1.0);
    const double* c = a.cov + 6 * (size_t)i;
#pragma unroll
    for (int e = 0; e < 6; ++e) atomicAdd(s + 4 + e, c[e]);
}

__global__ void k_voxel_final(VoxelArgs a) {
    const size_t nv = (size_t)a.nx * a.ny * a.nz;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nv; v += (size_t)gridDim.x * blockDim.x) {
        const double* s = a.sums + 10 * v;
        const double cnt = s[3];
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
        if (cnt > 0.0) {
            r0 = make_float4((float)(s[0] / cnt), (float)(s[1] / cnt), (float)(s[2] / cnt), 1.f);
            r1 = make_float4((float)(s[4] / cnt), (float)(s[5] / cnt), (float)(s[6] / cnt), (float)(s[7] / cnt));
            r2 = make_float4((float)(s[8] / cnt), (float)(s[9] / cnt), 0.f, 0.f);
        }
        a.rec[3 * v] = r0;
        a.rec[3 * v + 1] = r1;
        a.rec[3 * v + 2] = r2;
    }
}

// ------------------------------------------------------------------ the lookup pass

// R^T A R for a symmetric A given by its upper triangle (a00 a01 a02 a11 a12 a22),
// written back in place.
__device__ __forceinline__ void rot_sym(const float* R, float* u) {
    const float A[9] = {u[0], u[1], u[2], u[1], u[3], u[4], u[2], u[4], u[5]};
    float M[9];   // A R
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[r * 3 + c] = fmaf(A[r * 3], R[c], fmaf(A[r * 3 + 1], R[3 + c], A[r * 3 + 2] * R[6 + c]));
    int e = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) u[e++] = fmaf(R[r], M[c], fmaf(R[3 + r], M[3 + c], R[6 + r] * M[6 + c]));
}

// R^T A R for a general 3x3 A (row-major), in place.
__device__ __forceinline__ void rot_gen(const float* R, float* A) {
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[r * 3 + c] = fmaf(A[r * 3], R[c], fmaf(A[r * 3 + 1], R[3 + c], A[r * 3 + 2] * R[6 + c]));
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) A[r * 3 + c] = fmaf(R[r], M[c], fmaf(R[3 + r], M[3 + c], R[6 + r] * M[6 + c]));
}

// the gradient pass loads each point and normal one point ahead (1)
#ifndef GMCS_GICP_PAHEAD
#define GMCS_GICP_PAHEAD 1
#endif
// CTAs per SM the register allocation is sized for (1: no bound; the gradient pass
// takes 124 registers, 4 CTAs per SM; bounded to 5 CTAs it fits 96 registers but is
// slower with the look-ahead, 3.93 -> 4.05 ms)
#ifndef GMCS_GICP_MINBLOCKS
#define GMCS_GICP_MINBLOCKS 1
#endif
// the value pass: the point loaded when it is used (0); one point ahead it takes
// 2.49 -> 2.60 ms at 5 CTAs per SM, 2.54 / 2.48 ms bounded to 6 / 7)
#ifndef GMCS_GICP_PAHEAD_V
#define GMCS_GICP_PAHEAD_V 0
#endif
// value pass CTAs per SM: 8 fits 63 registers (2.49 -> 2.37 ms against 76
// registers and 6 CTAs unbounded; 9 spills)
#ifndef GMCS_GICP_MINBLOCKS_V
#define GMCS_GICP_MINBLOCKS_V 8
#endif
template <bool GRAD>
constexpr int gicp_minblocks() { return GRAD ? GMCS_GICP_MINBLOCKS : GMCS_GICP_MINBLOCKS_V; }
// the persistent (served) passes: their batch loop costs registers; the gradient
// pass takes 167 unbounded (3 CTAs per SM), 127 at 4; the value pass 94 (5 CTAs
// per SM), and spills if bounded to 6
#ifndef GMCS_GICP_B_MINBLOCKS
#define GMCS_GICP_B_MINBLOCKS 4
#endif
#ifndef GMCS_GICP_B_MINBLOCKS_V
#define GMCS_GICP_B_MINBLOCKS_V 1
#endif
template <bool GRAD>
constexpr int gicp_b_minblocks() { return GRAD ? GMCS_GICP_B_MINBLOCKS : GMCS_GICP_B_MINBLOCKS_V; }

template <bool GRAD>
__device__ __forceinline__ void gicp_body(const PassArgs& a, int vb) {
    constexpr int NACC = GRAD ? kAccGicp : 1;
    const WarpWork ww = warp_work(a, vb);
    const int i = ww.i, j0 = ww.j0, j1 = ww.j1;
    float acc[NACC];
#pragma unroll
    for (int e = 0; e < NACC; ++e) acc[e] = 0.f;

    // the particle's b and H totals live in a shared-memory column while the point
    // loops run (each slot adds its rotated sums once), not in 28 registers: 126 -> 96
    // registers, 5 CTAs per SM instead of 4 (gradient pass 4.61 -> 4.27 ms)
    __shared__ float sacc[GRAD ? kAccGicp : 1][kPassThreads];
    if (i < a.P && j0 < j1) {
        if constexpr (GRAD)
            for (int e = 1; e < kAccGicp; ++e) sacc[e][threadIdx.x] = 0.f;
        float Tt[12];
        load_pose(a.pose, a.ld, i, Tt);
        const float tau = a.tau, wn = a.cov_w, ce = a.cov_eps;
        float lsum = 0.f;
        for (int s = 0; s < a.k_nb; ++s) {
            const int k = a.nbr[(size_t)s * a.ld + i];
            if (k < 0) continue;
            const TableDesc td = a.tables[k];
            float Tk[12], rel[12];
            load_pose(a.kf + (size_t)k * kPoseC * a.ld, a.ld, i, Tk);
            pose_rel(Tk, Tt, rel);
            const float R00 = rel[0], R01 = rel[1], R02 = rel[2], t0 = rel[3];
            const float R10 = rel[4], R11 = rel[5], R12 = rel[6], t1 = rel[7];
            const float R20 = rel[8], R21 = rel[9], R22 = rel[10], t2 = rel[11];
            const float4* __restrict__ recs = reinterpret_cast<const float4*>(td.cells);
            const uint32_t ncx = (uint32_t)td.ncx, ncy = (uint32_t)td.ncy, ncz = (uint32_t)td.ncz;
            float bk[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float hk[21];
#pragma unroll
            for (int e = 0; e < 21; ++e) hk[e] = 0.f;
            float nin = 0.f;
            // the point's normal is loaded with the point, not after the voxel test, off
            // the record load's dependency chain (4.69 -> 4.61 ms); the gradient pass loads
            // both one point ahead (gradient pass 4.50 -> 3.93 ms; the value pass loses,
            // 2.49 -> 2.60 ms)
            constexpr bool kAhead = GRAD ? GMCS_GICP_PAHEAD : GMCS_GICP_PAHEAD_V;
            float4 pn = make_float4(0.f, 0.f, 0.f, 0.f), nn = pn;
            if constexpr (kAhead) {
                pn = __ldg(a.scan + j0);
                nn = __ldg(a.scov + j0);
            }
            for (int j = j0; j < j1; ++j) {
                float4 p, nj;
                if constexpr (kAhead) {
                    p = pn;
                    nj = nn;
                    const int jn = j + 1 < j1 ? j + 1 : j;
                    pn = __ldg(a.scan + jn);
                    nn = __ldg(a.scov + jn);
                } else {
                    p = __ldg(a.scan + j);
                    nj = __ldg(a.scov + j);
                }
                const float r0 = fmaf(R00, p.x, fmaf(R01, p.y, R02 * p.z));
                const float r1 = fmaf(R10, p.x, fmaf(R11, p.y, R12 * p.z));
                const float r2 = fmaf(R20, p.x, fmaf(R21, p.y, R22 * p.z));
                const float x0 = r0 + t0, x1 = r1 + t1, x2 = r2 + t2;
                const int cx = (int)floorf((x0 - td.ox) * td.inv_h);
                const int cy = (int)floorf((x1 - td.oy) * td.inv_h);
                const int cz = (int)floorf((x2 - td.oz) * td.inv_h);
                const bool inside = ((uint32_t)cx < ncx) & ((uint32_t)cy < ncy) & ((uint32_t)cz < ncz);
                float4 mv = make_float4(0.f, 0.f, 0.f, 0.f), v0 = mv, v1 = mv;
                if (inside) {
                    const size_t idx = ((size_t)cz * ncy + (size_t)cy) * ncx + (size_t)cx;
                    mv = __ldg(recs + 3 * idx);
                    v0 = __ldg(recs + 3 * idx + 1);
                    v1 = __ldg(recs + 3 * idx + 2);
                }
                if (!(mv.w > 0.f)) {
                    lsum -= tau;
                    continue;
                }
                const float e0 = mv.x - x0, e1 = mv.y - x1, e2 = mv.z - x2;
                // C = Sigma' + eps m m^T + (I - m m^T), m = R n; the diagonal of I - m m^T is
                // taken as the sum of the other two squares (no cancellation in the thin direction)
                const float m0 = fmaf(R00, nj.x, fmaf(R01, nj.y, R02 * nj.z));
                const float m1 = fmaf(R10, nj.x, fmaf(R11, nj.y, R12 * nj.z));
                const float m2 = fmaf(R20, nj.x, fmaf(R21, nj.y, R22 * nj.z));
                const float s0 = m0 * m0, s1 = m1 * m1, s2 = m2 * m2;
                const float a00 = fmaf(ce, s0, v0.x + (s1 + s2));
                const float a11 = fmaf(ce, s1, v0.w + (s0 + s2));
                const float a22 = fmaf(ce, s2, v1.y + (s0 + s1));
                const float wm0 = wn * m0, wm1 = wn * m1;
                const float a01 = fmaf(-wm0, m1, v0.y), a02 = fmaf(-wm0, m2, v0.z), a12 = fmaf(-wm1, m2, v1.x);
                // Omega = C^-1 by cofactors
                const float i00 = fmaf(a11, a22, -a12 * a12);
                const float i01 = fmaf(a02, a12, -a01 * a22);
                const float i02 = fmaf(a01, a12, -a02 * a11);
                const float i11 = fmaf(a00, a22, -a02 * a02);
                const float i12 = fmaf(a01, a02, -a00 * a12);
                const float i22 = fmaf(a00, a11, -a01 * a01);
                const float det = fmaf(a00, i00, fmaf(a01, i01, a02 * i02));
                // C is positive definite (eigenvalues >= ~1e-3), det well inside the
                // range where the approximate reciprocal (2 ulp) holds; an IEEE division
                // costs the pass 1.2 % (gradient 4.22 -> 4.27 ms)
                const float rd = __fdividef(1.f, det);
                // d^2 = e^T adj(C) e / det, the same float expression in both passes, so
                // that the gradient pass and the value pass cap the same points; the value
                // pass never forms Omega (2.46 -> 2.38 ms), the gradient pass takes
                // q = Omega e = adj(C) e / det from the same products
                const float a0 = fmaf(i00, e0, fmaf(i01, e1, i02 * e2));
                const float a1 = fmaf(i01, e0, fmaf(i11, e1, i12 * e2));
                const float a2 = fmaf(i02, e0, fmaf(i12, e1, i22 * e2));
                const float d2 = fmaf(e0, a0, fmaf(e1, a1, e2 * a2)) * rd;
                float o00, o01, o02, o11, o12, o22, q0, q1, q2;
                if constexpr (GRAD) {
                    o00 = i00 * rd; o01 = i01 * rd; o02 = i02 * rd;
                    o11 = i11 * rd; o12 = i12 * rd; o22 = i22 * rd;
                    q0 = a0 * rd; q1 = a1 * rd; q2 = a2 * rd;
                }
                if (!(d2 < tau)) {
                    lsum -= tau;
                    continue;
                }
                lsum -= d2;
                if constexpr (GRAD) {
                    // b_k = [x' x q; q]
                    bk[0] += fmaf(r1, q2, -r2 * q1);
                    bk[1] += fmaf(r2, q0, -r0 * q2);
                    bk[2] += fmaf(r0, q1, -r1 * q0);
                    bk[3] += q0;
                    bk[4] += q1;
                    bk[5] += q2;
                    // K = [x']x Omega (rows: -x2 O1 + x1 O2, x2 O0 - x0 O2, -x1 O0 + x0 O1)
                    const float K00 = fmaf(-r2, o01, r1 * o02), K01 = fmaf(-r2, o11, r1 * o12),
                                K02 = fmaf(-r2, o12, r1 * o22);
                    const float K10 = fmaf(r2, o00, -r0 * o02), K11 = fmaf(r2, o01, -r0 * o12),
                                K12 = fmaf(r2, o02, -r0 * o22);
                    const float K20 = fmaf(-r1, o00, r0 * o01), K21 = fmaf(-r1, o01, r0 * o11),
                                K22 = fmaf(-r1, o02, r0 * o12);
                    // rotation block -K [x']x
                    hk[0] -= fmaf(K01, r2, -K02 * r1);
                    hk[1] -= fmaf(K02, r0, -K00 * r2);
                    hk[2] -= fmaf(K00, r1, -K01 * r0);
                    hk[6] -= fmaf(K12, r0, -K10 * r2);
                    hk[7] -= fmaf(K10, r1, -K11 * r0);
                    hk[11] -= fmaf(K20, r1, -K21 * r0);
                    // cross block K
                    hk[3] += K00; hk[4] += K01; hk[5] += K02;
                    hk[8] += K10; hk[9] += K11; hk[10] += K12;
                    hk[12] += K20; hk[13] += K21; hk[14] += K22;
                    // translation block Omega
                    hk[15] += o00; hk[16] += o01; hk[17] += o02;
                    hk[18] += o11; hk[19] += o12; hk[20] += o22;
                    nin += 1.f;
                }
            }
            if constexpr (GRAD) {
                // back to the current pose's tangent space: b += D^T b_k, H += D^T H_k D, D = diag(R, R)
                const float R[9] = {R00, R01, R02, R10, R11, R12, R20, R21, R22};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    sacc[1 + c][threadIdx.x] += fmaf(R[c], bk[0], fmaf(R[3 + c], bk[1], R[6 + c] * bk[2]));
                    sacc[4 + c][threadIdx.x] += fmaf(R[c], bk[3], fmaf(R[3 + c], bk[4], R[6 + c] * bk[5]));
                }
                float tl[6] = {hk[0], hk[1], hk[2], hk[6], hk[7], hk[11]};
                float tr[9] = {hk[3], hk[4], hk[5], hk[8], hk[9], hk[10], hk[12], hk[13], hk[14]};
                float br[6] = {hk[15], hk[16], hk[17], hk[18], hk[19], hk[20]};
                rot_sym(R, tl);
                rot_gen(R, tr);
                rot_sym(R, br);
                // accumulator layout: H upper triangle row-major at acc[7..27]
#define GMCS_ACC(e) sacc[e][threadIdx.x]
                GMCS_ACC(7) += tl[0]; GMCS_ACC(8) += tl[1]; GMCS_ACC(9) += tl[2];
                GMCS_ACC(13) += tl[3]; GMCS_ACC(14) += tl[4]; GMCS_ACC(18) += tl[5];
                GMCS_ACC(10) += tr[0]; GMCS_ACC(11) += tr[1]; GMCS_ACC(12) += tr[2];
                GMCS_ACC(15) += tr[3]; GMCS_ACC(16) += tr[4]; GMCS_ACC(17) += tr[5];
                GMCS_ACC(19) += tr[6]; GMCS_ACC(20) += tr[7]; GMCS_ACC(21) += tr[8];
                GMCS_ACC(22) += br[0]; GMCS_ACC(23) += br[1]; GMCS_ACC(24) += br[2];
                GMCS_ACC(25) += br[3]; GMCS_ACC(26) += br[4]; GMCS_ACC(27) += br[5];
                GMCS_ACC(28) += nin;
#undef GMCS_ACC
            }
        }
        acc[0] = lsum;
        if constexpr (GRAD)
            for (int e = 1; e < kAccGicp; ++e) acc[e] = sacc[e][threadIdx.x];
    }
    store_partials<NACC>(a, acc, ww);
}

template <bool GRAD>
__global__ void __launch_bounds__(kPassThreads, gicp_minblocks<GRAD>()) k_gicp(PassArgs a) {
    gicp_body<GRAD>(a, blockIdx.x);
}

template <bool GRAD>
__global__ void __launch_bounds__(kPassThreads, gicp_b_minblocks<GRAD>()) k_gicp_b(const BatchList<PassArgs>* L) {
    GMCS_BATCH_LOOP(L, const PassArgs a = L->args[s]; gicp_body<GRAD>(a, vb));
}

// ------------------------------------------------------------------ launchers

int grid_knn_cov(int n) { return (n + 3) / 4; }   // 4 points (warps) per CTA

void launch_knn_cov(const KnnCovArgs& a, cudaStream_t s) {
    if (a.n <= 0) return;
    const int grid = grid_knn_cov(a.n);
    if (a.k <= 8) k_knn_cov<8><<<grid, 128, 0, s>>>(a);
    else if (a.k <= 16) k_knn_cov<16><<<grid, 128, 0, s>>>(a);
    else k_knn_cov<32><<<grid, 128, 0, s>>>(a);
}

template <typename K>
static int persistent_grid_g(K kernel, int threads) {
    int per_sm = 0, dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * sms;
}

template <int KM>
static int grid_knn_b() {
    static const int g = persistent_grid_g(k_knn_cov_b<KM>, 128);
    return g;
}
template <bool G>
static int grid_gicp_b() {
    static const int g = persistent_grid_g(k_gicp_b<G>, kPassThreads);
    return g;
}

void launch_knn_cov_b(const BatchList<KnnCovArgs>* L, int k, cudaStream_t s) {
    if (k <= 8) k_knn_cov_b<8><<<grid_knn_b<8>(), 128, 0, s>>>(L);
    else if (k <= 16) k_knn_cov_b<16><<<grid_knn_b<16>(), 128, 0, s>>>(L);
    else k_knn_cov_b<32><<<grid_knn_b<32>(), 128, 0, s>>>(L);
}

void launch_gicp_b(const BatchList<PassArgs>* L, bool grad, cudaStream_t s) {
    if (grad) k_gicp_b<true><<<grid_gicp_b<true>(), kPassThreads, 0, s>>>(L);
    else k_gicp_b<false><<<grid_gicp_b<false>(), kPassThreads, 0, s>>>(L);
}

void prepare_gicp_batched() {
    grid_knn_b<8>();
    grid_knn_b<16>();
    grid_knn_b<32>();
    grid_gicp_b<true>();
    grid_gicp_b<false>();
}

void launch_voxel_accum(const VoxelArgs& a, cudaStream_t s) {
    if (a.n > 0) k_voxel_accum<<<(a.n + 255) / 256, 256, 0, s>>>(a);
}

void launch_voxel_final(const VoxelArgs& a, cudaStream_t s) {
    const size_t nv = (size_t)a.nx * a.ny * a.nz;
    size_t b = (nv + 255) / 256;
    if (b > 148 * 32) b = 148 * 32;
    if (nv > 0) k_voxel_final<<<(int)b, 256, 0, s>>>(a);
}

void launch_gicp_pass(const PassArgs& a, bool grad, cudaStream_t s) {
    const int grid = grid_pass(a);
    if (grid <= 0) return;
    if (grad) k_gicp<true><<<grid, kPassThreads, 0, s>>>(a);
    else k_gicp<false><<<grid, kPassThreads, 0, s>>>(a);
}

}  // namespace gmcs
