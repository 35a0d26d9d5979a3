// k_filter.cu -- prediction, neighbour selection, the lookup pass and the move.
//
// The lookup pass is the hot kernel: for every (particle i, scan point j,
// neighbour keyframe k) it transforms p_j by the relative pose kT_t = (T_k^i)^-1 T_t^i
// (Eq. 4), looks the result up in keyframe k's likelihood table (trilinear
// value and lattice gradient from one packed cell record), and accumulates
//   l = log(L + eps)                         per-lookup log-likelihood
//   d l / d xi = [p x q; q], q = R^T grad_x l  its se(3) gradient (form of Eq. 6)
//   w = L / (L + eps), w p, w p p^T           Gauss-Newton moments
// Lanes of a warp own 32 consecutive particles and walk the same points, so
// particles that are close in pose space (the copies resampling leaves next to
// each other) read neighbouring cells in one instruction. The warps of a CTA
// split the points of one particle tile; CTA partial sums go to a scratch
// buffer and a per-particle finish kernel adds them in a fixed order, so the
// result does not depend on scheduling.
//
// The gradient is accumulated per neighbour in the table's lattice frame and
// rotated once per (particle, neighbour): with A = R/h the affine map p -> u,
// r_j = A p_j and gu_j = grad_u l_j,
//   sum_j d l/d v     = A^T sum_j gu_j
//   sum_j d l/d omega = h A^T sum_j (r_j x gu_j)
// which equals the per-point [p x q; q] summed, since R^T (R p x g) = p x R^T g.
#include "kernels.h"

namespace gmcs {

// ------------------------------------------------------------------ layout helpers

__global__ void k_scan_pack(const float* __restrict__ xyz, int n, float4* __restrict__ out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        out[j] = make_float4(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], 0.f);
}

__global__ void k_aos_to_soa(const float* __restrict__ aos, int P, int C, float* __restrict__ soa, size_t ld) {
    const size_t n = (size_t)P * C;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / C), c = (int)(e % C);
        soa[(size_t)c * ld + i] = aos[e];
    }
}

__global__ void k_soa_to_aos(const float* __restrict__ soa, size_t ld, int P, int C, float* __restrict__ aos) {
    const size_t n = (size_t)P * C;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / C), c = (int)(e % C);
        aos[e] = soa[(size_t)c * ld + i];
    }
}

// ------------------------------------------------------------------ prediction, Eq. 1

// Lower Cholesky factor of a positive semi-definite 6x6 matrix; a non-positive
// pivot zeroes its column (a zero-variance direction draws no noise).
__device__ __forceinline__ void chol6_psd(const float* A, float* L) {
#pragma unroll
    for (int e = 0; e < 36; ++e) L[e] = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float d = A[j * 6 + j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j * 6 + k] * L[j * 6 + k];
        if (d > 0.f) {
            const float ljj = sqrtf(d);
            L[j * 6 + j] = ljj;
            const float inv = 1.f / ljj;
#pragma unroll
            for (int i = j + 1; i < 6; ++i) {
                float s = A[i * 6 + j];
#pragma unroll
                for (int k = 0; k < j; ++k) s -= L[i * 6 + k] * L[j * 6 + k];
                L[i * 6 + j] = s * inv;
            }
        }
    }
}

__global__ void __launch_bounds__(128) k_predict(PredictArgs a) {
    __shared__ float sL[36];
    if (threadIdx.x == 0) chol6_psd(a.cov, sL);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.P) return;
    float z[6];
    if (a.z) {
#pragma unroll
        for (int d = 0; d < 6; ++d) z[d] = a.z[(size_t)i * 6 + d];
    } else {
        normal6(a.seed, (uint32_t)i, a.frame, z);
    }
    float delta[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        float s = 0.f;
#pragma unroll
        for (int c = 0; c <= r; ++c) s += sL[r * 6 + c] * z[c];
        delta[r] = s;
    }
    float T[12], TdT[12], E[12], out[12];
    load_pose(a.pose, a.ld, i, T);
    pose_mul(T, a.dT, TdT);
    se3_exp(delta, E);
    pose_mul(TdT, E, out);
    store_pose(a.pose, a.ld, i, out);
}

// ------------------------------------------------------------------ neighbour keyframes

// The k_nb smallest squared translation distances, formed as (dx*dx + dy*dy) + dz*dz
// with separate round-to-nearest operations; ties keep the lower keyframe index.
__global__ void __launch_bounds__(128) k_select(SelectArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.P) return;
    const float tx = a.pose[3 * a.ld + i], ty = a.pose[7 * a.ld + i], tz = a.pose[11 * a.ld + i];
    float bd[kMaxNb];
    int bk[kMaxNb];
#pragma unroll
    for (int s = 0; s < kMaxNb; ++s) { bd[s] = __int_as_float(0x7f800000); bk[s] = -1; }
    for (int k = 0; k < a.K; ++k) {
        const float* T = a.kf + (size_t)k * kPoseC * a.ld;
        const float dx = __fsub_rn(T[3 * a.ld + i], tx);
        const float dy = __fsub_rn(T[7 * a.ld + i], ty);
        const float dz = __fsub_rn(T[11 * a.ld + i], tz);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        // insertion into the sorted list of the first k_nb entries
        int pos = a.k_nb;
#pragma unroll
        for (int s = kMaxNb - 1; s >= 0; --s)
            if (s < a.k_nb && (bk[s] < 0 || d2 < bd[s])) pos = s;
        if (pos < a.k_nb) {
#pragma unroll
            for (int s = kMaxNb - 1; s > 0; --s)
                if (s > pos && s < a.k_nb) { bd[s] = bd[s - 1]; bk[s] = bk[s - 1]; }
#pragma unroll
            for (int s = 0; s < kMaxNb; ++s)
                if (s == pos) { bd[s] = d2; bk[s] = k; }
        }
    }
#pragma unroll
    for (int s = 0; s < kMaxNb; ++s) {
        if (s < a.k_nb) {
            a.nbr[(size_t)s * a.ld + i] = bk[s];
            if (a.nbr_out) a.nbr_out[(size_t)i * a.k_nb + s] = bk[s];
        }
    }
}

// ------------------------------------------------------------------ the lookup pass

template <int DT, bool GRAD>
__global__ void __launch_bounds__(kPassThreads) k_pass(PassArgs a) {
    constexpr int NACC = GRAD ? kAccGrad : 1;
    __shared__ float red[kPassWarps][NACC][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.x % a.ntiles;
    const int grp = blockIdx.x / a.ntiles;
    const int i = tile * 32 + lane;
    const bool live = i < a.P;
    const int chunk = grp * kPassWarps + warp;
    const int j0 = min(chunk * a.chunk_len, a.N);
    const int j1 = min(j0 + a.chunk_len, a.N);

    float acc[NACC];
#pragma unroll
    for (int e = 0; e < NACC; ++e) acc[e] = 0.f;

    if (live && j0 < j1) {
        float Tt[12];
        load_pose(a.pose, a.ld, i, Tt);
        float lsum = 0.f;   // in log2 units
        for (int s = 0; s < a.k_nb; ++s) {
            const int k = a.nbr[(size_t)s * a.ld + i];
            if (k < 0) continue;
            const TableDesc td = a.tables[k];
            float Tk[12], rel[12];
            load_pose(a.kf + (size_t)k * kPoseC * a.ld, a.ld, i, Tk);
            pose_rel(Tk, Tt, rel);
            // affine map p -> u = A p + b onto the lattice
            const float A00 = rel[0] * td.inv_h, A01 = rel[1] * td.inv_h, A02 = rel[2] * td.inv_h;
            const float A10 = rel[4] * td.inv_h, A11 = rel[5] * td.inv_h, A12 = rel[6] * td.inv_h;
            const float A20 = rel[8] * td.inv_h, A21 = rel[9] * td.inv_h, A22 = rel[10] * td.inv_h;
            const float b0 = (rel[3] - td.ox) * td.inv_h;
            const float b1 = (rel[7] - td.oy) * td.inv_h;
            const float b2 = (rel[11] - td.oz) * td.inv_h;
            const uint32_t ncx = (uint32_t)td.ncx, ncy = (uint32_t)td.ncy, ncz = (uint32_t)td.ncz;
            const void* __restrict__ cells = td.cells;
            const float eps = a.eps;
            float Gx = 0.f, Gy = 0.f, Gz = 0.f, Cx = 0.f, Cy = 0.f, Cz = 0.f;
#pragma unroll 2
            for (int j = j0; j < j1; ++j) {
                const float4 p = __ldg(a.scan + j);
                const float rx = A00 * p.x + A01 * p.y + A02 * p.z;
                const float ry = A10 * p.x + A11 * p.y + A12 * p.z;
                const float rz = A20 * p.x + A21 * p.y + A22 * p.z;
                const float ux = rx + b0, uy = ry + b1, uz = rz + b2;
                const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
                const int cx = (int)flx, cy = (int)fly, cz = (int)flz;
                const bool valid = ((uint32_t)cx < ncx) & ((uint32_t)cy < ncy) & ((uint32_t)cz < ncz);
                const uint32_t idx = valid ? ((uint32_t)cz * ncy + (uint32_t)cy) * ncx + (uint32_t)cx : 0u;
                float v[8];
                load_cell<DT>(cells, idx, valid, v);
                const float fx = ux - flx, fy = uy - fly, fz = uz - flz;
                // trilinear value, corner order (dx + 2 dy + 4 dz)
                const float d00 = v[1] - v[0], d10 = v[3] - v[2], d01 = v[5] - v[4], d11 = v[7] - v[6];
                const float e00 = fmaf(fx, d00, v[0]), e10 = fmaf(fx, d10, v[2]);
                const float e01 = fmaf(fx, d01, v[4]), e11 = fmaf(fx, d11, v[6]);
                const float dy0 = e10 - e00, dy1 = e11 - e01;
                const float g0 = fmaf(fy, dy0, e00), g1 = fmaf(fy, dy1, e01);
                const float Lz = g1 - g0;
                const float L = fmaf(fz, Lz, g0);
                const float den = L + eps;
                lsum += __log2f(den);
                if constexpr (GRAD) {
                    const float hx0 = fmaf(fy, d10 - d00, d00), hx1 = fmaf(fy, d11 - d01, d01);
                    const float Lx = fmaf(fz, hx1 - hx0, hx0);
                    const float Ly = fmaf(fz, dy1 - dy0, dy0);
                    const float inv = __fdividef(1.f, den);
                    const float gx = Lx * inv, gy = Ly * inv, gz = Lz * inv;
                    Gx += gx; Gy += gy; Gz += gz;
                    Cx = fmaf(ry, gz, fmaf(-rz, gy, Cx));
                    Cy = fmaf(rz, gx, fmaf(-rx, gz, Cy));
                    Cz = fmaf(rx, gy, fmaf(-ry, gx, Cz));
                    const float w = L * inv;
                    const float wx = w * p.x, wy = w * p.y, wz = w * p.z;
                    acc[7] += w;
                    acc[8] += wx; acc[9] += wy; acc[10] += wz;
                    acc[11] = fmaf(wx, p.x, acc[11]); acc[12] = fmaf(wx, p.y, acc[12]); acc[13] = fmaf(wx, p.z, acc[13]);
                    acc[14] = fmaf(wy, p.y, acc[14]); acc[15] = fmaf(wy, p.z, acc[15]); acc[16] = fmaf(wz, p.z, acc[16]);
                }
            }
            if constexpr (GRAD) {
                // d l/d omega = h A^T C,  d l/d v = A^T G
                const float h = td.h;
                acc[1] += h * (A00 * Cx + A10 * Cy + A20 * Cz);
                acc[2] += h * (A01 * Cx + A11 * Cy + A21 * Cz);
                acc[3] += h * (A02 * Cx + A12 * Cy + A22 * Cz);
                acc[4] += A00 * Gx + A10 * Gy + A20 * Gz;
                acc[5] += A01 * Gx + A11 * Gy + A21 * Gz;
                acc[6] += A02 * Gx + A12 * Gy + A22 * Gz;
            }
        }
        acc[0] = lsum * 0.69314718055994531f;
    }

#pragma unroll
    for (int e = 0; e < NACC; ++e) red[warp][e][lane] = acc[e];
    __syncthreads();
    const int base = tile * 32;
    for (int t = threadIdx.x; t < NACC * 32; t += kPassThreads) {
        const int e = t >> 5, l = t & 31;
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kPassWarps; ++w) s += red[w][e][l];
        if (base + l < a.P) a.part[((size_t)grp * NACC + e) * a.ld + base + l] = s;
    }
}

// ------------------------------------------------------------------ finish: sums, move (Eq. 5-7)

__device__ __forceinline__ void finish_sum(const FinishArgs& a, int i, int nacc, float* acc) {
    for (int e = 0; e < nacc; ++e) acc[e] = 0.f;
    for (int g = 0; g < a.groups; ++g)
        for (int e = 0; e < nacc; ++e) acc[e] += a.part[((size_t)g * nacc + e) * a.ld + i];
}

// psi = (H + lambda diag H)^-1 g with H = sigma^-2 [[tr Q I - Q, [S]x], [[S]x^T, W I]],
// solved by Cholesky after symmetric Jacobi scaling; then clamped.
__device__ bool gn_step(const float* g, const float* mom, const FinishArgs& a, float* psi) {
#pragma unroll
    for (int d = 0; d < 6; ++d) psi[d] = 0.f;
    const float W = mom[0];
    if (!(W >= a.w_min)) return false;
    const float Sx = mom[1], Sy = mom[2], Sz = mom[3];
    const float Qxx = mom[4], Qxy = mom[5], Qxz = mom[6], Qyy = mom[7], Qyz = mom[8], Qzz = mom[9];
    const float tr = Qxx + Qyy + Qzz;
    float H[36] = {
        tr - Qxx, -Qxy,     -Qxz,     0.f, -Sz, Sy,
        -Qxy,     tr - Qyy, -Qyz,     Sz,  0.f, -Sx,
        -Qxz,     -Qyz,     tr - Qzz, -Sy, Sx,  0.f,
        0.f,      Sz,       -Sy,      W,   0.f, 0.f,
        -Sz,      0.f,      Sx,       0.f, W,   0.f,
        Sy,       -Sx,      0.f,      0.f, 0.f, W};
    const float k = 1.f / (a.sigma * a.sigma);
    float D[6], b[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const float hd = H[d * 6 + d] * k * (1.f + a.lambda);
        if (!(hd > 0.f)) return false;
        D[d] = rsqrtf(hd);
    }
    // scaled system: (D H' D) y = D g, psi = D y
#pragma unroll
    for (int r = 0; r < 6; ++r) {
#pragma unroll
        for (int c = 0; c < 6; ++c) H[r * 6 + c] = (r == c) ? (1.f + a.lambda) * H[r * 6 + c] * k * D[r] * D[c]
                                                            : H[r * 6 + c] * k * D[r] * D[c];
        b[r] = g[r] * D[r];
    }
    float L[36];
#pragma unroll
    for (int e = 0; e < 36; ++e) L[e] = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float d = H[j * 6 + j];
#pragma unroll
        for (int q = 0; q < j; ++q) d -= L[j * 6 + q] * L[j * 6 + q];
        if (!(d > 0.f)) return false;
        const float ljj = sqrtf(d);
        L[j * 6 + j] = ljj;
#pragma unroll
        for (int r = j + 1; r < 6; ++r) {
            float s = H[r * 6 + j];
#pragma unroll
            for (int q = 0; q < j; ++q) s -= L[r * 6 + q] * L[j * 6 + q];
            L[r * 6 + j] = s / ljj;
        }
    }
    float y[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        float s = b[r];
#pragma unroll
        for (int q = 0; q < r; ++q) s -= L[r * 6 + q] * y[q];
        y[r] = s / L[r * 6 + r];
    }
#pragma unroll
    for (int r = 5; r >= 0; --r) {
        float s = y[r];
#pragma unroll
        for (int q = r + 1; q < 6; ++q) s -= L[q * 6 + r] * psi[q];
        psi[r] = s / L[r * 6 + r];
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) psi[d] *= D[d];
    const float nw = sqrtf(psi[0] * psi[0] + psi[1] * psi[1] + psi[2] * psi[2]);
    const float nv = sqrtf(psi[3] * psi[3] + psi[4] * psi[4] + psi[5] * psi[5]);
    if (nw > a.theta_max) { const float sc = a.theta_max / nw; psi[0] *= sc; psi[1] *= sc; psi[2] *= sc; }
    if (nv > a.t_max) { const float sc = a.t_max / nv; psi[3] *= sc; psi[4] *= sc; psi[5] *= sc; }
    return true;
}

template <bool GRAD>
__global__ void __launch_bounds__(128) k_finish(FinishArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.P) return;
    constexpr int NACC = GRAD ? kAccGrad : 1;
    float acc[NACC];
    finish_sum(a, i, NACC, acc);
    if (a.out_ll) a.out_ll[i] = acc[0];
    if (!GRAD) {
        if (a.logw) a.logw[i] += (double)acc[0];
        return;
    } else {
        if (a.out_g)
            for (int d = 0; d < 6; ++d) a.out_g[(size_t)i * 6 + d] = acc[1 + d];
        if (a.out_mom)
            for (int d = 0; d < 10; ++d) a.out_mom[(size_t)i * 10 + d] = acc[7 + d];
        if (a.do_move) {
            float psi[6];
            if (gn_step(acc + 1, acc + 7, a, psi)) {
                float T[12], E[12], out[12];
                load_pose(a.pose, a.ld, i, T);
                se3_exp(psi, E);
                pose_mul(T, E, out);
                store_pose(a.pose, a.ld, i, out);
            }
        }
    }
}

// ------------------------------------------------------------------ launchers

static int blocks_for(size_t n, int threads, int cap = 148 * 16) {
    size_t b = (n + threads - 1) / threads;
    if (b > (size_t)cap) b = cap;
    return (int)(b > 0 ? b : 1);
}

void launch_scan_pack(const float* xyz, int n, float4* out, cudaStream_t s) {
    if (n > 0) k_scan_pack<<<blocks_for(n, 256), 256, 0, s>>>(xyz, n, out);
}

void launch_aos_to_soa(const float* aos, int P, int C, float* soa, size_t ld, cudaStream_t s) {
    if (P > 0) k_aos_to_soa<<<blocks_for((size_t)P * C, 256), 256, 0, s>>>(aos, P, C, soa, ld);
}

void launch_soa_to_aos(const float* soa, size_t ld, int P, int C, float* aos, cudaStream_t s) {
    if (P > 0) k_soa_to_aos<<<blocks_for((size_t)P * C, 256), 256, 0, s>>>(soa, ld, P, C, aos);
}

void launch_predict(const PredictArgs& a, cudaStream_t s) {
    if (a.P > 0) k_predict<<<(a.P + 127) / 128, 128, 0, s>>>(a);
}

void launch_select(const SelectArgs& a, cudaStream_t s) {
    if (a.P > 0) k_select<<<(a.P + 127) / 128, 128, 0, s>>>(a);
}

void launch_pass(const PassArgs& a, int dtype, bool grad, cudaStream_t s) {
    const int grid = a.ntiles * a.groups;
    if (grid <= 0) return;
#define GMCS_PASS(DT, G) k_pass<DT, G><<<grid, kPassThreads, 0, s>>>(a)
    if (grad) {
        if (dtype == 0) GMCS_PASS(0, true); else if (dtype == 1) GMCS_PASS(1, true); else GMCS_PASS(2, true);
    } else {
        if (dtype == 0) GMCS_PASS(0, false); else if (dtype == 1) GMCS_PASS(1, false); else GMCS_PASS(2, false);
    }
#undef GMCS_PASS
}

void launch_finish(const FinishArgs& a, bool grad, cudaStream_t s) {
    if (a.P <= 0) return;
    if (grad) k_finish<true><<<(a.P + 127) / 128, 128, 0, s>>>(a);
    else k_finish<false><<<(a.P + 127) / 128, 128, 0, s>>>(a);
}

}  // namespace gmcs
