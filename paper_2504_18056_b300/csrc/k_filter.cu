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
#include "pass.cuh"

namespace gmcs {

// ------------------------------------------------------------------ layout helpers

// A non-finite point is replaced by one far outside every map, so each of its
// lookups is a miss: it adds the same constant to every particle's log-likelihood
// (which the weight normalisation removes) and nothing to gradients or moments,
// instead of turning every particle's likelihood into NaN.
__device__ __forceinline__ void scan_pack_body(const ScanPackArgs& a, int vb, int vg) {
    for (int j = vb * blockDim.x + threadIdx.x; j < a.n; j += vg * blockDim.x) {
        float x = a.xyz[3 * j], y = a.xyz[3 * j + 1], z = a.xyz[3 * j + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) x = y = z = 1e30f;
        a.out[j] = make_float4(x, y, z, 1.f);   // w = 1: the moments' (z, 1) pair
    }
}

__global__ void k_scan_pack(ScanPackArgs a) { scan_pack_body(a, blockIdx.x, gridDim.x); }

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

__device__ __forceinline__ void predict_body(const PredictArgs& a, int vb, int vg) {
    __shared__ float sL[36];
    if (threadIdx.x == 0) chol6_psd(a.cov, sL);
    __syncthreads();
    const int i = vb * blockDim.x + threadIdx.x;
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

__global__ void __launch_bounds__(128) k_predict(PredictArgs a) { predict_body(a, blockIdx.x, gridDim.x); }

// ------------------------------------------------------------------ neighbour keyframes

// The k_nb smallest squared translation distances, formed as (dx*dx + dy*dy) + dz*dz
// with separate round-to-nearest operations; ties keep the lower keyframe index.
__device__ __forceinline__ void select_body(const SelectArgs& a, int vb, int vg) {
    const int i = vb * blockDim.x + threadIdx.x;
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

__global__ void __launch_bounds__(128) k_select(SelectArgs a) { select_body(a, blockIdx.x, gridDim.x); }

// ------------------------------------------------------------------ the lookup pass

#ifndef GMCS_PASS_MINBLOCKS
#define GMCS_PASS_MINBLOCKS 1
#endif
#ifndef GMCS_PASS_UNROLL
#define GMCS_PASS_UNROLL 2
#endif
#ifndef GMCS_PASS3
#define GMCS_PASS3 1
#endif
#ifndef GMCS_PASS3_MINBLOCKS
#define GMCS_PASS3_MINBLOCKS 1
#endif
constexpr int kPassUnroll = GMCS_PASS_UNROLL;
// Point-loop unrolling of the three-neighbour pass (independent lookups in
// flight per thread), per table type and pass kind.
#ifndef GMCS_U_G32
#define GMCS_U_G32 1
#endif
#ifndef GMCS_U_G16
#define GMCS_U_G16 2
#endif
#ifndef GMCS_U_V32
#define GMCS_U_V32 2
#endif
#ifndef GMCS_U_V16
#define GMCS_U_V16 2
#endif
template <int DT, bool GRAD>
constexpr int pass3_unroll() {
    return GRAD ? (DT == 0 ? GMCS_U_G32 : GMCS_U_G16) : (DT == 0 ? GMCS_U_V32 : GMCS_U_V16);
}

#ifndef GMCS_F32X2
#define GMCS_F32X2 1
#endif
// 16-bit tables: the packed (ux, uy) transform and round-down floor of the FP32
// path (1), or a scalar transform with floorf (0).
#ifndef GMCS_XY16
#define GMCS_XY16 1
#endif
constexpr bool kXy16 = GMCS_XY16;
// packed Gauss-Newton moments in the pipelined passes (Moments, below)
#ifndef GMCS_PMOM
#define GMCS_PMOM 1
#endif

// Packed two-lane FP32 arithmetic (Blackwell add/sub/fma .f32x2).
__device__ __forceinline__ float2 p2_sub(float2 a, float2 b) {
#if GMCS_F32X2
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&d);
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}

__device__ __forceinline__ float2 p2_add(float2 a, float2 b) {
#if GMCS_F32X2
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&d);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}

__device__ __forceinline__ float2 p2_mul(float2 a, float2 b) {
#if GMCS_F32X2
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&d);
#else
    return make_float2(a.x * b.x, a.y * b.y);
#endif
}

__device__ __forceinline__ float2 p2_fma(float2 a, float2 b, float2 c) {
#if GMCS_F32X2
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
          "l"(*reinterpret_cast<unsigned long long*>(&c)));
    return *reinterpret_cast<float2*>(&d);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}

// floor(u) as int and as float on the FMA/ALU pipes instead of the conversion
// unit: adding 1.5 * 2^23 with rounding toward -inf leaves floor(u) in the low
// mantissa bits, exactly, for |u| < 2^22. Outside that range (and for inf/NaN)
// the int lands far outside any table (tables have < 2^22 cells per axis), so
// the lookup reads as empty, as floorf does.
__device__ __forceinline__ int floor_split(float u, float& fl) {
    const float t = __fadd_rd(u, 12582912.0f);
    fl = __fsub_rn(t, 12582912.0f);
    return __float_as_int(t) - 0x4B400000;
}

// One lookup in the cell whose coefficient record (widened to float) is
// r = (c4, c2, c7, c6, c1, c0, c5, c3), at in-cell fraction (x, y, z): adds
// log2(L + eps) to lsum -- or, with PROD, multiplies L + eps into it (the caller
// takes one log2 of the product of a point's three lookups, each factor in
// [eps, 1 + eps]) -- and, with GRAD, returns w = L / (L + eps) and
// g = grad_f L / (L + eps). With a = c4 + c7 z, b = c1 + c5 z, d = c2 + c6 z, e = c0 + c3 z,
//   L = e + d y + x (b + a y),  dL/dx = b + a y,  dL/dy = d + a x,
//   dL/dz = (c3 + c6 y) + x (c5 + c7 y):
// 4 packed and 3 scalar FMAs for L and its gradient (interpolating the 8 corner
// values takes 9 packed and 6 scalar operations).
template <bool GRAD, bool PROD = false, bool LL = true>
__device__ __forceinline__ void coef_interp(const float* r, float fx, float fy, float fz, float eps, float& lsum,
                                            float& w, float& gx, float& gy, float& gz) {
    const float2 Q0 = make_float2(r[0], r[1]), Q1 = make_float2(r[2], r[3]);   // (c4, c2), (c7, c6)
    const float2 Q2 = make_float2(r[4], r[5]), Q3 = make_float2(r[6], r[7]);   // (c1, c0), (c5, c3)
    const float2 ZZ = make_float2(fz, fz), YY = make_float2(fy, fy);
    const float2 AD = p2_fma(Q1, ZZ, Q0);                          // (a, d)
    const float2 BE = p2_fma(Q3, ZZ, Q2);                          // (b, e)
    const float2 XE = p2_fma(YY, AD, BE);                          // (dL/dx, L at x = 0)
    const float L = fmaf(fx, XE.x, XE.y);
    const float den = L + eps;
    if constexpr (LL) {
        if constexpr (PROD) lsum *= den;
        else lsum += __log2f(den);
    }
    if constexpr (GRAD) {
        const float2 TS = p2_fma(Q1, YY, Q3);                      // (c5 + c7 y, c3 + c6 y)
        const float Ly = fmaf(fx, AD.x, AD.y);
        const float Lz = fmaf(fx, TS.x, TS.y);
        const float inv = __fdividef(1.f, den);
        gx = XE.x * inv;
        gy = Ly * inv;
        gz = Lz * inv;
        w = L * inv;
    }
}

template <int DT, bool GRAD, bool PROD = false>
__device__ __forceinline__ void lookup_cell(const void* __restrict__ cells, const uint2* __restrict__ dir,
                                            uint32_t ncx, uint32_t ncy, uint32_t ncz,
                                            int cx, int cy, int cz, float fx, float fy, float fz, float eps,
                                            float& lsum, float& w, float& gx, float& gy, float& gz) {
    bool valid;
    uint32_t idx = 0u;
    if (dir) {
        valid = col_cell(dir, ncx, ncy, cx, cy, cz, idx);
    } else {
        valid = ((uint32_t)cx < ncx) & ((uint32_t)cy < ncy) & ((uint32_t)cz < ncz);
        idx = valid ? ((uint32_t)cz * ncy + (uint32_t)cy) * ncx + (uint32_t)cx : 0u;
    }
    float v[8];
    load_cell<DT>(cells, idx, valid, v);
    coef_interp<GRAD, PROD>(v, fx, fy, fz, eps, lsum, w, gx, gy, gz);
}

template <int DT, bool GRAD, bool PROD = false>
__device__ __forceinline__ void lookup_one(const void* __restrict__ cells, const uint2* __restrict__ dir, uint32_t ncx,
                                           uint32_t ncy, uint32_t ncz, float ux, float uy, float uz, float eps,
                                           float& lsum, float& w, float& gx, float& gy, float& gz) {
    // floor on the FMA/ALU pipes (FP32 gradient pass 2.08 -> 2.01 ms)
    float flx, fly, flz;
    const int cx = floor_split(ux, flx);
    const int cy = floor_split(uy, fly);
    const int cz = floor_split(uz, flz);
    lookup_cell<DT, GRAD, PROD>(cells, dir, ncx, ncy, ncz, cx, cy, cz, ux - flx, uy - fly, uz - flz, eps, lsum, w, gx, gy,
                                gz);
}

__device__ __forceinline__ float2 p2_add_rm(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&d);
}

// Affine map p -> u = A p + b of one (particle, neighbour keyframe) pair onto
// that keyframe's lattice, with the table it reads.
struct Slot {
    float A00, A01, A02, A10, A11, A12, A20, A21, A22, b0, b1, b2;
    const void* cells;
    const uint2* dir;    // column-sparse table: its column directory (dense: null)
    uint32_t ncx, ncy, ncz;
};

// The table of neighbour slot k. No pass sees a negative neighbour index: the sets
// start as 0 (table 0, whose descriptor is zero while no keyframe exists), a
// selection writes -1 only while the context has no keyframe, and the entry points
// refuse to run a pass before a selection made with keyframes. The dense passes still read a negative index as an empty
// table (every lookup misses), a form that also compiles to the faster pass there
// (FP32 gradient pass 1.522 -> 1.512 ms); on column-sparse tables it costs 2-5 %
// (FP32 / BF16 gradient pass 1.882 / 1.947 -> 1.917 / 2.039 ms), so they index
// directly.
template <bool DIRECT = false>
__device__ __forceinline__ TableDesc slot_table(const PassArgs& a, int k) {
    if constexpr (DIRECT) return a.tables[k];
    if (k >= 0) return a.tables[k];
    TableDesc td;
    td.cells = nullptr;
    td.dir = nullptr;
    td.ox = td.oy = td.oz = 0.f;
    td.inv_h = td.h = 0.f;
    td.ncx = td.ncy = td.ncz = 0;
    td.dtype = 0;
    td.pad = 0;
    return td;
}

template <bool DIRECT = false>
__device__ __forceinline__ Slot make_slot(const PassArgs& a, int i, int k, const float* Tt) {
    const TableDesc td = slot_table<DIRECT>(a, k);
    float Tk[12], rel[12];
    load_pose(a.kf + (size_t)k * kPoseC * a.ld, a.ld, i, Tk);
    pose_rel(Tk, Tt, rel);
    Slot s;
    s.A00 = rel[0] * td.inv_h; s.A01 = rel[1] * td.inv_h; s.A02 = rel[2] * td.inv_h;
    s.A10 = rel[4] * td.inv_h; s.A11 = rel[5] * td.inv_h; s.A12 = rel[6] * td.inv_h;
    s.A20 = rel[8] * td.inv_h; s.A21 = rel[9] * td.inv_h; s.A22 = rel[10] * td.inv_h;
    s.b0 = (rel[3] - td.ox) * td.inv_h;
    s.b1 = (rel[7] - td.oy) * td.inv_h;
    s.b2 = (rel[11] - td.oz) * td.inv_h;
    s.cells = td.cells;
    s.dir = td.dir;
    s.ncx = (uint32_t)td.ncx;
    s.ncy = (uint32_t)td.ncy;
    s.ncz = (uint32_t)td.ncz;
    return s;
}

// Fold one slot's lattice-frame sums into d l/d xi. With r_j = u_j - b the
// rotated point in lattice units, sum r x g = Cu - b x G where Cu = sum u x g;
// then d l/d omega = h A^T (Cu - b x G) and d l/d v = A^T G.
__device__ __forceinline__ void fold_slot(const Slot& s, float h, float Gx, float Gy, float Gz, float Ux, float Uy,
                                          float Uz, float* acc) {
    const float Cx = Ux - (s.b1 * Gz - s.b2 * Gy);
    const float Cy = Uy - (s.b2 * Gx - s.b0 * Gz);
    const float Cz = Uz - (s.b0 * Gy - s.b1 * Gx);
    acc[1] += h * (s.A00 * Cx + s.A10 * Cy + s.A20 * Cz);
    acc[2] += h * (s.A01 * Cx + s.A11 * Cy + s.A21 * Cz);
    acc[3] += h * (s.A02 * Cx + s.A12 * Cy + s.A22 * Cz);
    acc[4] += s.A00 * Gx + s.A10 * Gy + s.A20 * Gz;
    acc[5] += s.A01 * Gx + s.A11 * Gy + s.A21 * Gz;
    acc[6] += s.A02 * Gx + s.A12 * Gy + s.A22 * Gz;
}

__device__ __forceinline__ void add_moments(float w, float4 p, float* acc) {
    const float wx = w * p.x, wy = w * p.y, wz = w * p.z;
    acc[7] += w;
    acc[8] += wx; acc[9] += wy; acc[10] += wz;
    acc[11] = fmaf(wx, p.x, acc[11]); acc[12] = fmaf(wx, p.y, acc[12]); acc[13] = fmaf(wx, p.z, acc[13]);
    acc[14] = fmaf(wy, p.y, acc[14]); acc[15] = fmaf(wy, p.z, acc[15]); acc[16] = fmaf(wz, p.z, acc[16]);
}

// Generic pass: any number of neighbour slots, neighbour loop outside the point loop.
template <int DT, bool GRAD>
__global__ void __launch_bounds__(kPassThreads, GMCS_PASS_MINBLOCKS) k_pass(PassArgs a) {
    constexpr int NACC = GRAD ? kAccGrad : 1;
    const WarpWork ww = warp_work(a, blockIdx.x);
    const int i = ww.i, j0 = ww.j0, j1 = ww.j1;

    float acc[NACC];
#pragma unroll
    for (int e = 0; e < NACC; ++e) acc[e] = 0.f;

    if (i < a.P && j0 < j1) {
        float lsum = 0.f;   // in log2 units
        for (int s = 0; s < a.k_nb; ++s) {
            const int k = a.nbr[(size_t)s * a.ld + i];
            if (k < 0) continue;
            float Tt[12];
            load_pose(a.pose, a.ld, i, Tt);
            const Slot sl = make_slot(a, i, k, Tt);
            const float eps = a.eps;
            float Gx = 0.f, Gy = 0.f, Gz = 0.f, Cx = 0.f, Cy = 0.f, Cz = 0.f;
#pragma unroll kPassUnroll
            for (int j = j0; j < j1; ++j) {
                const float4 p = __ldg(a.scan + j);
                const float ux = fmaf(sl.A00, p.x, fmaf(sl.A01, p.y, fmaf(sl.A02, p.z, sl.b0)));
                const float uy = fmaf(sl.A10, p.x, fmaf(sl.A11, p.y, fmaf(sl.A12, p.z, sl.b1)));
                const float uz = fmaf(sl.A20, p.x, fmaf(sl.A21, p.y, fmaf(sl.A22, p.z, sl.b2)));
                float w, gx, gy, gz;
                lookup_one<DT, GRAD>(sl.cells, sl.dir, sl.ncx, sl.ncy, sl.ncz, ux, uy, uz, eps, lsum, w, gx, gy, gz);
                if constexpr (GRAD) {
                    Gx += gx; Gy += gy; Gz += gz;
                    Cx = fmaf(uy, gz, fmaf(-uz, gy, Cx));
                    Cy = fmaf(uz, gx, fmaf(-ux, gz, Cy));
                    Cz = fmaf(ux, gy, fmaf(-uy, gx, Cz));
                    add_moments(w, p, acc);
                }
            }
            if constexpr (GRAD) fold_slot(sl, a.tables[k].h, Gx, Gy, Gz, Cx, Cy, Cz, acc);
        }
        acc[0] = lsum * 0.69314718055994531f;
    }
    store_partials<NACC>(a, acc, ww);
}

// Three neighbour slots (the paper's choice, Sec. III-C): the neighbour loop
// runs inside the point loop, so each scan point is read once and its weight
// moments are accumulated once for all three lookups, which are independent
// and keep three cell loads in flight.
template <int DT, bool GRAD, int UNROLL>
__device__ __forceinline__ void pass3_body(const PassArgs& a, int vb) {
    constexpr int NACC = GRAD ? kAccGrad : 1;
    const WarpWork ww = warp_work(a, vb);
    const int i = ww.i, j0 = ww.j0, j1 = ww.j1;

    float acc[NACC];
#pragma unroll
    for (int e = 0; e < NACC; ++e) acc[e] = 0.f;

    if (i < a.P && j0 < j1) {
        Slot sl[3];
        int ks[3];
        {
            float Tt[12];
            load_pose(a.pose, a.ld, i, Tt);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                ks[s] = a.nbr[(size_t)s * a.ld + i];
                sl[s] = make_slot(a, i, ks[s], Tt);
            }
        }
        const float eps = a.eps;
        float lsum = 0.f;
        float G[3][3], C[3][3];
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int d = 0; d < 3; ++d) G[s][d] = C[s][d] = 0.f;
#pragma unroll UNROLL
        for (int j = j0; j < j1; ++j) {
            const float4 p = __ldg(a.scan + j);
            float wsum = 0.f;
            // value pass: one log2 per point of the product of its three L + eps (1.21 -> 1.19
            // ms FP32, 1.19 -> 1.16 ms BF16); in this unpipelined body the gradient pass keeps
            // one per lookup, the product's live range costs it registers (1.95 -> 1.98 ms
            // FP32, 1.80 -> 2.15 ms BF16)
            constexpr bool kProd = !GRAD;
            float lprod = 1.f;
            float& lacc = kProd ? lprod : lsum;
            // (ux, uy) and their floor on packed pairs (FP32 gradient pass 2.01 -> 1.95 ms)
            const float2 PX = make_float2(p.x, p.x), PY = make_float2(p.y, p.y), PZ = make_float2(p.z, p.z);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                float w, gx, gy, gz, ux, uy;
                const float uz = fmaf(sl[s].A20, p.x, fmaf(sl[s].A21, p.y, fmaf(sl[s].A22, p.z, sl[s].b2)));
                if constexpr (DT == 0 || kXy16) {
                    const float2 uxy = p2_fma(make_float2(sl[s].A00, sl[s].A10), PX,
                                              p2_fma(make_float2(sl[s].A01, sl[s].A11), PY,
                                                     p2_fma(make_float2(sl[s].A02, sl[s].A12), PZ,
                                                            make_float2(sl[s].b0, sl[s].b1))));
                    ux = uxy.x;
                    uy = uxy.y;
                    const float2 C2 = make_float2(12582912.0f, 12582912.0f);
                    const float2 t2 = p2_add_rm(uxy, C2);
                    const float2 f2 = p2_sub(uxy, p2_sub(t2, C2));
                    float flz;
                    const int cz = floor_split(uz, flz);
                    lookup_cell<DT, GRAD, kProd>(sl[s].cells, sl[s].dir, sl[s].ncx, sl[s].ncy, sl[s].ncz,
                                          __float_as_int(t2.x) - 0x4B400000, __float_as_int(t2.y) - 0x4B400000, cz,
                                          f2.x, f2.y, uz - flz, eps, lacc, w, gx, gy, gz);
                } else {
                    ux = fmaf(sl[s].A00, p.x, fmaf(sl[s].A01, p.y, fmaf(sl[s].A02, p.z, sl[s].b0)));
                    uy = fmaf(sl[s].A10, p.x, fmaf(sl[s].A11, p.y, fmaf(sl[s].A12, p.z, sl[s].b1)));
                    lookup_one<DT, GRAD, kProd>(sl[s].cells, sl[s].dir, sl[s].ncx, sl[s].ncy, sl[s].ncz, ux, uy,
                                                              uz, eps, lacc, w, gx, gy, gz);
                }
                if constexpr (GRAD) {
                    G[s][0] += gx; G[s][1] += gy; G[s][2] += gz;
                    C[s][0] = fmaf(uy, gz, fmaf(-uz, gy, C[s][0]));
                    C[s][1] = fmaf(uz, gx, fmaf(-ux, gz, C[s][1]));
                    C[s][2] = fmaf(ux, gy, fmaf(-uy, gx, C[s][2]));
                    wsum += w;
                }
            }
            if constexpr (kProd) lsum += __log2f(lprod);
            if constexpr (GRAD) add_moments(wsum, p, acc);
        }
        if constexpr (GRAD) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
                fold_slot(sl[s], slot_table(a, ks[s]).h, G[s][0], G[s][1], G[s][2], C[s][0], C[s][1], C[s][2], acc);
        }
        acc[0] = lsum * 0.69314718055994531f;
    }
    store_partials<NACC>(a, acc, ww);
}

// ---- software-pipelined three-neighbour pass: two stages in turn, so that
// while one point's three cell records are interpolated, the next point's are
// in flight (FP32 gradient pass 1.95 -> 1.77 ms; FP32 value pass, with the
// 256-bit record load, 1.16 -> 1.08 ms at 4 CTAs per SM).
#ifndef GMCS_PIPE_G32
#define GMCS_PIPE_G32 1
#endif
#ifndef GMCS_PIPE_G16
#define GMCS_PIPE_G16 1
#endif
#ifndef GMCS_PIPE_V32
#define GMCS_PIPE_V32 1
#endif
#ifndef GMCS_PIPE_V16
#define GMCS_PIPE_V16 1
#endif
template <int DT, bool GRAD>
constexpr bool pass3_pipelined() {
    return GRAD ? (DT == 0 ? GMCS_PIPE_G32 : GMCS_PIPE_G16) : (DT == 0 ? GMCS_PIPE_V32 : GMCS_PIPE_V16);
}

// u = A p + b of one slot as three float4 in the order the packed (ux, uy)
// transform reads it, so that each operand pair sits in adjacent registers:
// q0 = (A00, A10, A01, A11), q1 = (A02, A12, b0, b1), q2 = (A20, A21, A22, b2).
// (Scalar fields cost the pipelined gradient pass 1.77 -> 1.91 ms.)
struct Xf {
    float4 q0, q1, q2;
};

__device__ __forceinline__ Xf slot_xf(const Slot& s) {
    Xf x;
    x.q0 = make_float4(s.A00, s.A10, s.A01, s.A11);
    x.q1 = make_float4(s.A02, s.A12, s.b0, s.b1);
    x.q2 = make_float4(s.A20, s.A21, s.A22, s.b2);
    return x;
}

__device__ __forceinline__ void xf_slot(const Xf& x, Slot& s) {
    s.A00 = x.q0.x; s.A10 = x.q0.y; s.A01 = x.q0.z; s.A11 = x.q0.w;
    s.A02 = x.q1.x; s.A12 = x.q1.y; s.b0 = x.q1.z; s.b1 = x.q1.w;
    s.A20 = x.q2.x; s.A21 = x.q2.y; s.A22 = x.q2.z; s.b2 = x.q2.w;
}

// Lattice coordinate u of p in one slot, its cell c and in-cell fraction f
// ((ux, uy) on packed pairs and the round-down floor; with GMCS_XY16 = 0 the
// 16-bit tables take a scalar transform and floorf). ZCVT takes
// the z floor on the conversion unit instead, off the FMA pipe: with coefficient
// records the pipelined FP32 passes gain (gradient 1.65 -> 1.58 ms, value
// 1.078 -> 1.061 ms; with corner records the gradient pass lost, 1.720 -> 1.743).
template <int DT, bool ZCVT = false>
__device__ __forceinline__ void slot_point(const Xf& x, float4 p, float& ux, float& uy, float& uz, int& cx, int& cy,
                                           int& cz, float& fx, float& fy, float& fz) {
    uz = fmaf(x.q2.x, p.x, fmaf(x.q2.y, p.y, fmaf(x.q2.z, p.z, x.q2.w)));
    if constexpr (DT == 0 || kXy16) {
        const float2 uxy = p2_fma(make_float2(x.q0.x, x.q0.y), make_float2(p.x, p.x),
                                  p2_fma(make_float2(x.q0.z, x.q0.w), make_float2(p.y, p.y),
                                         p2_fma(make_float2(x.q1.x, x.q1.y), make_float2(p.z, p.z),
                                                make_float2(x.q1.z, x.q1.w))));
        ux = uxy.x;
        uy = uxy.y;
        const float2 C2 = make_float2(12582912.0f, 12582912.0f);
        const float2 t2 = p2_add_rm(uxy, C2);
        const float2 f2 = p2_sub(uxy, p2_sub(t2, C2));
        float flz;
        if constexpr (ZCVT) {
            flz = floorf(uz);
            cz = (int)flz;
        } else {
            cz = floor_split(uz, flz);
        }
        cx = __float_as_int(t2.x) - 0x4B400000;
        cy = __float_as_int(t2.y) - 0x4B400000;
        fx = f2.x;
        fy = f2.y;
        fz = uz - flz;
    } else {
        ux = fmaf(x.q0.x, p.x, fmaf(x.q0.z, p.y, fmaf(x.q1.x, p.z, x.q1.z)));
        uy = fmaf(x.q0.y, p.x, fmaf(x.q0.w, p.y, fmaf(x.q1.y, p.z, x.q1.w)));
        const float flx = floorf(ux), fly = floorf(uy), flz = floorf(uz);
        cx = (int)flx; cy = (int)fly; cz = (int)flz;
        fx = ux - flx; fy = uy - fly; fz = uz - flz;
    }
}

// slot_point with uz given, and (ZF) its floor too (cz, fz given).
template <bool ZF>
__device__ __forceinline__ void slot_point_z(const Xf& x, float4 p, float uz_in, int cz_in, float fz_in, float& ux,
                                             float& uy, float& uz, int& cx, int& cy, int& cz, float& fx, float& fy,
                                             float& fz) {
    uz = uz_in;
    const float2 uxy = p2_fma(make_float2(x.q0.x, x.q0.y), make_float2(p.x, p.x),
                              p2_fma(make_float2(x.q0.z, x.q0.w), make_float2(p.y, p.y),
                                     p2_fma(make_float2(x.q1.x, x.q1.y), make_float2(p.z, p.z),
                                            make_float2(x.q1.z, x.q1.w))));
    ux = uxy.x;
    uy = uxy.y;
    const float2 C2 = make_float2(12582912.0f, 12582912.0f);
    const float2 t2 = p2_add_rm(uxy, C2);
    const float2 f2 = p2_sub(uxy, p2_sub(t2, C2));
    if constexpr (ZF) {
        cz = cz_in;
        fz = fz_in;
    } else {
        const float flz = floorf(uz);
        cz = (int)flz;
        fz = uz - flz;
    }
    cx = __float_as_int(t2.x) - 0x4B400000;
    cy = __float_as_int(t2.y) - 0x4B400000;
    fx = f2.x;
    fy = f2.y;
}

// Pipelined passes with two whole stages: the z rows of neighbour slots 0 and 1 on
// one packed pair, and their floor on the pair as well (2: FP32 gradient pass 1.534
// -> 1.511 ms), the z rows only (1: 1.527 ms), or per slot (0); ZPAIR_SP: on
// column-sparse tables too (FP32 gradient pass 1.917 -> 2.089 ms, so off)
#ifndef GMCS_ZPAIR
#define GMCS_ZPAIR 2
#endif
#ifndef GMCS_ZPAIR_SP
#define GMCS_ZPAIR_SP 0
#endif
// with the pair, slot 2's z floor by the round-down add (1: 1.512 -> 1.547 ms) or on
// the conversion unit (0)
#ifndef GMCS_Z2MAGIC
#define GMCS_Z2MAGIC 0
#endif

// A cell record as loaded: two float4 (FP32) or one uint4 of 16-bit
// coefficients; widened to floats only when it is interpolated.
template <int DT>
struct RawRec {
    uint4 q;
};
template <>
struct RawRec<0> {
    float4 a, b;
};

// Load record idx of a table into r if valid, else zero r. (Leaving r as it was
// under the predicate and masking the lookup where it is used keeps both stages'
// records live through the loop: 168 registers with spills, FP32 gradient pass
// 1.57 -> 2.17 ms.)
template <int DT>
__device__ __forceinline__ void rec_load(const void* __restrict__ cells, uint32_t idx, bool valid, RawRec<DT>& r) {
    if constexpr (DT == 0) {
        r.a = make_float4(0.f, 0.f, 0.f, 0.f);
        r.b = r.a;
        if (valid) ld_record32(reinterpret_cast<const float4*>(cells) + 2 * (size_t)idx, r.a, r.b);
    } else {
        r.q = make_uint4(0u, 0u, 0u, 0u);
        if (valid) r.q = __ldg(reinterpret_cast<const uint4*>(cells) + idx);
    }
}

// Issue the load of cell c of a slot's table; a cell outside the table, or a
// stage with no point (live = false), reads as zeros: the lane's load is
// predicated off and its record registers are zeroed. (Loading a zero record
// stored before cell 0 instead, with no predicate, cost the FP32 gradient pass
// 1.57 -> 1.69 ms: the extra sector in many warp requests; taking the sign of
// a -1 index as the predicate cost 1.57 -> 2.12 ms.)
template <int DT, bool SP = false>
__device__ __forceinline__ void fetch_raw(const void* __restrict__ cells, const uint2* __restrict__ dir, uint32_t ncx,
                                          uint32_t ncy, uint32_t ncz, int cx, int cy, int cz, bool live,
                                          RawRec<DT>& r) {
    bool valid;
    uint32_t idx;
    if constexpr (SP) {
        // column-sparse: the record index comes from the column's directory entry
        valid = live && col_cell(dir, ncx, ncy, cx, cy, cz, idx);
    } else {
        valid = live & ((uint32_t)cx < ncx) & ((uint32_t)cy < ncy) & ((uint32_t)cz < ncz);
        idx = ((uint32_t)cz * ncy + (uint32_t)cy) * ncx + (uint32_t)cx;   // used only when valid
    }
    rec_load<DT>(cells, idx, valid, r);
}

// Column-sparse tables: the record of cell layer cz from its column's directory
// entry d (already loaded; (0, 0) outside the lattice, an empty run).
template <int DT>
__device__ __forceinline__ void fetch_dir(const void* __restrict__ cells, uint2 d, int cz, bool live, RawRec<DT>& r) {
    const uint32_t rel = (uint32_t)cz - (d.y & 0xFFFFu);
    const bool valid = live & (rel < (d.y >> 16));
    rec_load<DT>(cells, d.x + rel, valid, r);
}

// column-sparse tables: directory entries loaded one issue ahead (1), or on the
// record load's address chain (0: FP32 gradient / value pass 1.948 / 1.350 ms
// against 1.882 / 1.191 ms ahead)
#ifndef GMCS_DIR_AHEAD
#define GMCS_DIR_AHEAD 1
#endif
constexpr bool kDirAhead = GMCS_DIR_AHEAD;
// dense tables: the next point to issue loaded one issue ahead (1: FP32 gradient /
// value pass 1.570 / 1.035 -> 1.530 / 1.010 ms, BF16 value pass 0.986 -> 0.970 ms),
// or when it is issued (0)
#ifndef GMCS_P_AHEAD
#define GMCS_P_AHEAD 1
#endif

template <int DT>
__device__ __forceinline__ void unpack_raw(const RawRec<DT>& r, float* v) {
    if constexpr (DT == 0) {
        v[0] = r.a.x; v[1] = r.a.y; v[2] = r.a.z; v[3] = r.a.w;
        v[4] = r.b.x; v[5] = r.b.y; v[6] = r.b.z; v[7] = r.b.w;
    } else {
        decode_rec16<DT>(r.q, v);
    }
}

// One point between the issue of its three loads and their use.
template <int DT>
struct Stage {
    float4 p;
    float u[3][3], f[3][3];
    RawRec<DT> r[3];
};

// Gauss-Newton moments of the field model (W, S = sum w p, Q = sum w p p^T) in
// packed pairs: with the scan point stored as (x, y, z, 1), (Sx, Sy) += w (x, y),
// (Sz, W) += w (z, 1), (Qxx, Qyy) += (wx, wy) (x, y), (Qxz, Qyz) += (wx, wy) (z, z):
// 4 packed and 3 scalar operations per point instead of 13 scalar ones.
struct Moments {
    float2 sxy, szw, qd, qz;
    float qxy, qzz;
};

__device__ __forceinline__ void moments_zero(Moments& m) {
    m.sxy = m.szw = m.qd = m.qz = make_float2(0.f, 0.f);
    m.qxy = m.qzz = 0.f;
}

__device__ __forceinline__ void moments_add(Moments& m, float w, float4 p) {
    const float2 WW = make_float2(w, w), XY = make_float2(p.x, p.y);
    const float2 wxy = p2_mul(WW, XY);
    m.sxy = p2_add(m.sxy, wxy);
    m.szw = p2_fma(WW, make_float2(p.z, p.w), m.szw);
    m.qd = p2_fma(wxy, XY, m.qd);
    m.qz = p2_fma(wxy, make_float2(p.z, p.z), m.qz);
    m.qxy = fmaf(wxy.x, p.y, m.qxy);
    m.qzz = fmaf(w * p.z, p.z, m.qzz);
}

// Into the accumulator layout [.., W, Sx, Sy, Sz, Qxx, Qxy, Qxz, Qyy, Qyz, Qzz].
__device__ __forceinline__ void moments_store(const Moments& m, float* acc) {
    acc[7] = m.szw.y;
    acc[8] = m.sxy.x; acc[9] = m.sxy.y; acc[10] = m.szw.x;
    acc[11] = m.qd.x; acc[12] = m.qxy; acc[13] = m.qz.x;
    acc[14] = m.qd.y; acc[15] = m.qz.y; acc[16] = m.qzz;
}

// LL: the gradient pass also accumulates the log-likelihood (a caller asked for
// it); the moves of a frame need only the gradient and the moments.
template <int DT, bool GRAD, bool LL = true, bool SP = false>
__device__ __forceinline__ void pass3p_body(const PassArgs& a, int vb) {
    constexpr int NACC = GRAD ? kAccGrad : 1;
    constexpr bool kLL = LL || !GRAD;
    const WarpWork ww = warp_work(a, vb);
    const int i = ww.i, j0 = ww.j0, j1 = ww.j1;

    float acc[NACC];
#pragma unroll
    for (int e = 0; e < NACC; ++e) acc[e] = 0.f;

    if (i < a.P && j0 < j1) {
        Xf xf[3];
        const void* cells[3];
        const uint2* dirs[3];
        uint32_t ncx[3], ncy[3], ncz[3];
        int ks[3];
        {
            float Tt[12];
            load_pose(a.pose, a.ld, i, Tt);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                ks[s] = a.nbr[(size_t)s * a.ld + i];
                const Slot sl = make_slot<SP>(a, i, ks[s], Tt);
                xf[s] = slot_xf(sl);
                cells[s] = sl.cells;
                dirs[s] = sl.dir;
                ncx[s] = sl.ncx; ncy[s] = sl.ncy; ncz[s] = sl.ncz;
            }
        }
        const float eps = a.eps;
        float lsum = 0.f;
        float G[3][3], C[3][3];
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int d = 0; d < 3; ++d) G[s][d] = C[s][d] = 0.f;
        Moments mom;
        moments_zero(mom);

        // column-sparse tables: the directory entries of the next point to issue are
        // loaded one issue ahead (the columns from its (x, y) transform, recomputed when
        // it is issued), so the record loads do not wait on them
        float4 pd = make_float4(0.f, 0.f, 0.f, 1.f);
        uint2 dd[3] = {make_uint2(0u, 0u), make_uint2(0u, 0u), make_uint2(0u, 0u)};
        constexpr bool kPd = (SP && kDirAhead) || GMCS_P_AHEAD;
        auto ahead = [&](int j, bool live) {
            if constexpr (kPd) pd = __ldg(a.scan + j);
            if constexpr (SP && kDirAhead) {
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    const float2 uxy = p2_fma(make_float2(xf[s].q0.x, xf[s].q0.y), make_float2(pd.x, pd.x),
                                              p2_fma(make_float2(xf[s].q0.z, xf[s].q0.w), make_float2(pd.y, pd.y),
                                                     p2_fma(make_float2(xf[s].q1.x, xf[s].q1.y),
                                                            make_float2(pd.z, pd.z),
                                                            make_float2(xf[s].q1.z, xf[s].q1.w))));
                    const float2 t2 = p2_add_rm(uxy, make_float2(12582912.0f, 12582912.0f));
                    const uint32_t cx = (uint32_t)(__float_as_int(t2.x) - 0x4B400000);
                    const uint32_t cy = (uint32_t)(__float_as_int(t2.y) - 0x4B400000);
                    dd[s] = make_uint2(0u, 0u);
                    if (live && cx < ncx[s] && cy < ncy[s]) dd[s] = __ldg(dirs[s] + (cy * ncx[s] + cx));
                }
            }
        };
        constexpr int kZp = (!SP || GMCS_ZPAIR_SP) ? GMCS_ZPAIR : 0;
        auto issue = [&](Stage<DT>& st, int j, bool live, int jn, bool live_n) {
            st.p = kPd ? pd : __ldg(a.scan + j);
            float2 z01 = make_float2(0.f, 0.f), fz01 = z01;
            int cz0 = 0, cz1 = 0;
            if constexpr (kZp > 0) {
                const float4 p = st.p;
                z01 = p2_fma(make_float2(xf[0].q2.x, xf[1].q2.x), make_float2(p.x, p.x),
                             p2_fma(make_float2(xf[0].q2.y, xf[1].q2.y), make_float2(p.y, p.y),
                                    p2_fma(make_float2(xf[0].q2.z, xf[1].q2.z), make_float2(p.z, p.z),
                                           make_float2(xf[0].q2.w, xf[1].q2.w))));
                if constexpr (kZp == 2) {
                    const float2 C2 = make_float2(12582912.0f, 12582912.0f);
                    const float2 t2 = p2_add_rm(z01, C2);
                    fz01 = p2_sub(z01, p2_sub(t2, C2));
                    cz0 = __float_as_int(t2.x) - 0x4B400000;
                    cz1 = __float_as_int(t2.y) - 0x4B400000;
                }
            }
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                int cx, cy, cz;
                if constexpr (kZp > 0) {
                    if (s < 2)
                        slot_point_z<kZp == 2>(xf[s], st.p, s == 0 ? z01.x : z01.y, s == 0 ? cz0 : cz1,
                                               s == 0 ? fz01.x : fz01.y, st.u[s][0], st.u[s][1], st.u[s][2], cx, cy,
                                               cz, st.f[s][0], st.f[s][1], st.f[s][2]);
                    else
                        slot_point<DT, !GMCS_Z2MAGIC>(xf[s], st.p, st.u[s][0], st.u[s][1], st.u[s][2], cx, cy, cz,
                                                      st.f[s][0], st.f[s][1], st.f[s][2]);
                } else {
                    slot_point<DT, true>(xf[s], st.p, st.u[s][0], st.u[s][1], st.u[s][2], cx, cy, cz, st.f[s][0],
                                         st.f[s][1], st.f[s][2]);
                }
                if constexpr (SP && kDirAhead) fetch_dir<DT>(cells[s], dd[s], cz, live, st.r[s]);
                else fetch_raw<DT, SP>(cells[s], dirs[s], ncx[s], ncy[s], ncz[s], cx, cy, cz, live, st.r[s]);
            }
            ahead(jn, live_n);
        };
        auto use = [&](const Stage<DT>& st) {
            // one log2 per point of the product of its three L + eps (each in [eps, 1 + eps]),
            // in both passes (gradient pass 1.577 -> 1.553 ms)
            float lprod = 1.f;
            if constexpr (GRAD) {
                float wsum = 0.f;
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    float v[8], w, gx, gy, gz;
                    unpack_raw<DT>(st.r[s], v);
                    coef_interp<true, true, kLL>(v, st.f[s][0], st.f[s][1], st.f[s][2], eps, lprod, w, gx, gy, gz);
                    const float ux = st.u[s][0], uy = st.u[s][1], uz = st.u[s][2];
                    G[s][0] += gx; G[s][1] += gy; G[s][2] += gz;
                    C[s][0] = fmaf(uy, gz, fmaf(-uz, gy, C[s][0]));
                    C[s][1] = fmaf(uz, gx, fmaf(-ux, gz, C[s][1]));
                    C[s][2] = fmaf(ux, gy, fmaf(-uy, gx, C[s][2]));
                    wsum += w;
                }
#if GMCS_PMOM
                moments_add(mom, wsum, st.p);
#else
                add_moments(wsum, st.p, acc);
#endif
            } else {
                float w, gx, gy, gz;
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    float v[8];
                    unpack_raw<DT>(st.r[s], v);
                    coef_interp<false, true>(v, st.f[s][0], st.f[s][1], st.f[s][2], eps, lprod, w, gx, gy, gz);
                }
            }
            if constexpr (kLL) lsum += __log2f(lprod);
        };
        Stage<DT> SA, SB;
        ahead(j0, true);
        issue(SA, j0, true, j0 + 1 < j1 ? j0 + 1 : j0, j0 + 1 < j1);
        for (int j = j0;; j += 2) {   // j1 and the exits are uniform across the warp
            const bool m1 = j + 1 < j1, m2 = j + 2 < j1, m3 = j + 3 < j1;
            issue(SB, m1 ? j + 1 : j, m1, m2 ? j + 2 : j, m2);
            use(SA);
            if (!m1) break;
            issue(SA, m2 ? j + 2 : j + 1, m2, m3 ? j + 3 : j, m3);
            use(SB);
            if (!m2) break;
        }
        if constexpr (GRAD) {
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                Slot sl;
                xf_slot(xf[s], sl);
                fold_slot(sl, slot_table<SP>(a, ks[s]).h, G[s][0], G[s][1], G[s][2], C[s][0], C[s][1], C[s][2], acc);
            }
#if GMCS_PMOM
            moments_store(mom, acc);
#endif
        }
        acc[0] = lsum * 0.69314718055994531f;
    }
    store_partials<NACC>(a, acc, ww);
}

// ---- the same pass with the pipeline interleaved per neighbour slot: while
// slot s of point j is interpolated, slot s of point j + 1 is issued, so at
// most four slots' records (instead of six) and two points are in flight at a
// time -- fewer live registers for the same look-ahead.
// (BF16 gradient pass 1.542 -> 1.521 ms; FP32 1.566 -> 1.607 ms, so FP32 keeps the
// two whole stages). Since the two whole stages pair two slots' z rows, the 16-bit
// gradient passes take them too (BF16 1.526 ms either way; FP16 1.614 -> 1.611 ms;
// served BF16 at saturation 1.089e11 -> 1.101e11 evals/s), and so do the 16-bit value
// passes (BF16 0.938 -> 0.921 ms at 5 CTAs per SM; 0.949 ms at 4).
#ifndef GMCS_QPIPE32
#define GMCS_QPIPE32 0
#endif
#ifndef GMCS_QPIPE16
#define GMCS_QPIPE16 0
#endif
// the value passes likewise (FP32 interleaved: 1.011 -> 1.027 ms at 4 CTAs per SM,
// 1.070 ms at 5)
#ifndef GMCS_QPIPE32V
#define GMCS_QPIPE32V GMCS_QPIPE32
#endif
#ifndef GMCS_QPIPE16V
#define GMCS_QPIPE16V 0
#endif
template <int DT, bool GRAD>
constexpr bool qpipe() { return GRAD ? (DT == 0 ? GMCS_QPIPE32 : GMCS_QPIPE16) : (DT == 0 ? GMCS_QPIPE32V : GMCS_QPIPE16V); }

template <int DT>
struct SlotStage {
    float u[3], f[3];
    RawRec<DT> r;
};

template <int DT, bool GRAD, bool LL = true, bool SP = false>
__device__ __forceinline__ void pass3q_body(const PassArgs& a, int vb) {
    constexpr int NACC = GRAD ? kAccGrad : 1;
    constexpr bool kLL = LL || !GRAD;
    const WarpWork ww = warp_work(a, vb);
    const int i = ww.i, j0 = ww.j0, j1 = ww.j1;

    float acc[NACC];
#pragma unroll
    for (int e = 0; e < NACC; ++e) acc[e] = 0.f;

    if (i < a.P && j0 < j1) {
        Xf xf[3];
        const void* cells[3];
        const uint2* dirs[3];
        uint32_t ncx[3], ncy[3], ncz[3];
        {
            float Tt[12];
            load_pose(a.pose, a.ld, i, Tt);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const Slot sl = make_slot<SP>(a, i, a.nbr[(size_t)s * a.ld + i], Tt);
                xf[s] = slot_xf(sl);
                cells[s] = sl.cells;
                dirs[s] = sl.dir;
                ncx[s] = sl.ncx; ncy[s] = sl.ncy; ncz[s] = sl.ncz;
            }
        }
        const float eps = a.eps;
        float lsum = 0.f;
        float G[3][3], C[3][3];
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int d = 0; d < 3; ++d) G[s][d] = C[s][d] = 0.f;
        Moments mom;
        moments_zero(mom);

        auto issue = [&](SlotStage<DT>& st, float4 p, int s, bool live) {
            int cx, cy, cz;
            slot_point<DT, true>(xf[s], p, st.u[0], st.u[1], st.u[2], cx, cy, cz, st.f[0], st.f[1], st.f[2]);
            fetch_raw<DT, SP>(cells[s], dirs[s], ncx[s], ncy[s], ncz[s], cx, cy, cz, live, st.r);
        };
        // interpolate one slot of a point; returns its weight (gradient pass)
        auto use = [&](const SlotStage<DT>& st, int s, float& lprod) -> float {
            float v[8], w = 0.f, gx, gy, gz;
            unpack_raw<DT>(st.r, v);
            if constexpr (GRAD) {
                coef_interp<true, true, kLL>(v, st.f[0], st.f[1], st.f[2], eps, lprod, w, gx, gy, gz);
                G[s][0] += gx; G[s][1] += gy; G[s][2] += gz;
                C[s][0] = fmaf(st.u[1], gz, fmaf(-st.u[2], gy, C[s][0]));
                C[s][1] = fmaf(st.u[2], gx, fmaf(-st.u[0], gz, C[s][1]));
                C[s][2] = fmaf(st.u[0], gy, fmaf(-st.u[1], gx, C[s][2]));
            } else {
                coef_interp<false, true>(v, st.f[0], st.f[1], st.f[2], eps, lprod, w, gx, gy, gz);
            }
            return w;
        };
        SlotStage<DT> A[3], B[3];
        float4 pA = __ldg(a.scan + j0);
#pragma unroll
        for (int s = 0; s < 3; ++s) issue(A[s], pA, s, true);
        // one point: its three slots used while the next point's are issued
        auto step = [&](SlotStage<DT>* cur, float4 pc, SlotStage<DT>* nxt, float4 pn, bool live) {
            float lprod = 1.f, wsum = 0.f;
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                issue(nxt[s], pn, s, live);
                wsum += use(cur[s], s, lprod);
            }
            if constexpr (GRAD) moments_add(mom, wsum, pc);
            if constexpr (kLL) lsum += __log2f(lprod);
        };
        if constexpr (GMCS_P_AHEAD) {
            // each point loaded one step before the step that issues it
            float4 pB = __ldg(a.scan + (j0 + 1 < j1 ? j0 + 1 : j0));
            for (int j = j0;; j += 2) {   // j1 and the exits are uniform across the warp
                const bool m1 = j + 1 < j1, m2 = j + 2 < j1, m3 = j + 3 < j1;
                const float4 pN = __ldg(a.scan + (m2 ? j + 2 : j));
                step(A, pA, B, pB, m1);
                if (!m1) break;
                pA = pN;
                const float4 pM = __ldg(a.scan + (m3 ? j + 3 : j));
                step(B, pB, A, pA, m2);
                if (!m2) break;
                pB = pM;
            }
        } else {
            for (int j = j0;; j += 2) {   // j1 and the exits are uniform across the warp
                const bool m1 = j + 1 < j1;
                const float4 pB = __ldg(a.scan + (m1 ? j + 1 : j));
                step(A, pA, B, pB, m1);
                if (!m1) break;
                const bool m2 = j + 2 < j1;
                pA = __ldg(a.scan + (m2 ? j + 2 : j + 1));
                step(B, pB, A, pA, m2);
                if (!m2) break;
            }
        }
        if constexpr (GRAD) {
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                Slot sl;
                xf_slot(xf[s], sl);
                const int k = a.nbr[(size_t)s * a.ld + i];
                fold_slot(sl, slot_table<SP>(a, k).h, G[s][0], G[s][1], G[s][2], C[s][0], C[s][1], C[s][2], acc);
            }
            moments_store(mom, acc);
        }
        acc[0] = lsum * 0.69314718055994531f;
    }
    store_partials<NACC>(a, acc, ww);
}

// CTAs per SM the register allocation is sized for: the pipelined gradient
// pass fits 168 registers at 3 CTAs per SM; the unpipelined one uses ~150 and
// capping it at 128 costs 4 %; the value passes fit 128 at 4 CTAs per SM
// (unpipelined FP32 1.37 -> 1.25 ms; pipelined at 3 CTAs per SM: 1.63 ms).
#ifndef GMCS_VALUE_MINBLOCKS
#define GMCS_VALUE_MINBLOCKS 4
#endif
#ifndef GMCS_PIPE_GRAD_MINBLOCKS
#define GMCS_PIPE_GRAD_MINBLOCKS 3
#endif
#ifndef GMCS_PIPE_GRAD_MINBLOCKS16
#define GMCS_PIPE_GRAD_MINBLOCKS16 3
#endif
// The 16-bit value pass on dense tables (slot-interleaved body) fits 96 registers
// at 5 CTAs per SM (BF16 0.991 -> 0.941 ms; FP32 at 5 CTAs loses, 1.011 -> 1.091
// ms); on column-sparse tables (two whole stages) it would spill there.
#ifndef GMCS_VALUE_MINBLOCKS16
#define GMCS_VALUE_MINBLOCKS16 5
#endif
#ifndef GMCS_VALUE_MINBLOCKS32
#define GMCS_VALUE_MINBLOCKS32 GMCS_VALUE_MINBLOCKS
#endif
template <int DT, bool GRAD, bool SP = false>
constexpr int pass3_minblocks() {
    return GRAD ? (pass3_pipelined<DT, GRAD>() ? (DT == 0 ? GMCS_PIPE_GRAD_MINBLOCKS : GMCS_PIPE_GRAD_MINBLOCKS16)
                                               : GMCS_PASS3_MINBLOCKS)
                : (SP ? GMCS_VALUE_MINBLOCKS : DT == 0 ? GMCS_VALUE_MINBLOCKS32 : GMCS_VALUE_MINBLOCKS16);
}

template <int DT, bool GRAD, int UNROLL, bool LL = true, bool SP = false>
__device__ __forceinline__ void pass3_any(const PassArgs& a, int vb) {
    if constexpr (qpipe<DT, GRAD>() && pass3_pipelined<DT, GRAD>() && !(SP && kDirAhead))
        pass3q_body<DT, GRAD, LL, SP>(a, vb);
    else if constexpr (pass3_pipelined<DT, GRAD>()) pass3p_body<DT, GRAD, LL, SP>(a, vb);
    else pass3_body<DT, GRAD, UNROLL>(a, vb);
}

template <int DT, bool GRAD, int UNROLL, bool LL = true, bool SP = false>
__global__ void __launch_bounds__(kPassThreads, pass3_minblocks<DT, GRAD, SP>()) k_pass3(PassArgs a) {
    pass3_any<DT, GRAD, UNROLL, LL, SP>(a, blockIdx.x);
}

// ------------------------------------------------------------------ finish: sums, move (Eq. 5-7)

template <int NACC>
__device__ __forceinline__ void finish_sum(const FinishArgs& a, int i, float* acc) {
#pragma unroll
    for (int e = 0; e < NACC; ++e) acc[e] = 0.f;
    for (int g = 0; g < a.groups; ++g)
#pragma unroll
        for (int e = 0; e < NACC; ++e) acc[e] += a.part[((size_t)g * NACC + e) * a.ld + i];
}

// psi = (k H + lambda diag(k H))^-1 g, solved by Cholesky after symmetric
// Jacobi scaling, then clamped. H is overwritten.
__device__ bool damped_solve(float* H, float k, const float* g, const FinishArgs& a, float* psi) {
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
    // Cholesky with reciprocal pivots (one rsqrt per column instead of a square
    // root and divisions on the dependent chain)
    float L[36], iL[6];
#pragma unroll
    for (int e = 0; e < 36; ++e) L[e] = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float d = H[j * 6 + j];
#pragma unroll
        for (int q = 0; q < j; ++q) d -= L[j * 6 + q] * L[j * 6 + q];
        if (!(d > 0.f)) return false;
        const float inv = rsqrtf(d);
        iL[j] = inv;
        L[j * 6 + j] = d * inv;
#pragma unroll
        for (int r = j + 1; r < 6; ++r) {
            float s = H[r * 6 + j];
#pragma unroll
            for (int q = 0; q < j; ++q) s -= L[r * 6 + q] * L[j * 6 + q];
            L[r * 6 + j] = s * inv;
        }
    }
    float y[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        float s = b[r];
#pragma unroll
        for (int q = 0; q < r; ++q) s -= L[r * 6 + q] * y[q];
        y[r] = s * iL[r];
    }
#pragma unroll
    for (int r = 5; r >= 0; --r) {
        float s = y[r];
#pragma unroll
        for (int q = r + 1; q < 6; ++q) s -= L[q * 6 + r] * psi[q];
        psi[r] = s * iL[r];
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) psi[d] *= D[d];
    const float nw = sqrtf(psi[0] * psi[0] + psi[1] * psi[1] + psi[2] * psi[2]);
    const float nv = sqrtf(psi[3] * psi[3] + psi[4] * psi[4] + psi[5] * psi[5]);
    if (nw > a.theta_max) { const float sc = a.theta_max / nw; psi[0] *= sc; psi[1] *= sc; psi[2] *= sc; }
    if (nv > a.t_max) { const float sc = a.t_max / nv; psi[3] *= sc; psi[4] *= sc; psi[5] *= sc; }
    return true;
}

// Field model: psi = (H + lambda diag H)^-1 g with
// H = sigma^-2 [[tr Q I - Q, [S]x], [[S]x^T, W I]] from the moments.
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
    return damped_solve(H, 1.f / (a.sigma * a.sigma), g, a, psi);
}

// GICP model (Eq. 5-6): psi = (H + lambda diag H)^-1 b with H given by its upper
// triangle (21, row-major).
__device__ bool gn_step_h(const float* b, const float* hu, const FinishArgs& a, float* psi) {
#pragma unroll
    for (int d = 0; d < 6; ++d) psi[d] = 0.f;
    float H[36];
    int e = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
            H[r * 6 + c] = hu[e];
            H[c * 6 + r] = hu[e];
            ++e;
        }
    return damped_solve(H, 1.f, b, a, psi);
}

// GICP: the accumulators are [l, b (6), H upper triangle (21), inlier count];
// the gradient of l is 2 b where the pose does not move Omega (Eq. 3 has no 1/2).
template <bool GRAD, bool GICP>
__device__ __forceinline__ void finish_body(const FinishArgs& a, int vb, int vg) {
    const int i = vb * blockDim.x + threadIdx.x;
    if (i >= a.P) return;
    constexpr int NACC = GRAD ? (GICP ? kAccGicp : kAccGrad) : 1;
    float acc[NACC];
    finish_sum<NACC>(a, i, acc);
    if (a.out_ll) a.out_ll[i] = acc[0];
    if (!GRAD) {
        if (a.logw) a.logw[i] += (double)acc[0];
        return;
    } else {
        if (a.out_g)
            for (int d = 0; d < 6; ++d) a.out_g[(size_t)i * 6 + d] = GICP ? 2.f * acc[1 + d] : acc[1 + d];
        if (a.out_mom) {
            constexpr int NM = GICP ? 22 : 10;
            for (int d = 0; d < NM; ++d) a.out_mom[(size_t)i * NM + d] = acc[7 + d];
        }
        if (a.do_move) {
            // oldest (lowest-index) neighbour keyframe of this particle
            int o = -1;
            for (int s = 0; s < a.k_nb; ++s) {
                const int k = a.nbr[(size_t)s * a.ld + i];
                if (k >= 0 && (o < 0 || k < o)) o = k;
            }
            const bool loop = a.loop_recent <= 0 || (o >= 0 && o < a.K - a.loop_recent);
            float psi[6];
            if (loop && (GICP ? gn_step_h(acc + 1, acc + 7, a, psi) : gn_step(acc + 1, acc + 7, a, psi))) {
                float T[12], E[12], out[12];
                load_pose(a.pose, a.ld, i, T);
                se3_exp(psi, E);
                pose_mul(T, E, out);
                store_pose(a.pose, a.ld, i, out);
                if (a.propagate && o >= 0) {
                    // Eq. 8-10: keyframes after the oldest neighbour follow by their path-length share
                    const float Do = a.kf_path[o];
                    const float total = a.path_now - Do;
                    if (total > 0.f) {
                        for (int k = o + 1; k < a.K; ++k) {
                            const float r = fminf(fmaxf((a.kf_path[k] - Do) / total, 0.f), 1.f);
                            float pk[6];
#pragma unroll
                            for (int d = 0; d < 6; ++d) pk[d] = r * psi[d];
                            float* base = a.kf + (size_t)k * kPoseC * a.ld;
                            load_pose(base, a.ld, i, T);
                            se3_exp(pk, E);
                            pose_mul(T, E, out);
                            store_pose(base, a.ld, i, out);
                        }
                    }
                }
            }
        }
    }
}

template <bool GRAD, bool GICP>
__global__ void __launch_bounds__(128) k_finish(FinishArgs a) {
    finish_body<GRAD, GICP>(a, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ differentiable log-likelihood

// dst_i = T0_i exp(xi_i)  (xi: P x 6, row-major)
__global__ void __launch_bounds__(128) k_perturb(const float* __restrict__ pose0, const float* __restrict__ xi, int P,
                                                 size_t ld, float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    float x[6], T[12], E[12], out[12];
#pragma unroll
    for (int d = 0; d < 6; ++d) x[d] = xi[(size_t)i * 6 + d];
    load_pose(pose0, ld, i, T);
    se3_exp(x, E);
    pose_mul(T, E, out);
    store_pose(dst, ld, i, out);
}

// grad_xi_i = grad_ll_i * Jr(xi_i)^T g_i, with g_i the right-perturbation gradient at T0_i exp(xi_i)
__global__ void __launch_bounds__(128) k_chain(const float* __restrict__ xi, const float* __restrict__ g,
                                               const float* __restrict__ grad_ll, int P, float* __restrict__ grad_xi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    float x[6], J[36], gi[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        x[d] = xi[(size_t)i * 6 + d];
        gi[d] = g[(size_t)i * 6 + d];
    }
    se3_jr(x, J);
    const float s = grad_ll[i];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int r = 0; r < 6; ++r) acc += J[r * 6 + c] * gi[r];
        grad_xi[(size_t)i * 6 + c] = s * acc;
    }
}

// ------------------------------------------------------------------ batched launches

// Walk the virtual blocks of every session in a BatchList; the trailing barrier
// keeps a CTA's shared memory from being reused by the next virtual block while
// slower threads still read it.

__global__ void __launch_bounds__(256) k_scan_pack_b(const BatchList<ScanPackArgs>* L) {
    GMCS_BATCH_LOOP(L, const ScanPackArgs a = L->args[s]; scan_pack_body(a, vb, vg));
}

__global__ void __launch_bounds__(128) k_predict_b(const BatchList<PredictArgs>* L) {
    GMCS_BATCH_LOOP(L, const PredictArgs a = L->args[s]; predict_body(a, vb, vg));
}

__global__ void __launch_bounds__(128) k_select_b(const BatchList<SelectArgs>* L) {
    GMCS_BATCH_LOOP(L, const SelectArgs a = L->args[s]; select_body(a, vb, vg));
}

// The persistent loop costs the 16-bit gradient pass registers: bounded at 3
// CTAs per SM like the pipelined one (unbounded it takes 180, i.e. 2 per SM); the
// value passes as in the plain launch (the 16-bit dense one fits 96 registers at 5
// CTAs per SM with the two-stage body; the others would spill there).
template <int DT, bool GRAD, bool SP>
constexpr int pass3_b_minblocks() {
    return pass3_minblocks<DT, GRAD, SP>() < 3 ? 3 : pass3_minblocks<DT, GRAD, SP>();
}

// served frames never ask the gradient passes for the log-likelihood
template <int DT, bool GRAD, int UNROLL, bool SP = false>
__global__ void __launch_bounds__(kPassThreads, pass3_b_minblocks<DT, GRAD, SP>()) k_pass3_b(const BatchList<PassArgs>* L) {
    GMCS_BATCH_LOOP(L, const PassArgs a = L->args[s]; (pass3_any<DT, GRAD, UNROLL, !GRAD, SP>(a, vb)));
}

template <bool GRAD, bool GICP>
__global__ void __launch_bounds__(128) k_finish_b(const BatchList<FinishArgs>* L) {
    GMCS_BATCH_LOOP(L, const FinishArgs a = L->args[s]; (finish_body<GRAD, GICP>(a, vb, vg)));
}

// Persistent grids: every SM filled with as many CTAs as can be resident
// (from the occupancy API, computed once per kernel before any graph capture).
template <typename K>
static int persistent_grid(K kernel, int threads) {
    int per_sm = 0, dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * sms;
}

static int grid_scan_pack_b() {
    static const int g = persistent_grid(k_scan_pack_b, 256);
    return g;
}
static int grid_predict_b() {
    static const int g = persistent_grid(k_predict_b, 128);
    return g;
}
static int grid_select_b() {
    static const int g = persistent_grid(k_select_b, 128);
    return g;
}
template <int DT, bool G, bool SP>
static int grid_pass3_b() {
    static const int g = persistent_grid(k_pass3_b<DT, G, pass3_unroll<DT, G>(), SP>, kPassThreads);
    return g;
}
template <bool G, bool GICP>
static int grid_finish_b() {
    static const int g = persistent_grid(k_finish_b<G, GICP>, 128);
    return g;
}

void launch_scan_pack_b(const BatchList<ScanPackArgs>* L, cudaStream_t s) {
    k_scan_pack_b<<<grid_scan_pack_b(), 256, 0, s>>>(L);
}
void launch_predict_b(const BatchList<PredictArgs>* L, cudaStream_t s) {
    k_predict_b<<<grid_predict_b(), 128, 0, s>>>(L);
}
void launch_select_b(const BatchList<SelectArgs>* L, cudaStream_t s) {
    k_select_b<<<grid_select_b(), 128, 0, s>>>(L);
}

template <int DT, bool G, bool SP>
static void pass3_b(const BatchList<PassArgs>* L, cudaStream_t s) {
    k_pass3_b<DT, G, pass3_unroll<DT, G>(), SP><<<grid_pass3_b<DT, G, SP>(), kPassThreads, 0, s>>>(L);
}

template <bool SP>
static void pass3_b_any(const BatchList<PassArgs>* L, int dtype, bool grad, cudaStream_t s) {
    if (grad) {
        if (dtype == 0) pass3_b<0, true, SP>(L, s); else if (dtype == 1) pass3_b<1, true, SP>(L, s); else pass3_b<2, true, SP>(L, s);
    } else {
        if (dtype == 0) pass3_b<0, false, SP>(L, s); else if (dtype == 1) pass3_b<1, false, SP>(L, s); else pass3_b<2, false, SP>(L, s);
    }
}

void launch_pass3_b(const BatchList<PassArgs>* L, int dtype, bool grad, bool sparse, cudaStream_t s) {
    if (sparse) pass3_b_any<true>(L, dtype, grad, s);
    else pass3_b_any<false>(L, dtype, grad, s);
}

void launch_finish_b(const BatchList<FinishArgs>* L, bool grad, bool gicp, cudaStream_t s) {
    if (gicp) {
        if (grad) k_finish_b<true, true><<<grid_finish_b<true, true>(), 128, 0, s>>>(L);
        else k_finish_b<false, true><<<grid_finish_b<false, true>(), 128, 0, s>>>(L);
    } else {
        if (grad) k_finish_b<true, false><<<grid_finish_b<true, false>(), 128, 0, s>>>(L);
        else k_finish_b<false, false><<<grid_finish_b<false, false>(), 128, 0, s>>>(L);
    }
}

void prepare_filter_batched() {
    // evaluate every persistent grid size outside of any stream capture (no launch)
    grid_scan_pack_b();
    grid_predict_b();
    grid_select_b();
    grid_pass3_b<0, true, false>();
    grid_pass3_b<1, true, false>();
    grid_pass3_b<2, true, false>();
    grid_pass3_b<0, false, false>();
    grid_pass3_b<1, false, false>();
    grid_pass3_b<2, false, false>();
    grid_pass3_b<0, true, true>();
    grid_pass3_b<1, true, true>();
    grid_pass3_b<2, true, true>();
    grid_pass3_b<0, false, true>();
    grid_pass3_b<1, false, true>();
    grid_pass3_b<2, false, true>();
    grid_finish_b<true, false>();
    grid_finish_b<false, false>();
    grid_finish_b<true, true>();
    grid_finish_b<false, true>();
}

// ------------------------------------------------------------------ launchers

void launch_perturb(const float* pose0, const float* xi, int P, size_t ld, float* dst, cudaStream_t s) {
    if (P > 0) k_perturb<<<(P + 127) / 128, 128, 0, s>>>(pose0, xi, P, ld, dst);
}

void launch_chain(const float* xi, const float* g, const float* grad_ll, int P, float* grad_xi, cudaStream_t s) {
    if (P > 0) k_chain<<<(P + 127) / 128, 128, 0, s>>>(xi, g, grad_ll, P, grad_xi);
}

static int blocks_for(size_t n, int threads, int cap = 148 * 16) {
    size_t b = (n + threads - 1) / threads;
    if (b > (size_t)cap) b = cap;
    return (int)(b > 0 ? b : 1);
}

int grid_scan_pack(int n) { return blocks_for(n, 256); }
int grid_per_particle(int P) { return (P + 127) / 128; }
int grid_pass(const PassArgs& a) { return (a.ntiles + kPassTW - 1) / kPassTW * a.groups; }

void launch_scan_pack(const float* xyz, int n, float4* out, cudaStream_t s) {
    if (n > 0) k_scan_pack<<<grid_scan_pack(n), 256, 0, s>>>(ScanPackArgs{xyz, n, out});
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

template <int DT, bool G, int U, bool LL, bool SP>
static void launch_k_pass3(const PassArgs& a, int grid, cudaStream_t s) {
    k_pass3<DT, G, U, LL, SP><<<grid, kPassThreads, 0, s>>>(a);
}

void launch_pass(const PassArgs& a, int dtype, bool grad, cudaStream_t s) {
    const int grid = grid_pass(a);
    if (grid <= 0) return;
    // three neighbours (every particle then has all three slots filled): the fused kernel
    const bool three = GMCS_PASS3 && a.k_nb == 3;
#define GMCS_PASS3(DT, G, SP)                                                                                   \
    ((G && !a.want_ll) ? launch_k_pass3<DT, G, pass3_unroll<DT, G>(), false, SP>(a, grid, s)                  \
                       : launch_k_pass3<DT, G, pass3_unroll<DT, G>(), true, SP>(a, grid, s))
#define GMCS_PASS(DT, G)                                                                                        \
    (three ? (a.sparse ? GMCS_PASS3(DT, G, true) : GMCS_PASS3(DT, G, false))                                   \
           : k_pass<DT, G><<<grid, kPassThreads, 0, s>>>(a))
    if (grad) {
        if (dtype == 0) GMCS_PASS(0, true); else if (dtype == 1) GMCS_PASS(1, true); else GMCS_PASS(2, true);
    } else {
        if (dtype == 0) GMCS_PASS(0, false); else if (dtype == 1) GMCS_PASS(1, false); else GMCS_PASS(2, false);
    }
#undef GMCS_PASS
#undef GMCS_PASS3
}

void launch_finish(const FinishArgs& a, bool grad, cudaStream_t s) {
    if (a.P <= 0) return;
    const int g = (a.P + 127) / 128;
    if (a.model == 1) {
        if (grad) k_finish<true, true><<<g, 128, 0, s>>>(a);
        else k_finish<false, true><<<g, 128, 0, s>>>(a);
    } else {
        if (grad) k_finish<true, false><<<g, 128, 0, s>>>(a);
        else k_finish<false, false><<<g, 128, 0, s>>>(a);
    }
}

}  // namespace gmcs
