// common.cuh -- device-side types and helpers of the particle-update library.
//
// Layouts (device memory, all particle arrays padded to the context's
// particle capacity `ld`):
//   current poses       float [12][ld]          component c of particle i at c*ld + i
//   keyframe poses      float [K][12][ld]       (k*12 + c)*ld + i
//   neighbour indices   int   [k_nb][ld]
//   log-weights         double[ld]
//   scan                float4[N]               (x, y, z, 0) in the sensor frame
//   tables              per keyframe, one record per lattice cell, cells ordered
//                       x fastest, holding the 8 coefficients of the cell's
//                       trilinear polynomial: FP32 records are 32 B (two float4),
//                       BF16/FP16 records 16 B (one uint4, two coefficients per
//                       32-bit word).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gmcs {

constexpr int kPoseC = 12;   // row-major 3x4 [R | t]
constexpr int kMaxNb = 8;

struct TableDesc {
    const void* cells;   // packed cell records
    const uint2* dir;    // column-sparse tables: per (x, y) column (first record, zlo | count << 16); dense: null
    float ox, oy, oz;    // lattice origin in the keyframe frame
    float inv_h;         // 1 / h
    int ncx, ncy, ncz;   // cells per axis (vertices - 1)
    int dtype;           // 0 f32, 1 bf16, 2 f16
    float h;
    int pad;
};
static_assert(sizeof(TableDesc) == 56, "TableDesc layout");

// ---------------------------------------------------------------- pose algebra

// C = A * B for row-major 3x4 poses held in registers.
__device__ __forceinline__ void pose_mul(const float* A, const float* B, float* C) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float a0 = A[r * 4 + 0], a1 = A[r * 4 + 1], a2 = A[r * 4 + 2];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float s = a0 * B[0 * 4 + c] + a1 * B[1 * 4 + c] + a2 * B[2 * 4 + c];
            if (c == 3) s += A[r * 4 + 3];
            C[r * 4 + c] = s;
        }
    }
}

// Relative pose rel = inv(Tk) * Tt: R = Rk^T Rt, t = Rk^T (tt - tk)  (Eq. 4).
__device__ __forceinline__ void pose_rel(const float* Tk, const float* Tt, float* rel) {
    const float dx = Tt[3] - Tk[3], dy = Tt[7] - Tk[7], dz = Tt[11] - Tk[11];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            rel[r * 4 + c] = Tk[0 * 4 + r] * Tt[0 * 4 + c] + Tk[1 * 4 + r] * Tt[1 * 4 + c] + Tk[2 * 4 + r] * Tt[2 * 4 + c];
        rel[r * 4 + 3] = Tk[0 * 4 + r] * dx + Tk[1 * 4 + r] * dy + Tk[2 * 4 + r] * dz;
    }
}

// exp of xi = [omega; v] in SE(3): R = I + a W + b W^2, t = (I + b W + c W^2) v with
// a = sin th / th, b = (1 - cos th) / th^2 = 2 (sin(th/2) / th)^2, c = (th - sin th) / th^3;
// power series where the closed forms lose float precision.
__device__ __forceinline__ void se3_exp(const float* xi, float* T) {
    const float wx = xi[0], wy = xi[1], wz = xi[2];
    const float th2 = wx * wx + wy * wy + wz * wz;
    float a, b, c;
    if (th2 < 1e-6f) {
        a = 1.f - th2 * (1.f / 6.f);
        b = 0.5f - th2 * (1.f / 24.f);
        c = (1.f / 6.f) - th2 * (1.f / 120.f);
    } else {
        const float th = sqrtf(th2);
        const float sh = sinf(0.5f * th) / th;
        a = sinf(th) / th;
        b = 2.f * sh * sh;
        if (th2 < 0.25f)
            c = (1.f / 6.f) - th2 * ((1.f / 120.f) - th2 * ((1.f / 5040.f) - th2 * (1.f / 362880.f)));
        else
            c = (th - sinf(th)) / (th2 * th);
    }
    // W^2 = w w^T - th2 I
    const float w[3] = {wx, wy, wz};
    const float W[9] = {0.f, -wz, wy, wz, 0.f, -wx, -wy, wx, 0.f};
    float V[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float W2 = w[r] * w[k] - (r == k ? th2 : 0.f);
            const float I = (r == k) ? 1.f : 0.f;
            T[r * 4 + k] = I + a * W[r * 3 + k] + b * W2;
            V[r * 3 + k] = I + b * W[r * 3 + k] + c * W2;
        }
#pragma unroll
    for (int r = 0; r < 3; ++r) T[r * 4 + 3] = V[r * 3 + 0] * xi[3] + V[r * 3 + 1] * xi[4] + V[r * 3 + 2] * xi[5];
}

// Right Jacobian of SE(3) for xi = [omega; v]: exp(xi + d) = exp(xi) exp(Jr d) to
// first order. Jr(xi) = Jl(-xi); the left Jacobian in this order is [[J, 0], [Q, J]]
// with J = I + b W + c1 W^2 (W = phi^) and, for rho = v, phi = omega,
//   Q = rho^/2 + c1 (W R + R W + W R W) + c2 (W W R + R W W - 3 W R W) + c3 (W R W W + W W R W),
//   c1 = (th - sin th)/th^3, c2 = (th^2 + 2 cos th - 2)/(2 th^4), c3 = (2 th - 3 sin th + th cos th)/(2 th^5)
// (Barfoot, State Estimation for Robotics); power series below th = 0.5 in float.
__device__ __forceinline__ void mat3mul(const float* A, const float* B, float* C) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) C[r * 3 + c] = A[r * 3] * B[c] + A[r * 3 + 1] * B[3 + c] + A[r * 3 + 2] * B[6 + c];
}

__device__ __forceinline__ void se3_jr(const float* xi, float* J) {
    const float px = -xi[0], py = -xi[1], pz = -xi[2];
    const float rx = -xi[3], ry = -xi[4], rz = -xi[5];
    const float th2 = px * px + py * py + pz * pz;
    float b, c1, c2, c3;
    if (th2 < 0.25f) {
        b = 0.5f - th2 * (1.f / 24.f) + th2 * th2 * (1.f / 720.f) - th2 * th2 * th2 * (1.f / 40320.f);
        c1 = (1.f / 6.f) - th2 * (1.f / 120.f) + th2 * th2 * (1.f / 5040.f) - th2 * th2 * th2 * (1.f / 362880.f);
        c2 = (1.f / 24.f) - th2 * (1.f / 720.f) + th2 * th2 * (1.f / 40320.f);
        c3 = (1.f / 120.f) - th2 * (1.f / 2520.f) + th2 * th2 * (1.f / 120960.f);
    } else {
        const float th = sqrtf(th2), sn = sinf(th), cs = cosf(th);
        b = (1.f - cs) / th2;
        c1 = (th - sn) / (th2 * th);
        c2 = (th2 + 2.f * cs - 2.f) / (2.f * th2 * th2);
        c3 = (2.f * th - 3.f * sn + th * cs) / (2.f * th2 * th2 * th);
    }
    const float W[9] = {0.f, -pz, py, pz, 0.f, -px, -py, px, 0.f};
    const float R[9] = {0.f, -rz, ry, rz, 0.f, -rx, -ry, rx, 0.f};
    float WW[9], WR[9], RW[9], WRW[9], WWR[9], RWW[9], WRWW[9], WWRW[9];
    mat3mul(W, W, WW);
    mat3mul(W, R, WR);
    mat3mul(R, W, RW);
    mat3mul(WR, W, WRW);
    mat3mul(W, WR, WWR);
    mat3mul(RW, W, RWW);
    mat3mul(WRW, W, WRWW);
    mat3mul(W, WRW, WWRW);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int e = r * 3 + c;
            const float Jso = (r == c ? 1.f : 0.f) + b * W[e] + c1 * WW[e];
            const float Q = 0.5f * R[e] + c1 * (WR[e] + RW[e] + WRW[e]) + c2 * (WWR[e] + RWW[e] - 3.f * WRW[e]) +
                            c3 * (WRWW[e] + WWRW[e]);
            J[r * 6 + c] = Jso;
            J[r * 6 + 3 + c] = 0.f;
            J[(3 + r) * 6 + c] = Q;
            J[(3 + r) * 6 + 3 + c] = Jso;
        }
}

__device__ __forceinline__ void load_pose(const float* __restrict__ base, size_t ld, int i, float* T) {
#pragma unroll
    for (int c = 0; c < kPoseC; ++c) T[c] = base[(size_t)c * ld + i];
}

__device__ __forceinline__ void store_pose(float* __restrict__ base, size_t ld, int i, const float* T) {
#pragma unroll
    for (int c = 0; c < kPoseC; ++c) base[(size_t)c * ld + i] = T[c];
}

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten rounds,
// each two 32x32 -> 64-bit products mixed into the counter, key advanced by the
// Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

constexpr uint32_t kTagNormal = 0x4E4F524Du;    // 'NORM': motion-noise counters
constexpr uint32_t kTagResample = 0x52534D50u;  // 'RSMP': resampling offset counter

// (k + 1/2) 2^-23 from the top 23 bits: exactly representable in float.
__device__ __forceinline__ float u23(uint32_t x) { return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f); }

// Six standard normals of particle i at frame t (Box-Muller on three uniform pairs).
__device__ __forceinline__ void normal6(uint64_t seed, uint32_t i, uint32_t t, float* z) {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 a = philox4x32_10(make_uint4(i, t, 0u, kTagNormal), key);
    const uint4 b = philox4x32_10(make_uint4(i, t, 1u, kTagNormal), key);
    const uint32_t x[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const float r = sqrtf(-2.f * logf(u23(x[2 * p])));
        float s, c;
        sincospif(2.f * u23(x[2 * p + 1]), &s, &c);
        z[2 * p] = r * c;
        z[2 * p + 1] = r * s;
    }
}

// ---------------------------------------------------------------- table cells

// Corner (dx, dy, dz) of a cell in the 8-value corner arrays the table build
// and the vertex read-back use: the x = 0 face first, z pairs adjacent.
__host__ __device__ constexpr int rec_slot(int dx, int dy, int dz) { return dz + 2 * dy + 4 * dx; }

// A cell record holds the 8 coefficients of the cell's trilinear polynomial in
// the in-cell fraction (x, y, z) in [0, 1)^3,
//   L = c0 + c1 x + c2 y + c3 z + c4 xy + c5 xz + c6 yz + c7 xyz,
// in the order (c4, c2), (c7, c6), (c1, c0), (c5, c3) that the packed evaluation
// reads as float pairs. Slot of coefficient i in that order:
__host__ __device__ constexpr int coef_slot(int i) {
    return i == 0 ? 5 : i == 1 ? 4 : i == 2 ? 1 : i == 3 ? 7 : i == 4 ? 0 : i == 5 ? 6 : i == 6 ? 3 : 2;
}

// Coefficients from the corner values v[rec_slot(dx, dy, dz)] by inclusion-
// exclusion over the corners, into record order. FP32 differences of differences
// (the field is in [0, 1]: each coefficient within ~2.4e-7 of its exact value);
// FP64 here made the table build 5x slower on this part's FP64 rate.
__device__ __forceinline__ void corners_to_coef(const float* v, float* rec) {
    const float v000 = v[rec_slot(0, 0, 0)], v100 = v[rec_slot(1, 0, 0)], v010 = v[rec_slot(0, 1, 0)];
    const float v001 = v[rec_slot(0, 0, 1)], v110 = v[rec_slot(1, 1, 0)], v101 = v[rec_slot(1, 0, 1)];
    const float v011 = v[rec_slot(0, 1, 1)], v111 = v[rec_slot(1, 1, 1)];
    const float c[8] = {v000,
                         v100 - v000,
                         v010 - v000,
                         v001 - v000,
                         (v110 - v100) - (v010 - v000),
                         (v101 - v100) - (v001 - v000),
                         (v011 - v010) - (v001 - v000),
                         ((v111 - v110) - (v101 - v100)) - ((v011 - v010) - (v001 - v000))};
#pragma unroll
    for (int i = 0; i < 8; ++i) rec[coef_slot(i)] = c[i];
}

// The value at corner (dx, dy, dz) of a coefficient record in record order (in
// double, rounded once).
__host__ __device__ inline float coef_corner(const float* rec, int dx, int dy, int dz) {
    double s = rec[coef_slot(0)];
    if (dx) s += rec[coef_slot(1)];
    if (dy) s += rec[coef_slot(2)];
    if (dz) s += rec[coef_slot(3)];
    if (dx && dy) s += rec[coef_slot(4)];
    if (dx && dz) s += rec[coef_slot(5)];
    if (dy && dz) s += rec[coef_slot(6)];
    if (dx && dy && dz) s += rec[coef_slot(7)];
    return (float)s;
}

// 16-bit records: word e (e = 0..3) of the uint4 holds record slots e (high
// half) and 4 + e (low half). FP16: both halves are binary16 values, rounded to
// nearest. BF16: the low half is a bfloat16 value B (rounded to nearest), and the
// whole 32-bit word, read as an FP32 number, is the other coefficient A -- the
// word is the one with low half B whose FP32 value is nearest to A, so A keeps
// bfloat16 precision (within half a bfloat16 ulp) and a lookup widens only the
// four low halves (one shift each) instead of all eight values.
__device__ __forceinline__ uint32_t bf16_hi_word(float A, uint32_t lo16) {
    const uint32_t base = (__float_as_uint(A) & 0xFFFF0000u) | lo16;
    uint32_t best = base;
    double err = fabs((double)A - (double)__uint_as_float(base));
    const uint32_t mag = (base >> 16) & 0x7FFFu;   // exponent and upper mantissa of the high half
    if (mag > 0u) {
        const uint32_t c = base - 0x10000u;
        const double e = fabs((double)A - (double)__uint_as_float(c));
        if (e < err) { err = e; best = c; }
    }
    if (mag < 0x7F7Fu) {
        const uint32_t c = base + 0x10000u;
        const double e = fabs((double)A - (double)__uint_as_float(c));
        if (e < err) { err = e; best = c; }
    }
    return best;
}

// Encode a record (8 FP32 coefficients in record order) as a 16-bit record.
__device__ __forceinline__ uint4 encode_rec16(const float* r, int dtype) {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (dtype == 1) {
            const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(r[4 + e]));
            w[e] = bf16_hi_word(r[e], lo);
        } else {
            const uint32_t lo = __half_as_ushort(__float2half_rn(r[4 + e]));
            const uint32_t hi = __half_as_ushort(__float2half_rn(r[e]));
            w[e] = lo | (hi << 16);
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Decode a 16-bit record into the 8 coefficients in record order.
template <int DT>
__device__ __forceinline__ void decode_rec16(uint4 q, float* r) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (DT == 1) {
            r[e] = __uint_as_float(w[e]);
            r[4 + e] = __uint_as_float(w[e] << 16);
        } else {
            r[e] = __half2float(__ushort_as_half((unsigned short)(w[e] >> 16)));
            r[4 + e] = __half2float(__ushort_as_half((unsigned short)(w[e] & 0xFFFFu)));
        }
    }
}

// One 32-byte FP32 cell record (32-byte aligned) in a single 256-bit read-only
// load: one L1 tag lookup per record instead of two for a pair of 128-bit
// loads (lookup passes 1.77 -> 1.72 ms gradient, 1.19 -> 1.16 ms value).
__device__ __forceinline__ void ld_record32(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Column-sparse tables store, for every tile of kColTile x kColTile (x, y) columns
// of cells, only the cells from the lowest to the highest z layer in which any of
// the tile's cells has a nonzero polynomial (the field is zero farther than r_t
// from every keyframe point, so a tile holds one short run of layers near the
// surfaces it crosses). dir[(cy / T) * ntx + cx / T] = (index of the run's first
// record, zlo | layers << 16), ntx = ceil(ncx / T); within the run the records go
// layer by layer, each layer's T x T cells x fastest. A cell outside the run reads
// as zero. Returns whether (cx, cy, cz) is stored, and its record index.
#ifndef GMCS_COL_TILE_LOG2
#define GMCS_COL_TILE_LOG2 0
#endif
constexpr int kColTileLog2 = GMCS_COL_TILE_LOG2;
constexpr int kColTile = 1 << kColTileLog2;

__host__ __device__ inline uint32_t col_tiles(uint32_t n) { return (n + kColTile - 1) >> kColTileLog2; }

__device__ __forceinline__ bool col_cell(const uint2* __restrict__ dir, uint32_t ncx, uint32_t ncy, int cx, int cy,
                                         int cz, uint32_t& idx) {
    if (!(((uint32_t)cx < ncx) & ((uint32_t)cy < ncy))) return false;
    const uint32_t tx = (uint32_t)cx >> kColTileLog2, ty = (uint32_t)cy >> kColTileLog2;
    const uint2 d = __ldg(dir + (ty * col_tiles(ncx) + tx));
    const uint32_t rel = (uint32_t)cz - (d.y & 0xFFFFu);
    idx = d.x + ((rel << (2 * kColTileLog2)) | (((uint32_t)cy & (kColTile - 1)) << kColTileLog2) |
                 ((uint32_t)cx & (kColTile - 1)));
    return rel < (d.y >> 16);
}

// The coefficient record of cell `idx` widened to float in record order; zeros
// without a load when !valid.
template <int DT>
__device__ __forceinline__ void load_cell(const void* __restrict__ cells, uint32_t idx, bool valid, float* v) {
    if (DT == 0) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (valid) ld_record32(reinterpret_cast<const float4*>(cells) + 2 * (size_t)idx, a, b);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        if (valid) q = __ldg(reinterpret_cast<const uint4*>(cells) + idx);
        decode_rec16<DT>(q, v);
    }
}

}  // namespace gmcs
