// k_order.cu -- a locality order of the particles for the lookup passes.
//
// A pass gives each warp 32 particles; when they are close in pose space their
// lookups read the same or neighbouring cells and L1 serves most of them. The
// filter's particles are close after resampling (copies of one parent sit side by
// side), but a set the caller perturbs or spreads (the differentiable
// log-likelihood of gmcs_loglik) is not. This order sorts the particles by a
// Morton code of six pose features -- the translation and the rotation's skew part
// times a typical point range of 5 m, all in metres on one scale, 5 bits each over
// the set's bounding box -- as a counting sort into 2^20 buckets (the code's top
// 20 bits) with atomic scatter. (On 100,000 poses spread 0.3 m / 5 deg, 4,096
// points, 50 tables: forward / backward 13.0 / 13.4 ms with a translation-only
// order into 2^16 buckets, 11.4 / 11.3 ms with the six features into 2^16, 10.7 /
// 10.3 ms into 2^20; a range of 2, 3, 10 or 20 m orders worse than 5.) The order
// within a bucket is arbitrary; results do not depend on it, since every particle
// is computed in one lane from its own data.
#include "kernels.h"

namespace gmcs {

namespace {

#ifndef GMCS_ORDER_BITS
#define GMCS_ORDER_BITS 20
#endif
constexpr int kOrderBits = GMCS_ORDER_BITS;
constexpr uint32_t kOrderBuckets = 1u << kOrderBits;
constexpr int kMm = 16;   // scratch words of the feature bounds (min 0..5, max 8..13)

// Features of a pose: its translation (1), or its translation and the skew part of
// its rotation scaled by a typical point range (2: a point at range r moves by
// about r times the rotation's change, so the six features are displacements in
// metres and share one quantisation scale).
#ifndef GMCS_ORDER_MODE
#define GMCS_ORDER_MODE 2
#endif
constexpr int kOrderDims = GMCS_ORDER_MODE == 2 ? 6 : 3;
#ifndef GMCS_ORDER_RANGE
#define GMCS_ORDER_RANGE 5.0f
#endif

__device__ __forceinline__ void pose_features(const float* __restrict__ pose, size_t ld, int i, float* f) {
    f[0] = pose[3 * ld + i];
    f[1] = pose[7 * ld + i];
    f[2] = pose[11 * ld + i];
    if constexpr (kOrderDims == 6) {
        const float h = 0.5f * GMCS_ORDER_RANGE;
        f[3] = h * (pose[9 * ld + i] - pose[6 * ld + i]);    // R21 - R12
        f[4] = h * (pose[2 * ld + i] - pose[8 * ld + i]);    // R02 - R20
        f[5] = h * (pose[4 * ld + i] - pose[1 * ld + i]);    // R10 - R01
    }
}

// Spread the low 5 bits of x to every sixth bit.
__device__ __forceinline__ uint32_t spread6(uint32_t x) {
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b) m |= ((x >> b) & 1u) << (6 * b);
    return m;
}

// An int whose signed order is the float order (for atomic min / max).
__device__ __forceinline__ int ordered(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float unordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Spread the low 10 bits of x to every third bit.
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_order_init(int* mm, uint32_t* cnt) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < kOrderBuckets; k += gridDim.x * blockDim.x) cnt[k] = 0;
    if (blockIdx.x == 0 && threadIdx.x < kMm) mm[threadIdx.x] = threadIdx.x < 8 ? 0x7fffffff : (int)0x80000000;
}

__global__ void k_order_bbox(const float* __restrict__ pose, size_t ld, int P, int* mm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float t[kOrderDims];
#pragma unroll
    for (int a = 0; a < kOrderDims; ++a) t[a] = 0.f;
    const bool in = i < P;
    if (in) pose_features(pose, ld, i, t);
#pragma unroll
    for (int a = 0; a < kOrderDims; ++a) {
        int lo = in && isfinite(t[a]) ? ordered(t[a]) : 0x7fffffff;
        int hi = in && isfinite(t[a]) ? ordered(t[a]) : (int)0x80000000;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(mm + a, lo);
            atomicMax(mm + 8 + a, hi);
        }
    }
}

__global__ void k_order_count(const float* __restrict__ pose, size_t ld, int P, const int* __restrict__ mm,
                              uint32_t* __restrict__ key, uint32_t* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    uint32_t m = 0;
    if constexpr (kOrderDims == 3) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float lo = unordered(mm[a]), hi = unordered(mm[8 + a]);
            const float t = pose[(4 * a + 3) * ld + i];
            const float span = hi - lo;
            float q = span > 0.f ? (t - lo) / span * 1023.f : 0.f;
            q = isfinite(q) ? fminf(fmaxf(q, 0.f), 1023.f) : 0.f;
            m |= spread3((uint32_t)q) << a;
        }
    } else {
        // six features on one scale: the widest span gets 32 steps
        float f[6], wmax = 0.f;
        pose_features(pose, ld, i, f);
#pragma unroll
        for (int a = 0; a < 6; ++a) wmax = fmaxf(wmax, unordered(mm[8 + a]) - unordered(mm[a]));
        const float sc = wmax > 0.f ? 31.f / wmax : 0.f;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            float q = (f[a] - unordered(mm[a])) * sc;
            q = isfinite(q) ? fminf(fmaxf(q, 0.f), 31.f) : 0.f;
            m |= spread6((uint32_t)q) << (5 - a);
        }
    }
    const uint32_t k = m >> (30 - kOrderBits);
    key[i] = k;
    atomicAdd(cnt + k, 1u);
}

// Exclusive scan of v over a CTA of 1024 threads; total: the CTA's sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& total) {
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;   // inclusive within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;   // inclusive over the warps
    }
    __syncthreads();
    total = wsum[31];
    return (warp > 0 ? wsum[warp - 1] : 0u) + x - v;
}

// Exclusive scan of the bucket counts in place, in three launches: each CTA scans
// 1,024 counts and leaves its total, one CTA scans the totals, each CTA adds its
// offset.
__global__ void __launch_bounds__(1024) k_order_scan_tiles(uint32_t* cnt, uint32_t* tot) {
    const uint32_t k = blockIdx.x * 1024u + threadIdx.x;
    uint32_t t;
    cnt[k] = block_exclusive_scan(cnt[k], t);
    if (threadIdx.x == 0) tot[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_order_scan_totals(uint32_t* tot, int n) {
    uint32_t t;
    const uint32_t v = (int)threadIdx.x < n ? tot[threadIdx.x] : 0u;
    const uint32_t e = block_exclusive_scan(v, t);
    if ((int)threadIdx.x < n) tot[threadIdx.x] = e;
}

__global__ void __launch_bounds__(1024) k_order_scan_add(uint32_t* cnt, const uint32_t* tot) {
    cnt[blockIdx.x * 1024u + threadIdx.x] += tot[blockIdx.x];
}

__global__ void k_order_scatter(const uint32_t* __restrict__ key, int P, uint32_t* __restrict__ cnt,
                                int* __restrict__ perm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    perm[atomicAdd(cnt + key[i], 1u)] = i;
}

}  // namespace

constexpr uint32_t kOrderTiles = kOrderBuckets / 1024;
static_assert(kOrderBuckets % 1024 == 0 && kOrderTiles <= 1024, "bucket tiles of the scan");

size_t order_scratch_words(int P) { return (size_t)kOrderBuckets + kMm + kOrderTiles + (size_t)P; }

void launch_locality_order(const float* pose, size_t ld, int P, uint32_t* scratch, int* perm, cudaStream_t s) {
    if (P <= 0) return;
    uint32_t* cnt = scratch;
    int* mm = reinterpret_cast<int*>(scratch + kOrderBuckets);
    uint32_t* tot = scratch + kOrderBuckets + kMm;
    uint32_t* key = tot + kOrderTiles;
    const int blocks = (P + 255) / 256;
    k_order_init<<<64, 256, 0, s>>>(mm, cnt);
    k_order_bbox<<<blocks, 256, 0, s>>>(pose, ld, P, mm);
    k_order_count<<<blocks, 256, 0, s>>>(pose, ld, P, mm, key, cnt);
    k_order_scan_tiles<<<kOrderTiles, 1024, 0, s>>>(cnt, tot);
    k_order_scan_totals<<<1, 1024, 0, s>>>(tot, (int)kOrderTiles);
    k_order_scan_add<<<kOrderTiles, 1024, 0, s>>>(cnt, tot);
    k_order_scatter<<<blocks, 256, 0, s>>>(key, P, cnt, perm);
}

}  // namespace gmcs
