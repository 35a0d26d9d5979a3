// k_order.cu -- a locality order of the particles for the lookup passes.
//
// A pass gives each warp 32 particles; when they are close in pose space their
// lookups read the same or neighbouring cells and L1 serves most of them. The
// filter's particles are close after resampling (copies of one parent sit side by
// side), but a set the caller perturbs or spreads (the differentiable
// log-likelihood of gmcs_loglik) is not. This order sorts the particles by a
// Morton code of their translation: a counting sort into 65,536 buckets (the top
// 16 bits of a 30-bit Morton code over the set's bounding box) with atomic
// scatter. The order within a bucket is arbitrary; results do not depend on it,
// since every particle is computed in one lane from its own data.
#include "kernels.h"

namespace gmcs {

namespace {

constexpr int kOrderBits = 16;
constexpr uint32_t kOrderBuckets = 1u << kOrderBits;
constexpr int kMm = 16;   // scratch words of the feature bounds (min 0..5, max 8..13)

// Features of a pose: its translation (1), or its translation and the skew part of
// its rotation scaled by a typical point range (2: a point at range r moves by
// about r times the rotation's change, so the six features are displacements in
// metres and share one quantisation scale).
#ifndef GMCS_ORDER_MODE
#define GMCS_ORDER_MODE 1
#endif
constexpr int kOrderDims = GMCS_ORDER_MODE == 2 ? 6 : 3;
#ifndef GMCS_ORDER_RANGE
#define GMCS_ORDER_RANGE 10.0f
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

// Exclusive scan of the bucket counts, in place: one CTA of 1024 threads, 64 each.
__global__ void __launch_bounds__(1024) k_order_scan(uint32_t* cnt) {
    constexpr int kPer = kOrderBuckets / 1024;
    __shared__ uint32_t part[1024];
    uint32_t* mine = cnt + threadIdx.x * kPer;
    uint32_t s = 0;
    for (int k = 0; k < kPer; ++k) s += mine[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan of the per-thread sums
        const uint32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0u;
    for (int k = 0; k < kPer; ++k) {
        const uint32_t c = mine[k];
        mine[k] = run;
        run += c;
    }
}

__global__ void k_order_scatter(const uint32_t* __restrict__ key, int P, uint32_t* __restrict__ cnt,
                                int* __restrict__ perm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    perm[atomicAdd(cnt + key[i], 1u)] = i;
}

}  // namespace

size_t order_scratch_words(int P) { return (size_t)kOrderBuckets + (size_t)P + kMm; }

void launch_locality_order(const float* pose, size_t ld, int P, uint32_t* scratch, int* perm, cudaStream_t s) {
    if (P <= 0) return;
    uint32_t* cnt = scratch;
    int* mm = reinterpret_cast<int*>(scratch + kOrderBuckets);
    uint32_t* key = scratch + kOrderBuckets + kMm;
    const int blocks = (P + 255) / 256;
    k_order_init<<<64, 256, 0, s>>>(mm, cnt);
    k_order_bbox<<<blocks, 256, 0, s>>>(pose, ld, P, mm);
    k_order_count<<<blocks, 256, 0, s>>>(pose, ld, P, mm, key, cnt);
    k_order_scan<<<1, 1024, 0, s>>>(cnt);
    k_order_scatter<<<blocks, 256, 0, s>>>(key, P, cnt, perm);
}

}  // namespace gmcs
