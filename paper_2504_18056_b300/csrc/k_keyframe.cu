// k_keyframe.cu -- keyframe insertion by overlap (Sec. III-E).
//
// Every keyframe carries an occupancy lattice of voxel edge kf_voxel over its
// points' bounding box (one voxel of margin). The overlap rate of a scan is the
// share of its points that, moved into the last keyframe's frame by the
// odometry, fall into an occupied voxel. The transform is taken in FP64 with
// every product and sum rounded separately, the voxel is floor((x - o) / h),
// so the count is exact.
#include <math.h>

#include "kernels.h"

namespace gmcs {

// Float -> int with the same order (negative floats have their magnitude bits flipped).
__device__ __forceinline__ int ordered(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__global__ void k_bbox(BBoxArgs a) {
    int mn[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, mx[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const float4 p = a.pts[i];
        const int v[3] = {ordered(p.x), ordered(p.y), ordered(p.z)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            mn[d] = min(mn[d], v[d]);
            mx[d] = max(mx[d], v[d]);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            mn[d] = min(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], off));
            mx[d] = max(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], off));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            atomicMin(a.mm + d, mn[d]);
            atomicMax(a.mm + 3 + d, mx[d]);
        }
    }
}

__device__ __forceinline__ bool voxel_of(double x, double y, double z, double ox, double oy, double oz, double h,
                                         int nx, int ny, int nz, size_t* v) {
    const double fx = floor((x - ox) / h), fy = floor((y - oy) / h), fz = floor((z - oz) / h);
    if (!(fx >= 0.0 && fx < (double)nx && fy >= 0.0 && fy < (double)ny && fz >= 0.0 && fz < (double)nz))
        return false;
    *v = ((size_t)fz * ny + (size_t)fy) * nx + (size_t)fx;
    return true;
}

__global__ void k_occ_fill(OccArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float4 p = a.pts[i];
    size_t v;
    if (voxel_of((double)p.x, (double)p.y, (double)p.z, a.ox, a.oy, a.oz, a.h, a.nx, a.ny, a.nz, &v)) a.occ[v] = 1;
}

__global__ void k_overlap(OverlapArgs a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool hit = false;
    if (j < a.n) {
        const float4 p = a.scan[j];
        const double px = (double)p.x, py = (double)p.y, pz = (double)p.z;
        double x[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            double s = __dadd_rn(__dmul_rn(a.T[4 * r], px), __dmul_rn(a.T[4 * r + 1], py));
            s = __dadd_rn(s, __dmul_rn(a.T[4 * r + 2], pz));
            x[r] = __dadd_rn(s, a.T[4 * r + 3]);
        }
        size_t v;
        hit = voxel_of(x[0], x[1], x[2], a.ox, a.oy, a.oz, a.h, a.nx, a.ny, a.nz, &v) && a.occ[v] != 0;
    }
    const unsigned b = __ballot_sync(0xffffffffu, hit);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(a.count, (unsigned)__popc(b));
}

__global__ void k_bbox_init(int* mm) {
    if (threadIdx.x < 3) mm[threadIdx.x] = 0x7fffffff;
    else if (threadIdx.x < 6) mm[threadIdx.x] = (int)0x80000000;
}

void launch_bbox(const BBoxArgs& a, cudaStream_t s) {
    k_bbox_init<<<1, 32, 0, s>>>(a.mm);
    if (a.n > 0) {
        int b = (a.n + 255) / 256;
        if (b > 148 * 4) b = 148 * 4;
        k_bbox<<<b, 256, 0, s>>>(a);
    }
}

void launch_occ_fill(const OccArgs& a, cudaStream_t s) {
    if (a.n > 0) k_occ_fill<<<(a.n + 255) / 256, 256, 0, s>>>(a);
}

void launch_overlap(const OverlapArgs& a, cudaStream_t s) {
    if (a.n > 0) k_overlap<<<(a.n + 255) / 256, 256, 0, s>>>(a);
}

}  // namespace gmcs
