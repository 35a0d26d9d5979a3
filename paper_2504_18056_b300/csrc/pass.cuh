// pass.cuh -- work split and partial sums shared by the lookup passes
// (voxel likelihood field and GICP): a CTA's warps cover kPassTW particle tiles
// of 32 lanes x kPassCW point chunks; partial sums go to [group][acc][particle]
// scratch that the finish kernel adds in a fixed order.
#pragma once
#include "kernels.h"

namespace gmcs {

// Map a CTA warp to (particle index, point range, chunk group).
struct WarpWork {
    int i, j0, j1, tg, cg;
};

__device__ __forceinline__ WarpWork warp_work(const PassArgs& a, int vb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntg = (a.ntiles + kPassTW - 1) / kPassTW;
    WarpWork w;
    w.tg = vb % ntg;
    w.cg = vb / ntg;
    const int tile = w.tg * kPassTW + warp % kPassTW;
    const int chunk = w.cg * kPassCW + warp / kPassTW;
    w.i = tile * 32 + lane;
    if (a.perm && w.i < a.P) w.i = a.perm[w.i];   // the lanes' particles in the given order
    w.j0 = min(chunk * a.chunk_len, a.N);
    w.j1 = min(w.j0 + a.chunk_len, a.N);
    return w;
}

// CTA partial sums -> scratch [group][acc][particle]; warps sharing a tile add
// their chunks in a fixed order.
template <int NACC>
__device__ __forceinline__ void store_partials(const PassArgs& a, const float* acc, const WarpWork& ww) {
    if constexpr (kPassCW == 1) {
        if (ww.i < a.P)
#pragma unroll
            for (int e = 0; e < NACC; ++e) a.part[((size_t)ww.cg * NACC + e) * a.ld + ww.i] = acc[e];
    } else {
        __shared__ float red[kPassCW][NACC][kPassTW * 32];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int col = (warp % kPassTW) * 32 + lane;
#pragma unroll
        for (int e = 0; e < NACC; ++e) red[warp / kPassTW][e][col] = acc[e];
        __syncthreads();
        const int base = ww.tg * kPassTW * 32;
        for (int t = threadIdx.x; t < NACC * kPassTW * 32; t += kPassThreads) {
            const int e = t / (kPassTW * 32), l = t % (kPassTW * 32);
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < kPassCW; ++c) s += red[c][e][l];
            if (base + l < a.P) a.part[((size_t)ww.cg * NACC + e) * a.ld + (a.perm ? a.perm[base + l] : base + l)] = s;
        }
    }
}


}  // namespace gmcs
