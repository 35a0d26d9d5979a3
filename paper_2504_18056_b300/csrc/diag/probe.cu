// probe.cu -- gather-bandwidth and FP32 FMA-rate calibration (no counterpart in
// the paper).
//
// The lookup pass reads one cell record per lookup from tables whose touched
// cells mostly stay in L1/L2, so neither the HBM copy rate nor the FP32 peak
// alone bounds it. This probe measures the rate of random record gathers from a
// buffer of a given size (an L2-resident size gives the L2 gather ceiling):
// every thread reads `per_thread` records at pseudo-random indices (a 32-bit
// integer hash of its global index and the step, no index traffic) with the
// loads the lookup pass issues (one 256-bit load per 32-byte record, one
// 128-bit load per 16-byte record), and folds them into a sink.
#include <cuda_runtime.h>

#include "../../../include/gmcs_diag.h"

namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    // integer finaliser (xor-shift-multiply), used only to scatter indices
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <int VEC>   // 16-byte vectors per record: 2 (32 B) or 1 (16 B)
__global__ void __launch_bounds__(256) k_probe_gather(const float4* __restrict__ buf, uint32_t nrec, int per_thread,
                                                      float* __restrict__ sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    for (int s = 0; s < per_thread; ++s) {
        const uint32_t r = mix32(tid * 0x9e3779b9u + (uint32_t)s * 0x85ebca6bu) % nrec;
        const float4* p = buf + (size_t)r * VEC;
        if constexpr (VEC == 2) {
            float4 a, b;
            asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                : "l"(p));
            acc += (a.x + a.y + a.z + a.w) + (b.x + b.y + b.z + b.w);
        } else {
            const float4 q = __ldg(p);
            acc += q.x + q.y + q.z + q.w;
        }
    }
    sink[tid] = acc;
}

// Eight independent FMA chains per thread (x <- x a + b with |a| < 1, so the
// values stay finite): with a few warps per scheduler the FMA pipe never waits on
// a chain's latency.
__global__ void __launch_bounds__(256) k_probe_ffma(float* __restrict__ sink, int iters, float a, float b) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (float)(tid & 1023) * 1e-3f + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    sink[tid] = s;
}

}  // namespace

extern "C" int gmcs_probe_ffma(void* cuda_stream, double* tflops, int* sm_count) {
    if (!tflops) return GMCS_E_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return GMCS_E_CUDA;
    }
    if (sm_count) *sm_count = sms;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GMCS_OK;
    if (cudaMalloc((void**)&sink, sizeof(float) * (size_t)blocks * threads) != cudaSuccess) {
        cudaGetLastError();
        return GMCS_E_OOM;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = GMCS_E_CUDA;
    if (!rc) {
        float best = 1e30f;
        for (int it = 0; it < 6; ++it) {   // 1 warm-up + 5 timed, best kept
            cudaEventRecord(e0, s);
            k_probe_ffma<<<blocks, threads, 0, s>>>(sink, iters, 0.9999999f, 1e-7f);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = GMCS_E_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (it > 0 && ms < best) best = ms;
        }
        if (!rc) *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
    }
    if (cudaGetLastError() != cudaSuccess && !rc) rc = GMCS_E_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}

extern "C" int gmcs_probe_gather(uint64_t buffer_bytes, int rec_bytes, void* cuda_stream, double* gbs) {
    if (!gbs || (rec_bytes != 16 && rec_bytes != 32) || buffer_bytes < (uint64_t)rec_bytes ||
        buffer_bytes / rec_bytes >= ((uint64_t)1 << 32))
        return GMCS_E_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256, per_thread = 256;
    float4* buf = nullptr;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GMCS_OK;
    if (cudaMalloc((void**)&buf, buffer_bytes) != cudaSuccess ||
        cudaMalloc((void**)&sink, sizeof(float) * (size_t)blocks * threads) != cudaSuccess) {
        cudaGetLastError();
        rc = GMCS_E_OOM;
    }
    if (!rc && (cudaMemsetAsync(buf, 0, buffer_bytes, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                cudaEventCreate(&e1) != cudaSuccess))
        rc = GMCS_E_CUDA;
    if (!rc) {
        const uint32_t nrec = (uint32_t)(buffer_bytes / rec_bytes);
        float best = 1e30f;
        for (int it = 0; it < 6; ++it) {   // 1 warm-up + 5 timed, best kept
            cudaEventRecord(e0, s);
            if (rec_bytes == 32) k_probe_gather<2><<<blocks, threads, 0, s>>>(buf, nrec, per_thread, sink);
            else k_probe_gather<1><<<blocks, threads, 0, s>>>(buf, nrec, per_thread, sink);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = GMCS_E_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (it > 0 && ms < best) best = ms;
        }
        if (!rc) *gbs = (double)blocks * threads * per_thread * rec_bytes / (best * 1e-3) / 1e9;
    }
    if (cudaGetLastError() != cudaSuccess && !rc) rc = GMCS_E_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    return rc;
}
