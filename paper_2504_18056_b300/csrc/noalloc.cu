// noalloc.cu -- systematic resampling for callers that cannot allocate device memory.
//
// gmcs_resample keeps its prefix-sum scratch in a context that gmcs_create
// allocated with cudaMalloc. Some callers cannot call cudaMalloc at all: code
// that runs under a memory manager owning the whole device budget, or a
// real-time loop where an allocation's implicit device synchronisation and
// unbounded latency are not acceptable. gmcs_resample_noalloc runs the same
// three kernels (quantise + block scan, scan of block totals, binary search)
// with its scratch in a file-scope __device__ array instead, sized for up to
// GMCS_NOALLOC_MAX_P particles. It allocates nothing and needs no context.
//
// The array's name in host code is only a host-side handle, not a device
// address, so the first call on each device asks the runtime for the array's
// device address (cudaGetSymbolAddress, with that device current) and caches
// it for later calls on that device, keyed by the unique id of the device's
// current context: after cudaDeviceReset the library's module is loaded into a
// new context, and the next call looks the address up again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/gmcs.h"
#include "kernels.h"

using namespace gmcs;

namespace {

constexpr int kNoallocBlocks = (GMCS_NOALLOC_MAX_P + kScanBlock - 1) / kScanBlock;
// block-local prefix sums (one per particle), then block totals / offsets (+1 for the grand total)
constexpr size_t kNoallocWords = (size_t)GMCS_NOALLOC_MAX_P + kNoallocBlocks + 1;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
    unsigned long long ctx_id = 0;   // unique id of the context the address belongs to (0: none)
    unsigned long long* ptr = nullptr;
};
Cached g_scratch_dev[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 if none or unknown),
// through driver entry points the runtime hands out (no link to the driver
// library is needed).
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        cudaGetLastError();
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array in the current device's current context
// (looked up once per device and context).
int scratch_on_current_device(unsigned long long** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return GMCS_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    Cached& c = g_scratch_dev[dev];
    const unsigned long long id = current_ctx_id();
    if (!c.ptr || id == 0 || id != c.ctx_id) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {   // makes the context current
            cudaGetLastError();
            return GMCS_E_CUDA;
        }
        c.ptr = static_cast<unsigned long long*>(p);
        c.ctx_id = current_ctx_id();
    }
    *out = c.ptr;
    return GMCS_OK;
}

}  // namespace

extern "C" int gmcs_resample_noalloc(const double* w, int P, double u, int* anc, void* cuda_stream) {
    if (!w || !anc || P <= 0) return GMCS_E_INVALID;
    if (P > GMCS_NOALLOC_MAX_P) return GMCS_E_CAPACITY;
    if (!(u >= 0.0 && u < 1.0)) return GMCS_E_INVALID;
    cudaPointerAttributes aw, aa;
    if (cudaPointerGetAttributes(&aw, w) != cudaSuccess || cudaPointerGetAttributes(&aa, anc) != cudaSuccess) {
        cudaGetLastError();
        return GMCS_E_INVALID;
    }
    if ((aw.type != cudaMemoryTypeDevice && aw.type != cudaMemoryTypeManaged) ||
        (aa.type != cudaMemoryTypeDevice && aa.type != cudaMemoryTypeManaged))
        return GMCS_E_INVALID;
    unsigned long long* scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nb = (P + kScanBlock - 1) / kScanBlock;
    unsigned long long* cl = scratch;
    unsigned long long* btot = scratch + GMCS_NOALLOC_MAX_P;
    // every word the kernels read is written first in this call: cl[0..P) and
    // btot[0..nb] by the scan kernels, so no clearing is needed
    ScanArgs sa;
    sa.logw = nullptr;
    sa.w = w;
    sa.res = nullptr;
    sa.w_out = nullptr;
    sa.P = P;
    sa.cl = cl;
    sa.btot = btot;
    launch_resample_scan(sa, s);
    launch_scan_totals(btot, nb, s);
    SearchArgs se;
    se.cl = cl;
    se.boff = btot;
    se.nblocks = nb;
    se.P = P;
    se.u = u;
    se.u_from_philox = 0;
    se.seed = 0;
    se.frame = 0;
    se.res = nullptr;
    se.anc = anc;
    launch_resample_search(se, s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GMCS_OK : GMCS_E_CUDA;
}
