// checkpoint.cu -- save and restore a filter session (gmcs_save / gmcs_load).
//
// A checkpoint is a little-endian binary file: a header (magic, version, the
// context's config, particle and keyframe counts, frame counter, odometry path
// and relative odometry), then the particles (current poses P x 12 floats,
// log-weights P doubles), then per keyframe its table exactly as stored on the
// device (cells, lattice, storage type), its occupancy lattice, its odometry path
// length and every particle's pose of it (P x 12 floats). Restoring it into an
// empty context (its config is replaced by the saved one) and stepping with the
// same inputs reproduces the saved session's frames bit for bit (the draws are
// counter-based on the restored seed and frame counter).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/gmcs.h"
#include "context.h"
#include "kernels.h"

using namespace gmcs;

namespace {

const char kMagic[8] = {'G', 'M', 'C', 'S', 'C', 'K', 'P', 'T'};
constexpr uint32_t kVersion = 2;   // 2: FP32 field tables hold trilinear coefficients

struct Header {
    char magic[8];
    uint32_t version;
    uint32_t frame;
    gmcs_config cfg;
    int32_t P, K;
    double path_now;
    double odo[12];
};

int st(cudaError_t e) { return e == cudaSuccess ? GMCS_OK : GMCS_E_CUDA; }

struct File {
    std::FILE* f;
    explicit File(std::FILE* p) : f(p) {}
    ~File() {
        if (f) std::fclose(f);
    }
    bool put(const void* p, size_t n) { return n == 0 || std::fwrite(p, 1, n, f) == n; }
    bool get(void* p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }
};

// P x 12 poses from a SoA block of the context to the host.
int poses_out(gmcs_ctx* c, const float* soa, std::vector<float>& host) {
    launch_soa_to_aos(soa, c->ld, c->P, 12, c->part, c->stream);
    c->launches++;
    c->kind_launches[K_MISC]++;
    host.resize((size_t)12 * c->P);
    int rc = st(cudaGetLastError());
    if (!rc) rc = st(cudaMemcpyAsync(host.data(), c->part, sizeof(float) * host.size(), cudaMemcpyDeviceToHost,
                                     c->stream));
    if (!rc) rc = st(cudaStreamSynchronize(c->stream));
    return rc;
}

int poses_in(gmcs_ctx* c, const std::vector<float>& host, float* soa) {
    int rc = st(cudaMemcpyAsync(c->part, host.data(), sizeof(float) * host.size(), cudaMemcpyHostToDevice,
                                c->stream));
    if (rc) return rc;
    launch_aos_to_soa(c->part, c->P, 12, soa, c->ld, c->stream);
    c->launches++;
    c->kind_launches[K_MISC]++;
    rc = st(cudaGetLastError());
    if (!rc) rc = st(cudaStreamSynchronize(c->stream));
    return rc;
}

}  // namespace

extern "C" int gmcs_save(gmcs_ctx* c, const char* path) {
    if (!c || !path) return GMCS_E_INVALID;
    if (!c->have_particles) return GMCS_E_STATE;
    int rc = st(cudaStreamSynchronize(c->stream));
    if (rc) return rc;
    File out(std::fopen(path, "wb"));
    if (!out.f) return GMCS_E_IO;
    Header h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.version = kVersion;
    h.frame = c->frame;
    h.cfg = c->cfg;
    h.P = c->P;
    h.K = c->K;
    h.path_now = c->path_now;
    std::memcpy(h.odo, c->odo, sizeof(h.odo));
    if (!out.put(&h, sizeof(h))) return GMCS_E_IO;
    std::vector<float> poses;
    if ((rc = poses_out(c, c->pose[c->cur], poses))) return rc;
    std::vector<double> logw(c->P);
    if ((rc = st(cudaMemcpy(logw.data(), c->logw, sizeof(double) * c->P, cudaMemcpyDeviceToHost)))) return rc;
    if (!out.put(poses.data(), sizeof(float) * poses.size()) || !out.put(logw.data(), sizeof(double) * logw.size()))
        return GMCS_E_IO;
    std::vector<unsigned char> buf;
    for (int k = 0; k < c->K; ++k) {
        const HostTable& t = c->tables[k];
        const int32_t dtype = t.dtype;
        const uint64_t bytes = t.bytes, occ_bytes = t.occ_bytes;
        if (!out.put(&dtype, sizeof(dtype)) || !out.put(&t.grid, sizeof(t.grid)) || !out.put(&bytes, sizeof(bytes)))
            return GMCS_E_IO;
        buf.resize(bytes);
        if ((rc = st(cudaMemcpy(buf.data(), t.cells, bytes, cudaMemcpyDeviceToHost)))) return rc;
        if (!out.put(buf.data(), bytes)) return GMCS_E_IO;
        if (!out.put(&t.occ_grid, sizeof(t.occ_grid)) || !out.put(&occ_bytes, sizeof(occ_bytes))) return GMCS_E_IO;
        buf.resize(occ_bytes);
        if ((rc = st(cudaMemcpy(buf.data(), t.occ, occ_bytes, cudaMemcpyDeviceToHost)))) return rc;
        if (!out.put(buf.data(), occ_bytes)) return GMCS_E_IO;
        const double d = c->kf_path[k];
        if (!out.put(&d, sizeof(d))) return GMCS_E_IO;
        if ((rc = poses_out(c, c->kf[c->cur] + (size_t)k * kPoseC * c->ld, poses))) return rc;
        if (!out.put(poses.data(), sizeof(float) * poses.size())) return GMCS_E_IO;
    }
    return std::fflush(out.f) == 0 ? GMCS_OK : GMCS_E_IO;
}

extern "C" int gmcs_load(gmcs_ctx* c, const char* path) {
    if (!c || !path) return GMCS_E_INVALID;
    if (c->K != 0) return GMCS_E_STATE;   // restore into an empty context
    File in(std::fopen(path, "rb"));
    if (!in.f) return GMCS_E_IO;
    Header h;
    if (!in.get(&h, sizeof(h)) || std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.version != kVersion)
        return GMCS_E_IO;
    if (h.P <= 0 || h.K < 0) return GMCS_E_IO;
    if (h.P > c->Pmax || h.K > c->Kmax) return GMCS_E_CAPACITY;
    std::vector<float> poses((size_t)12 * h.P);
    std::vector<double> logw(h.P);
    if (!in.get(poses.data(), sizeof(float) * poses.size()) || !in.get(logw.data(), sizeof(double) * logw.size()))
        return GMCS_E_IO;
    int rc = gmcs_init_particles(c, poses.data(), h.P, logw.data());
    if (rc) return rc;
    for (int k = 0; k < h.K; ++k) {
        HostTable t;
        int32_t dtype = 0;
        uint64_t bytes = 0, occ_bytes = 0;
        if (!in.get(&dtype, sizeof(dtype)) || !in.get(&t.grid, sizeof(t.grid)) || !in.get(&bytes, sizeof(bytes)))
            return GMCS_E_IO;
        t.dtype = dtype;
        t.bytes = bytes;
        std::vector<unsigned char> buf(bytes);
        if (!in.get(buf.data(), bytes)) return GMCS_E_IO;
        if (cudaMalloc(&t.cells, bytes) != cudaSuccess) {
            cudaGetLastError();
            return GMCS_E_OOM;
        }
        rc = st(cudaMemcpy(t.cells, buf.data(), bytes, cudaMemcpyHostToDevice));
        if (!rc && (!in.get(&t.occ_grid, sizeof(t.occ_grid)) || !in.get(&occ_bytes, sizeof(occ_bytes)))) rc = GMCS_E_IO;
        if (!rc) {
            buf.resize(occ_bytes);
            if (!in.get(buf.data(), occ_bytes)) rc = GMCS_E_IO;
        }
        if (!rc && cudaMalloc((void**)&t.occ, occ_bytes > 0 ? occ_bytes : 1) != cudaSuccess) {
            cudaGetLastError();
            t.occ = nullptr;
            rc = GMCS_E_OOM;
        }
        t.occ_bytes = occ_bytes;
        if (!rc) rc = st(cudaMemcpy(t.occ, buf.data(), occ_bytes, cudaMemcpyHostToDevice));
        double d = 0.0;
        if (!rc && !in.get(&d, sizeof(d))) rc = GMCS_E_IO;
        if (!rc && !in.get(poses.data(), sizeof(float) * poses.size())) rc = GMCS_E_IO;
        if (!rc) rc = poses_in(c, poses, c->kf[c->cur] + (size_t)k * kPoseC * c->ld);
        if (!rc) {
            TableDesc td;
            std::memset(&td, 0, sizeof(td));
            td.cells = t.cells;
            td.ox = (float)t.grid.origin[0];
            td.oy = (float)t.grid.origin[1];
            td.oz = (float)t.grid.origin[2];
            td.inv_h = (float)(1.0 / t.grid.h);
            td.h = (float)t.grid.h;
            const int edge = t.dtype == 3 ? 0 : 1;   // field tables: cells = vertices - 1
            td.ncx = t.grid.n[0] - edge;
            td.ncy = t.grid.n[1] - edge;
            td.ncz = t.grid.n[2] - edge;
            td.dtype = t.dtype;
            const float df = (float)d;
            rc = st(cudaMemcpy(c->d_tables + k, &td, sizeof(td), cudaMemcpyHostToDevice));
            if (!rc) rc = st(cudaMemcpy(c->d_kf_path + k, &df, sizeof(df), cudaMemcpyHostToDevice));
        }
        if (rc) {
            cudaFree(t.cells);
            cudaFree(t.occ);
            return rc;
        }
        c->kf_path.push_back(d);
        c->dev_bytes += t.bytes + t.occ_bytes;
        c->tables.push_back(t);
        c->K = k + 1;
    }
    c->cfg = h.cfg;   // the saved session's settings (seed, model, policies) continue
    c->frame = h.frame;
    c->path_now = h.path_now;
    std::memcpy(c->odo, h.odo, sizeof(h.odo));
    return GMCS_OK;
}
