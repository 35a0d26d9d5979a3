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

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gmcs.h"
#include "context.h"
#include "kernels.h"

using namespace gmcs;

namespace {

const char kMagic[8] = {'G', 'M', 'C', 'S', 'C', 'K', 'P', 'T'};
constexpr uint32_t kVersion = 3;   // 3: 16-bit field tables hold coefficient records too

struct Header {
    char magic[8];
    uint32_t version;
    uint32_t frame;
    gmcs_config cfg;
    int32_t P, K;
    double path_now;
    double odo[12];
};

// Per keyframe, before its table bytes.
struct TableHead {
    int32_t dtype;
    int32_t layout;   // GMCS_LAYOUT_* (field tables)
    gmcs_grid grid;
    uint64_t bytes;
};
static_assert(sizeof(TableHead) == 64, "checkpoint table header");

int st(cudaError_t e) { return e == cudaSuccess ? GMCS_OK : GMCS_E_CUDA; }

struct File {
    std::FILE* f;
    explicit File(std::FILE* p) : f(p) {}
    ~File() {
        if (f) std::fclose(f);
    }
    bool put(const void* p, size_t n) { return n == 0 || std::fwrite(p, 1, n, f) == n; }
    bool get(void* p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }
    int64_t tell() { return (int64_t)ftello(f); }
    bool seek(int64_t off) { return fseeko(f, (off_t)off, SEEK_SET) == 0; }
    int64_t size() {
        const int64_t here = tell();
        if (here < 0 || fseeko(f, 0, SEEK_END) != 0) return -1;
        const int64_t n = tell();
        return seek(here) ? n : -1;
    }
};

bool finite_grid(const gmcs_grid& g) {
    return std::isfinite(g.origin[0]) && std::isfinite(g.origin[1]) && std::isfinite(g.origin[2]) &&
           std::isfinite(g.h) && g.h > 0.0;
}

// Directory bytes of a column-sparse table (the records start 256-byte aligned).
uint64_t dir_tiles_of(const gmcs_grid& g) { return (uint64_t)col_tiles(g.n[0] - 1) * col_tiles(g.n[1] - 1); }
uint64_t dir_bytes_of(const gmcs_grid& g) { return (dir_tiles_of(g) * 8 + 255) / 256 * 256; }

// Whether a keyframe's table size fits its storage type, layout and lattice as
// the library writes them: GICP voxel maps 48 bytes per voxel; dense field tables
// one record per cell; column-sparse field tables the directory and then between
// one record and one per cell (the directory itself is checked once read).
bool table_bytes_ok(const TableHead& t, const gmcs_config& cfg) {
    if (!finite_grid(t.grid)) return false;
    if (t.dtype == 3) {
        if (cfg.model != GMCS_MODEL_GICP || t.layout != GMCS_LAYOUT_DENSE) return false;
        uint64_t nv = 1;
        for (int a = 0; a < 3; ++a) {
            if (t.grid.n[a] < 1) return false;
            nv *= (uint64_t)t.grid.n[a];
        }
        return nv < ((uint64_t)1 << 31) && t.bytes == nv * 48;
    }
    if (t.dtype < 0 || t.dtype > 2 || cfg.model != GMCS_MODEL_FIELD || t.dtype != cfg.table_dtype ||
        t.layout != cfg.table_layout)
        return false;
    uint64_t nc = 1;
    for (int a = 0; a < 3; ++a) {
        if (t.grid.n[a] < 2 || t.grid.n[a] > (1 << 22)) return false;
        nc *= (uint64_t)(t.grid.n[a] - 1);
    }
    if (nc >= ((uint64_t)1 << 31)) return false;
    const uint64_t rec = t.dtype == 0 ? 32 : 16;
    if (t.layout == GMCS_LAYOUT_DENSE) return t.bytes == nc * rec;
    if (t.layout != GMCS_LAYOUT_COLUMNS || t.grid.n[2] > 65536) return false;
    const uint64_t db = dir_bytes_of(t.grid);
    const uint64_t most = dir_tiles_of(t.grid) * kColTile * kColTile * (uint64_t)(t.grid.n[2] - 1);
    return t.bytes >= db + rec && (t.bytes - db) % rec == 0 && t.bytes - db <= std::max<uint64_t>(most, 1) * rec;
}

// A column directory read from a file: every run inside the lattice's z range
// and inside the records that follow.
bool directory_ok(const unsigned char* buf, const TableHead& t) {
    const uint64_t ncol = dir_tiles_of(t.grid);
    const uint64_t nrec = (t.bytes - dir_bytes_of(t.grid)) / (t.dtype == 0 ? 32 : 16);
    const uint32_t ncz = (uint32_t)(t.grid.n[2] - 1);
    for (uint64_t k = 0; k < ncol; ++k) {
        uint2 d;
        std::memcpy(&d, buf + 8 * k, sizeof(d));
        const uint32_t zlo = d.y & 0xFFFFu, cnt = d.y >> 16;
        if ((uint64_t)zlo + cnt > ncz || (uint64_t)d.x + (uint64_t)cnt * kColTile * kColTile > nrec) return false;
    }
    return true;
}

uint64_t expected_occ_bytes(const gmcs_grid& g) {
    if (!finite_grid(g)) return 0;
    uint64_t nv = 1;
    for (int a = 0; a < 3; ++a) {
        if (g.n[a] < 1) return 0;
        nv *= (uint64_t)g.n[a];
    }
    return nv < ((uint64_t)1 << 32) ? nv : 0;
}

// Walk a whole checkpoint on the host, reading only headers and skipping
// payloads, and check every size against the lattice it belongs to and the
// file's length. Leaves the file positioned just after the header.
int validate(File& in, Header& h) {
    const int64_t fsize = in.size();
    if (fsize < 0 || !in.seek(0)) return GMCS_E_IO;
    if (!in.get(&h, sizeof(h)) || std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.version != kVersion)
        return GMCS_E_IO;
    if (!config_valid(&h.cfg) || h.P <= 0 || h.K < 0 || h.K > (1 << 20) || !std::isfinite(h.path_now))
        return GMCS_E_IO;
    const int64_t pose_bytes = (int64_t)sizeof(float) * 12 * h.P;
    int64_t pos = in.tell() + pose_bytes + (int64_t)sizeof(double) * h.P;
    for (int k = 0; k < h.K; ++k) {
        TableHead t;
        if (pos > fsize || !in.seek(pos) || !in.get(&t, sizeof(t))) return GMCS_E_IO;
        if (!table_bytes_ok(t, h.cfg)) return GMCS_E_IO;
        if (t.dtype != 3 && t.layout == GMCS_LAYOUT_COLUMNS) {   // read and check the column directory
            const uint64_t db = dir_bytes_of(t.grid);
            if (pos + (int64_t)sizeof(t) + (int64_t)db > fsize) return GMCS_E_IO;
            std::vector<unsigned char> dbuf(db);
            if (!in.get(dbuf.data(), db) || !directory_ok(dbuf.data(), t)) return GMCS_E_IO;
        }
        pos += (int64_t)sizeof(t) + (int64_t)t.bytes;
        gmcs_grid og;
        uint64_t occ_bytes = 0;
        if (pos > fsize || !in.seek(pos) || !in.get(&og, sizeof(og)) || !in.get(&occ_bytes, sizeof(occ_bytes)))
            return GMCS_E_IO;
        const uint64_t want_occ = expected_occ_bytes(og);
        if (want_occ == 0 || occ_bytes != want_occ) return GMCS_E_IO;
        pos += (int64_t)(sizeof(og) + sizeof(occ_bytes) + occ_bytes);
        double d = 0.0;
        if (pos > fsize || !in.seek(pos) || !in.get(&d, sizeof(d)) || !std::isfinite(d)) return GMCS_E_IO;
        pos += (int64_t)sizeof(d) + pose_bytes;
    }
    if (pos != fsize) return GMCS_E_IO;
    return in.seek(sizeof(h)) ? GMCS_OK : GMCS_E_IO;
}

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

namespace {

int save_impl(gmcs_ctx* c, const char* path) {
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
        TableHead th;
        std::memset(&th, 0, sizeof(th));
        th.dtype = t.dtype;
        th.layout = t.layout;
        th.grid = t.grid;
        th.bytes = t.bytes;
        const uint64_t occ_bytes = t.occ_bytes;
        if (!out.put(&th, sizeof(th))) return GMCS_E_IO;
        buf.resize(t.bytes);
        if ((rc = st(cudaMemcpy(buf.data(), t.cells, t.bytes, cudaMemcpyDeviceToHost)))) return rc;
        if (!out.put(buf.data(), t.bytes)) return GMCS_E_IO;
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

// Drop what a failed load restored: tables, keyframe count, particles.
void unload(gmcs_ctx* c) {
    cudaStreamSynchronize(c->stream);
    for (auto& t : c->tables) {
        c->dev_bytes -= std::min(c->dev_bytes, t.bytes + t.occ_bytes);
        cudaFree(t.cells);
        cudaFree(t.occ);
    }
    c->tables.clear();
    c->kf_path.clear();
    c->K = 0;
    c->P = 0;
    c->nbr_K = 0;
    cudaMemsetAsync(c->nbr, 0, sizeof(int) * GMCS_MAX_NB * c->ld, c->stream);
    cudaMemsetAsync(c->d_tables, 0, sizeof(TableDesc) * (size_t)c->Kmax, c->stream);
    cudaStreamSynchronize(c->stream);
    c->have_particles = false;
    c->last_valid = false;
    cudaGetLastError();
}

int load_impl(gmcs_ctx* c, const char* path, bool* touched) {
    File in(std::fopen(path, "rb"));
    if (!in.f) return GMCS_E_IO;
    Header h;
    int rc = validate(in, h);
    if (rc) return rc;
    if (h.P > c->Pmax || h.K > c->Kmax) return GMCS_E_CAPACITY;
    std::vector<float> poses((size_t)12 * h.P);
    std::vector<double> logw(h.P);
    if (!in.get(poses.data(), sizeof(float) * poses.size()) || !in.get(logw.data(), sizeof(double) * logw.size()))
        return GMCS_E_IO;
    *touched = true;
    rc = gmcs_init_particles(c, poses.data(), h.P, logw.data());
    if (rc) return rc;
    std::vector<unsigned char> buf;
    for (int k = 0; k < h.K; ++k) {
        TableHead th;
        if (!in.get(&th, sizeof(th))) return GMCS_E_IO;
        HostTable t;
        t.dtype = th.dtype;
        t.layout = th.layout;
        t.grid = th.grid;
        t.bytes = th.bytes;
        t.dir_bytes = (th.dtype != 3 && th.layout == GMCS_LAYOUT_COLUMNS) ? dir_bytes_of(th.grid) : 0;
        buf.resize(t.bytes);
        if (!in.get(buf.data(), t.bytes)) return GMCS_E_IO;
        if (t.dir_bytes && !directory_ok(buf.data(), th)) return GMCS_E_IO;
        if (cudaMalloc(&t.cells, t.bytes) != cudaSuccess) {
            cudaGetLastError();
            return GMCS_E_OOM;
        }
        uint64_t occ_bytes = 0;
        rc = st(cudaMemcpy(t.cells, buf.data(), t.bytes, cudaMemcpyHostToDevice));
        if (!rc && (!in.get(&t.occ_grid, sizeof(t.occ_grid)) || !in.get(&occ_bytes, sizeof(occ_bytes)))) rc = GMCS_E_IO;
        if (!rc) {
            buf.resize(occ_bytes);
            if (!in.get(buf.data(), occ_bytes)) rc = GMCS_E_IO;
        }
        if (!rc && cudaMalloc((void**)&t.occ, occ_bytes) != cudaSuccess) {
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
            td.cells = table_records(t);
            td.dir = table_dir(t);
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

}  // namespace

extern "C" int gmcs_save(gmcs_ctx* c, const char* path) {
    if (!c || !path) return GMCS_E_INVALID;
    try {
        return save_impl(c, path);
    } catch (const std::bad_alloc&) {
        return GMCS_E_OOM;
    } catch (...) {
        return GMCS_E_IO;
    }
}

extern "C" int gmcs_load(gmcs_ctx* c, const char* path) {
    if (!c || !path) return GMCS_E_INVALID;
    if (c->K != 0) return GMCS_E_STATE;   // restore into an empty context
    int rc;
    bool touched = false;   // the context's particles were replaced
    try {
        rc = load_impl(c, path, &touched);
    } catch (const std::bad_alloc&) {
        rc = GMCS_E_OOM;
    } catch (...) {
        rc = GMCS_E_IO;
    }
    if (rc && touched) unload(c);
    return rc;
}

extern "C" int gmcs_checkpoint_info(const char* path, gmcs_config* cfg, int* P, int* K, uint32_t* frame) {
    if (!path) return GMCS_E_INVALID;
    try {
        File in(std::fopen(path, "rb"));
        if (!in.f) return GMCS_E_IO;
        Header h;
        const int rc = validate(in, h);
        if (rc) return rc;
        if (cfg) *cfg = h.cfg;
        if (P) *P = h.P;
        if (K) *K = h.K;
        if (frame) *frame = h.frame;
        return GMCS_OK;
    } catch (...) {
        return GMCS_E_IO;
    }
}
