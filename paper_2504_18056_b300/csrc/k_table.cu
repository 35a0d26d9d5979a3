// k_table.cu -- keyframe likelihood tables (map insertion, not on the per-frame path).
//
// A keyframe table holds, at every lattice vertex, exp(-d^2 / 2 sigma^2) with d
// the distance to the nearest keyframe point, 0 where d > r_t. It is built in
// two launches: each point relaxes the squared distance of every vertex within
// r_t (atomicMin on the float bit pattern, which orders like the value for
// non-negative floats), then every cell turns its 8 corner values into the
// coefficients of its trilinear polynomial, stored as one record, so that a
// lookup is a single 32 B (FP32) or 16 B (BF16/FP16) load.
#include "kernels.h"

namespace gmcs {

__global__ void k_fill_u32(unsigned* __restrict__ p, size_t n, unsigned v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// Offset (o + h i) - p of a vertex coordinate from a point coordinate, carried in
// float pairs: the product h_hi * i and the sum with o_hi are split into value and
// exact rounding error (fma product error, two-sum), so the offset keeps ~1e-7 m
// accuracy even 100 m from the origin where a plain float sum loses ~1e-5 m.
__device__ __forceinline__ float vertex_offset(float o_hi, float o_lo, float h_hi, float h_lo, int i, float p) {
    // explicit round-to-nearest operations: no contraction may merge these steps
    const float fi = (float)i;
    const float prod = __fmul_rn(h_hi, fi);
    const float perr = fmaf(h_hi, fi, -prod);
    const float s = __fadd_rn(o_hi, prod);
    const float bb = __fsub_rn(s, o_hi);
    const float serr = __fadd_rn(__fsub_rn(o_hi, __fsub_rn(s, bb)), __fsub_rn(prod, bb));
    const float lo = serr + perr + o_lo + h_lo * fi;
    return __fsub_rn(s, p) + lo;
}

// One CTA per point; its threads walk the box of vertices within r_t.
__global__ void k_splat(SplatArgs a) {
    const int j = blockIdx.x;
    if (j >= a.n) return;
    const float p3[3] = {a.pts[3 * j], a.pts[3 * j + 1], a.pts[3 * j + 2]};
    // vertex index range covering [p - r_t, p + r_t], widened by one vertex so that
    // float rounding of the bounds cannot drop a vertex; the value pass applies the
    // exact d^2 <= r_t^2 test
    const float inv_h = 1.0f / a.h_hi;
    int lo[3], hi[3];
    const int n3[3] = {a.nx, a.ny, a.nz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        lo[ax] = max(0, (int)floorf((p3[ax] - a.r_t - a.o_hi[ax]) * inv_h) - 1);
        hi[ax] = min(n3[ax] - 1, (int)ceilf((p3[ax] + a.r_t - a.o_hi[ax]) * inv_h) + 1);
    }
    if (lo[0] > hi[0] || lo[1] > hi[1] || lo[2] > hi[2]) return;
    const int sx = hi[0] - lo[0] + 1, sy = hi[1] - lo[1] + 1, sz = hi[2] - lo[2] + 1;
    const int total = sx * sy * sz;
    const float r2 = a.r_t * a.r_t;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int ix = lo[0] + t % sx;
        const int iy = lo[1] + (t / sx) % sy;
        const int iz = lo[2] + t / (sx * sy);
        const float dx = vertex_offset(a.o_hi[0], a.o_lo[0], a.h_hi, a.h_lo, ix, p3[0]);
        const float dy = vertex_offset(a.o_hi[1], a.o_lo[1], a.h_hi, a.h_lo, iy, p3[1]);
        const float dz = vertex_offset(a.o_hi[2], a.o_lo[2], a.h_hi, a.h_lo, iz, p3[2]);
        const float d2 = dx * dx + dy * dy + dz * dz;
        if (d2 <= r2 * 1.0001f) {
            const size_t v = ((size_t)iz * a.ny + iy) * a.nx + ix;
            atomicMin(&a.d2[v], __float_as_uint(d2));
        }
    }
}

__device__ __forceinline__ float field_value(unsigned bits, float inv_two_sigma2, float r_t2) {
    const float d2 = __uint_as_float(bits);
    return (d2 <= r_t2) ? expf(-d2 * inv_two_sigma2) : 0.0f;
}

// The 8 corner values of cell (cx, cy, cz) -> its coefficient record at `out`.
__device__ __forceinline__ void pack_cell(const PackArgs& a, int cx, int cy, int cz, size_t out) {
    float v[8];
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const size_t vi = ((size_t)(cz + dz) * a.ny + (cy + dy)) * a.nx + (cx + dx);
                v[rec_slot(dx, dy, dz)] = field_value(a.d2[vi], a.inv_two_sigma2, a.r_t2);
            }
    float r[8];
    corners_to_coef(v, r);
    if (a.dtype == 0) {
        float4* o = reinterpret_cast<float4*>(a.cells) + 2 * out;
        o[0] = make_float4(r[0], r[1], r[2], r[3]);
        o[1] = make_float4(r[4], r[5], r[6], r[7]);
    } else {
        reinterpret_cast<uint4*>(a.cells)[out] = encode_rec16(r, a.dtype);
    }
}

// Dense tables: one thread per cell. Column-sparse tables: one thread per tile of
// columns, packing the cells of its run (cells past the lattice's edge in x or y,
// which no lookup reads, stay unwritten).
__global__ void k_pack(PackArgs a) {
    const int ncx = a.nx - 1, ncy = a.ny - 1, ncz = a.nz - 1;
    if (a.dir) {
        const uint32_t ntx = col_tiles(ncx), nty = col_tiles(ncy);
        const size_t ntile = (size_t)ntx * nty;
        for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < ntile; t += (size_t)gridDim.x * blockDim.x) {
            const uint2 d = a.dir[t];
            const int tx = (int)(t % ntx), ty = (int)(t / ntx);
            const int zlo = (int)(d.y & 0xFFFFu), cnt = (int)(d.y >> 16);
            for (int k = 0; k < cnt; ++k)
                for (int ly = 0; ly < kColTile; ++ly)
                    for (int lx = 0; lx < kColTile; ++lx) {
                        const int cx = tx * kColTile + lx, cy = ty * kColTile + ly;
                        if (cx < ncx && cy < ncy)
                            pack_cell(a, cx, cy, zlo + k,
                                      (size_t)d.x + (((size_t)k * kColTile + ly) * kColTile + lx));
                    }
        }
        return;
    }
    const size_t ncell = (size_t)ncx * ncy * ncz;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < ncell; c += (size_t)gridDim.x * blockDim.x) {
        const int cx = (int)(c % ncx);
        const int cy = (int)((c / ncx) % ncy);
        const int cz = (int)(c / ((size_t)ncx * ncy));
        pack_cell(a, cx, cy, cz, c);
    }
}

// Column-sparse tables: per tile of columns, the run from its lowest to its
// highest cell layer with a nonzero corner value, as zlo | layers << 16 (0: empty).
__global__ void k_col_range(const unsigned* __restrict__ d2, int nx, int ny, int nz, float inv_two_sigma2,
                            float r_t2, uint32_t* __restrict__ out) {
    const int ncx = nx - 1, ncy = ny - 1, ncz = nz - 1;
    const uint32_t ntx = col_tiles(ncx), nty = col_tiles(ncy);
    const size_t ntile = (size_t)ntx * nty;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < ntile; t += (size_t)gridDim.x * blockDim.x) {
        const int x0 = (int)(t % ntx) * kColTile, y0 = (int)(t / ntx) * kColTile;
        const int x1 = min(x0 + kColTile, ncx), y1 = min(y0 + kColTile, ncy);   // cells [x0, x1) x [y0, y1)
        int lo = -1, hi = -2;
        for (int iz = 0; iz < nz; ++iz) {
            // vertex layer iz of the tile (vertices x0..x1, y0..y1) holds a nonzero value:
            // cell layers iz - 1 and iz are nonzero
            bool nzv = false;
            for (int iy = y0; iy <= y1 && !nzv; ++iy)
                for (int ix = x0; ix <= x1 && !nzv; ++ix)
                    nzv = field_value(d2[((size_t)iz * ny + iy) * nx + ix], inv_two_sigma2, r_t2) > 0.f;
            if (nzv) {
                const int c0 = iz > 0 ? iz - 1 : 0, c1 = iz < ncz ? iz : ncz - 1;
                if (lo < 0) lo = c0;
                hi = c1;
            }
        }
        out[t] = lo < 0 ? 0u : ((uint32_t)lo | ((uint32_t)(hi - lo + 1) << 16));
    }
}

// The coefficients (record order) of cell (cx, cy, cz) as stored; zeros for a cell
// a column-sparse table does not store.
__device__ __forceinline__ void read_cell(const void* __restrict__ cells, const uint2* __restrict__ dir, int dtype,
                                          int ncx, int ncy, int cx, int cy, int cz, float* r) {
    size_t c;
    if (dir) {
        uint32_t idx;
        if (!col_cell(dir, (uint32_t)ncx, (uint32_t)ncy, cx, cy, cz, idx)) {
#pragma unroll
            for (int k = 0; k < 8; ++k) r[k] = 0.f;
            return;
        }
        c = idx;
    } else {
        c = ((size_t)cz * ncy + cy) * ncx + cx;
    }
    if (dtype == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = reinterpret_cast<const float*>(cells)[8 * c + k];
    } else if (dtype == 1) {
        decode_rec16<1>(reinterpret_cast<const uint4*>(cells)[c], r);
    } else {
        decode_rec16<2>(reinterpret_cast<const uint4*>(cells)[c], r);
    }
}

// Vertex values read back from the cell records (vertex i lives in cell
// min(i, nc-1), at its corner; the sum of the stored coefficients).
__global__ void k_unpack(const void* __restrict__ cells, const uint2* __restrict__ dir, int dtype, int nx, int ny,
                         int nz, float* __restrict__ out) {
    const size_t nv = (size_t)nx * ny * nz;
    const int ncx = nx - 1, ncy = ny - 1, ncz = nz - 1;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nv; v += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(v % nx), iy = (int)((v / nx) % ny), iz = (int)(v / ((size_t)nx * ny));
        const int cx = min(ix, ncx - 1), cy = min(iy, ncy - 1), cz = min(iz, ncz - 1);
        float r[8];
        read_cell(cells, dir, dtype, ncx, ncy, cx, cy, cz, r);
        out[v] = coef_corner(r, ix - cx, iy - cy, iz - cz);
    }
}

// Coefficients c0..c7 (natural order) of cells [c0, c0 + n) (numbered x fastest),
// as stored (zeros for cells a column-sparse table does not store).
__global__ void k_records(const void* __restrict__ cells, const uint2* __restrict__ dir, int dtype, int nx, int ny,
                          size_t c0, size_t n, float* __restrict__ out) {
    const int ncx = nx - 1, ncy = ny - 1;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t c = c0 + e;
        const int cx = (int)(c % ncx), cy = (int)((c / ncx) % ncy), cz = (int)(c / ((size_t)ncx * ncy));
        float r[8];
        read_cell(cells, dir, dtype, ncx, ncy, cx, cy, cz, r);
#pragma unroll
        for (int k = 0; k < 8; ++k) out[8 * e + k] = r[coef_slot(k)];
    }
}

static int grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b > 148 * 32) b = 148 * 32;
    return (int)(b > 0 ? b : 1);
}

void launch_fill_u32(unsigned* p, size_t n, unsigned v, cudaStream_t s) {
    k_fill_u32<<<grid_for(n, 256), 256, 0, s>>>(p, n, v);
}

void launch_splat(const SplatArgs& a, cudaStream_t s) {
    if (a.n > 0) k_splat<<<a.n, 128, 0, s>>>(a);
}

void launch_pack(const PackArgs& a, cudaStream_t s) {
    const size_t n = a.dir ? (size_t)col_tiles(a.nx - 1) * col_tiles(a.ny - 1) : (size_t)(a.nx - 1) * (a.ny - 1) * (a.nz - 1);
    k_pack<<<grid_for(n, 256), 256, 0, s>>>(a);
}

void launch_col_range(const unsigned* d2, int nx, int ny, int nz, float inv_two_sigma2, float r_t2, uint32_t* out,
                      cudaStream_t s) {
    k_col_range<<<grid_for((size_t)col_tiles(nx - 1) * col_tiles(ny - 1), 256), 256, 0, s>>>(d2, nx, ny, nz,
                                                                                            inv_two_sigma2, r_t2, out);
}

void launch_unpack(const void* cells, const uint2* dir, int dtype, int nx, int ny, int nz, float* out, cudaStream_t s) {
    k_unpack<<<grid_for((size_t)nx * ny * nz, 256), 256, 0, s>>>(cells, dir, dtype, nx, ny, nz, out);
}

void launch_records(const void* cells, const uint2* dir, int dtype, int nx, int ny, int nz, size_t c0, size_t n,
                    float* out, cudaStream_t s) {
    (void)nz;
    if (n > 0) k_records<<<grid_for(n, 256), 256, 0, s>>>(cells, dir, dtype, nx, ny, c0, n, out);
}

}  // namespace gmcs
