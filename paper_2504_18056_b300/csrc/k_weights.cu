// k_weights.cu -- importance weighting (Eq. 11) and systematic resampling.
//
// Weights live as FP64 log-weights. One launch adds the frame's log-likelihood,
// finds M = max logw (argmax, lowest index on ties), S = sum exp(logw - M) and
// S2 = sum exp(2 (logw - M)): each CTA takes its own max and its sums against
// it (per thread, per warp by shuffles, per CTA through shared memory); the
// last CTA to finish (a ticket counter) takes the global max and rescales the
// CTA sums to it, always in the same order. The normalised weight is
// w_i = exp(logw_i - M - log S), ESS = S^2 / S2.
//
// Resampling quantises w_i to q_i = rint(w_i 2^52) so that every prefix sum
// is an exact integer below 2^53 (exactly representable as a double), takes
// C_i by a block scan plus a scan of block totals, and finds for each output
// slot m the ancestor a_m = min{i : C_i > tau_m}, tau_m = ((u + m) / P) S in
// IEEE double with explicit round-to-nearest operations, by binary search.
// The result is independent of the scan order and bit-identical to a serial
// evaluation of the same definition.
#include <math.h>

#include "kernels.h"

namespace gmcs {

namespace {

// (max log-weight, its lowest index) and the max frame log-likelihood
struct MaxArg {
    double m;
    int i;
    double lm;
};

__device__ __forceinline__ MaxArg max_combine(MaxArg a, MaxArg b) {
    const bool take_b = (b.m > a.m) || (b.m == a.m && b.i < a.i);
    MaxArg r = take_b ? b : a;
    r.lm = fmax(a.lm, b.lm);
    return r;
}

constexpr int kWeighThreads = 256;

// CTA-wide argmax; the result is returned to every thread.
__device__ MaxArg max_block(MaxArg v) {
    __shared__ MaxArg sh[32];
    __shared__ MaxArg out;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        MaxArg o;
        o.m = __shfl_down_sync(0xffffffffu, v.m, off);
        o.i = __shfl_down_sync(0xffffffffu, v.i, off);
        o.lm = __shfl_down_sync(0xffffffffu, v.lm, off);
        v = max_combine(v, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (warp == 0) {
        v = (lane < nw) ? sh[lane] : MaxArg{-INFINITY, 0x7fffffff, -INFINITY};
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            MaxArg o;
            o.m = __shfl_down_sync(0xffffffffu, v.m, off);
            o.i = __shfl_down_sync(0xffffffffu, v.i, off);
            o.lm = __shfl_down_sync(0xffffffffu, v.lm, off);
            v = max_combine(v, o);
        }
        if (lane == 0) out = v;
    }
    __syncthreads();
    return out;
}

// CTA-wide sums of (s, s2) in a fixed order; the result is valid in thread 0.
__device__ double2 sum_block(double2 v) {
    __shared__ double2 sh[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, off);
        v.y += __shfl_down_sync(0xffffffffu, v.y, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (warp == 0) {
        v = (lane < nw) ? sh[lane] : make_double2(0.0, 0.0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, off);
            v.y += __shfl_down_sync(0xffffffffu, v.y, off);
        }
    }
    __syncthreads();
    return v;
}

}  // namespace

// Max first, then sums of exp against that max: the only exponentials are one
// per particle (independent) and one per CTA partial in the last CTA, instead
// of a chain of them through an online (max, sum) reduction (37 -> 24 us at
// 100,000 particles).
__device__ __forceinline__ void weigh_body(const WeighArgs& a, int vb, int vg) {
    MaxArg mx{-INFINITY, 0x7fffffff, -INFINITY};
    for (int i = vb * blockDim.x + threadIdx.x; i < a.P; i += vg * blockDim.x) {
        double v = a.logw[i];
        if (a.ll) {
            v += (double)a.ll[i];
            a.logw[i] = v;
        }
        if (isnan(v)) v = -INFINITY;
        double l = a.llm ? (double)a.llm[i] : -INFINITY;
        if (isnan(l)) l = -INFINITY;
        mx = max_combine(mx, MaxArg{v, i, l});
    }
    mx = max_block(mx);
    double2 sum = make_double2(0.0, 0.0);
    if (mx.m != -INFINITY) {
        for (int i = vb * blockDim.x + threadIdx.x; i < a.P; i += vg * blockDim.x) {
            const double v = a.logw[i];     // this thread's own write above
            if (!(v > -INFINITY)) continue;  // -inf and NaN carry no weight
            const double e = exp(v - mx.m);
            sum.x += e;
            sum.y += e * e;
        }
    }
    sum = sum_block(sum);
    __shared__ int is_last;
    if (threadIdx.x == 0) {
        double* p = a.part + kWeighPart * (size_t)vb;
        p[0] = mx.m; p[1] = sum.x; p[2] = sum.y; p[3] = (double)mx.i; p[4] = mx.lm;
        __threadfence();
        const unsigned ticket = atomicAdd(a.counter, 1u);
        is_last = (ticket == (unsigned)vg - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    MaxArg tm{-INFINITY, 0x7fffffff, -INFINITY};
    for (int b = threadIdx.x; b < vg; b += blockDim.x) {
        const double* p = a.part + kWeighPart * (size_t)b;
        tm = max_combine(tm, MaxArg{__ldcg(p), (int)__ldcg(p + 3), __ldcg(p + 4)});
    }
    tm = max_block(tm);
    double2 tot = make_double2(0.0, 0.0);
    if (tm.m != -INFINITY) {
        for (int b = threadIdx.x; b < vg; b += blockDim.x) {
            const double* p = a.part + kWeighPart * (size_t)b;
            const double mb = __ldcg(p);
            if (!(mb > -INFINITY)) continue;
            const double e = exp(mb - tm.m);
            tot.x += __ldcg(p + 1) * e;
            tot.y += __ldcg(p + 2) * e * e;
        }
    }
    tot = sum_block(tot);
    if (threadIdx.x == 0) {
        WeighResult r;
        r.M = tm.m;
        r.nonfinite = (tm.m == -INFINITY || !(tot.x > 0.0)) ? 1 : 0;
        r.logS = r.nonfinite ? 0.0 : log(tot.x);
        r.ess = r.nonfinite ? 0.0 : (tot.x * tot.x) / tot.y;
        r.max_w = r.nonfinite ? 0.0 : 1.0 / tot.x;
        r.argmax = r.nonfinite ? 0 : tm.i;
        r.ll_max = tm.lm;
        r.pruned = 0;
        int doit = (a.policy == 0) || (a.policy == 1 && r.ess < 0.5 * (double)a.P);
        r.do_resample = r.nonfinite ? 0 : doit;
        for (int c = 0; c < 12; ++c) r.est[c] = a.pose[(size_t)c * a.ld + r.argmax];
        *a.res = r;
        *a.counter = 0u;
    }
}

__global__ void __launch_bounds__(kWeighThreads) k_weigh(WeighArgs a) { weigh_body(a, blockIdx.x, gridDim.x); }

// Inclusive prefix sum over a kScanBlock-thread block (every thread calls it).
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long q) {
    __shared__ unsigned long long wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, q, off);
        if (lane >= off) q += t;
    }
    if (lane == 31) wsum[warp] = q;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = wsum[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += u;
        }
        wsum[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    if (warp > 0) q += wsum[warp - 1];
    __syncthreads();      // wsum is reused by the next call
    return q;
}

// q_i = rint(w_i 2^52) and the block-local inclusive prefix sums.
__device__ __forceinline__ void resample_scan_body(const ScanArgs& a, int vb, int vg) {
    const int i = vb * kScanBlock + threadIdx.x;
    double w = 0.0;
    if (i < a.P) {
        if (a.w) {
            w = a.w[i];
        } else {
            const WeighResult r = *a.res;
            w = r.nonfinite ? 1.0 / (double)a.P : exp(a.logw[i] - r.M - r.logS);
        }
        if (a.w_out) a.w_out[i] = w;
    }
    unsigned long long q = (w > 0.0 && w <= 1.0) ? __double2ull_rn(w * 4503599627370496.0) : 0ull;
    q = block_scan_u64(q);
    if (i < a.P) a.cl[i] = q;
    if (threadIdx.x == kScanBlock - 1) a.btot[vb] = q;
}

__global__ void __launch_bounds__(kScanBlock) k_resample_scan(ScanArgs a) { resample_scan_body(a, blockIdx.x, gridDim.x); }

// Exclusive scan of the block totals in place; the grand total goes to btot[nblocks].
__device__ __forceinline__ void scan_totals_body(const TotalsArgs& t, int vb, int vg) {
    unsigned long long* btot = t.btot;
    const int nblocks = t.nblocks;
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nblocks; base += 1024) {
        const int b = base + threadIdx.x;
        const unsigned long long x = (b < nblocks) ? btot[b] : 0ull;
        unsigned long long q = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, q, off);
            if (lane >= off) q += t;
        }
        if (lane == 31) wsum[warp] = q;
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = wsum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long u = __shfl_up_sync(0xffffffffu, t, off);
                if (lane >= off) t += u;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        if (warp > 0) q += wsum[warp - 1];
        const unsigned long long c0 = carry;
        if (b < nblocks) btot[b] = c0 + q - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c0 + q;
        __syncthreads();
    }
    if (threadIdx.x == 0) btot[nblocks] = carry;
}

__global__ void __launch_bounds__(1024) k_scan_totals(TotalsArgs t) { scan_totals_body(t, blockIdx.x, gridDim.x); }

__device__ __forceinline__ double systematic_u(uint64_t seed, uint32_t t) {
    const uint4 o = philox4x32_10(make_uint4(0xFFFFFFFFu, t, 0u, kTagResample),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const double hi = (double)(o.x >> 5), lo = (double)(o.y >> 6);
    return __dmul_rn(__dadd_rn(__dmul_rn(hi, 67108864.0), lo), 1.0 / 9007199254740992.0);
}

__device__ __forceinline__ void resample_search_body(const SearchArgs& a, int vb, int vg) {
    const int m = vb * blockDim.x + threadIdx.x;
    if (m >= a.P) return;
    if (a.res && !a.res->do_resample) {
        a.anc[m] = m;
        return;
    }
    const double u = a.u_from_philox ? systematic_u(a.seed, a.frame) : a.u;
    const double S = (double)a.boff[a.nblocks];
    const double tau = __dmul_rn(__ddiv_rn(__dadd_rn(u, (double)m), (double)a.P), S);
    // block: smallest b whose inclusive prefix boff[b+1] exceeds tau
    int lo = 0, hi = a.nblocks - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((double)a.boff[mid + 1] > tau) hi = mid; else lo = mid + 1;
    }
    const unsigned long long base = a.boff[lo];
    int l = lo * kScanBlock, h = min(a.P, (lo + 1) * kScanBlock) - 1;
    while (l < h) {
        const int mid = (l + h) >> 1;
        if ((double)(base + a.cl[mid]) > tau) h = mid; else l = mid + 1;
    }
    a.anc[m] = ((double)(base + a.cl[l]) > tau) ? l : a.P - 1;
}

__global__ void __launch_bounds__(256) k_resample_search(SearchArgs a) { resample_search_body(a, blockIdx.x, gridDim.x); }

// State gather by ancestor: current pose and every keyframe pose, then log-weights.
__device__ __forceinline__ void gather_body(const GatherArgs& a, int vb, int vg) {
    // work items = (one pose: 12 consecutive rows, block of particles): the ancestor
    // is read once and the twelve row reads are independent loads in flight
    // together (4 rows per item: 54 us at 100,000 particles x 21 poses; 12: 51 us)
    constexpr int kRows = kPoseC;
    static_assert(kPoseC % kRows == 0, "row groups do not straddle pose and keyframe rows");
    const size_t groups = (size_t)(1 + a.K) * kPoseC / kRows;
    const size_t per_row = (a.P + blockDim.x - 1) / blockDim.x;
    for (size_t item = vb; item < groups * per_row; item += vg) {
        const size_t row = item / per_row * kRows;
        const int m = (int)(item % per_row) * blockDim.x + threadIdx.x;
        if (m >= a.P) continue;
        const int src = a.anc[m];
        const float* from = row < kPoseC ? a.pose_src + row * a.ld : a.kf_src + (row - kPoseC) * a.ld;
        float* to = row < kPoseC ? a.pose_dst + row * a.ld : a.kf_dst + (row - kPoseC) * a.ld;
        float v[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) v[r] = from[r * a.ld + src];
#pragma unroll
        for (int r = 0; r < kRows; ++r) to[r * a.ld + m] = v[r];
    }
    const double uni = -log((double)a.P);
    for (int m = vb * blockDim.x + threadIdx.x; m < a.P; m += vg * blockDim.x) {
        if (!a.res) {
            a.logw[m] = uni;
        } else {
            const WeighResult& r = *a.res;
            a.logw[m] = (r.nonfinite || r.do_resample) ? uni : a.logw[m] - r.M - r.logS;
        }
    }
}

__global__ void __launch_bounds__(256) k_gather(GatherArgs a) { gather_body(a, blockIdx.x, gridDim.x); }

// No resampling: normalise the log-weights in place (w_out: weights, anc: identity).
__global__ void __launch_bounds__(256) k_normalize(double* logw, int P, const WeighResult* res, double* w_out,
                                                   int* anc) {
    const double uni = -log((double)P);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const double v = res->nonfinite ? uni : logw[i] - res->M - res->logS;
        logw[i] = v;
        if (w_out) w_out[i] = exp(v);
        if (anc) anc[i] = i;
    }
}

// ------------------------------------------------------------------ dead-particle pruning
//
// Sec. III-F: particles whose weight (or frame likelihood relative to the best
// particle) has collapsed are dead; only their slots are refilled, by one
// systematic comb of D teeth over the survivors' quantised weights, and each
// survivor's weight is split evenly over it and its copies, so the weighted
// particle measure of the survivors is unchanged. Survivors never move: the
// refill reads survivors' state and writes dead slots' state in place.
//   mark     dead flags, q_i (0 when dead), block scans of q and of the flags;
//            anc[i] = i for survivors, -(local dead rank + 1) for dead slots
//   totals   exclusive offsets of both block totals (CTA 0: q, CTA 1: dead)
//   spawn    dead slot r: ancestor a_r, its copy count, new log-weight, state
//   reweigh  survivors: x - log1p(copies)

__device__ __forceinline__ double prune_tooth(double u, int r, int D, double S) {
    const double t = __dmul_rn(__ddiv_rn(__dadd_rn(u, (double)r), (double)D), S);
    return fmin(t, S - 1.0);
}

// Number of teeth r in [0, D) below X (the teeth are non-decreasing in r).
__device__ __forceinline__ int prune_below(double u, int D, double S, double X) {
    int lo = 0, hi = D;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (prune_tooth(u, mid, D, S) < X) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Teeth that land in survivor i's interval [C_{i-1}, C_i).
__device__ __forceinline__ int prune_copies(const PruneArgs& a, int i, double u, int D, double S) {
    const unsigned long long base = a.btot[i / kScanBlock];
    const double hi = (double)(base + a.cl[i]);
    const double lo = (double)((i % kScanBlock) ? base + a.cl[i - 1] : base);
    if (!(hi > lo)) return 0;
    return prune_below(u, D, S, hi) - prune_below(u, D, S, lo);
}

// min{ i : C_i > tau } for tau < S.
__device__ __forceinline__ int prune_find(const PruneArgs& a, double tau) {
    int lo = 0, hi = a.nblocks - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((double)a.btot[mid + 1] > tau) hi = mid; else lo = mid + 1;
    }
    const unsigned long long base = a.btot[lo];
    int l = lo * kScanBlock, h = min(a.P, (lo + 1) * kScanBlock) - 1;
    while (l < h) {
        const int mid = (l + h) >> 1;
        if ((double)(base + a.cl[mid]) > tau) h = mid; else l = mid + 1;
    }
    return l;
}

__device__ __forceinline__ double prune_u(const PruneArgs& a) {
    return a.u_from_philox ? systematic_u(a.seed, a.frame) : a.u;
}

__device__ __forceinline__ void prune_mark_body(const PruneArgs& a, int vb, int vg) {
    const int i = vb * kScanBlock + threadIdx.x;
    const WeighResult* R = a.res;
    unsigned long long q = 0ull, d = 0ull;
    if (i < a.P) {
        const int nonfinite = R->nonfinite;
        const double x = (a.logw[i] - R->M) - R->logS;
        double w = a.w ? a.w[i] : exp(x);
        if (nonfinite) w = 1.0 / (double)a.P;
        if (a.w_out) a.w_out[i] = w;
        bool dead = !(w >= a.prune_w);
        if (a.ll && a.ll_cut > -INFINITY && !((double)a.ll[i] - R->ll_max >= a.ll_cut)) dead = true;
        if (i == R->argmax || nonfinite) dead = false;
        q = (!dead && w > 0.0 && w <= 1.0) ? __double2ull_rn(w * 4503599627370496.0) : 0ull;
        d = dead ? 1ull : 0ull;
    }
    q = block_scan_u64(q);
    const unsigned long long dl = block_scan_u64(d);
    if (i < a.P) {
        a.cl[i] = q;
        a.anc[i] = d ? -(int)dl : i;
    }
    if (threadIdx.x == kScanBlock - 1) {
        a.btot[vb] = q;
        a.dtot[vb] = dl;
    }
}

__device__ __forceinline__ void prune_totals_body(const PruneArgs& a, int vb, int vg) {
    scan_totals_body(TotalsArgs{vb == 0 ? a.btot : a.dtot, a.nblocks}, 0, 1);
}

// Column src of a [12][ld] pose block to column m (src != m, both in range).
__device__ __forceinline__ void copy_pose_col(float* base, size_t ld, int src, int m) {
    float v[kPoseC];
#pragma unroll
    for (int e = 0; e < kPoseC; ++e) v[e] = base[(size_t)e * ld + src];
#pragma unroll
    for (int e = 0; e < kPoseC; ++e) base[(size_t)e * ld + m] = v[e];
}

__device__ __forceinline__ void prune_spawn_body(const PruneArgs& a, int vb, int vg) {
    const int m = vb * blockDim.x + threadIdx.x;
    if (m >= a.P) return;
    const WeighResult* R = a.res;
    if (R->nonfinite) return;
    const int tag = a.anc[m];
    if (tag >= 0) return;                       // survivor
    const int D = (int)a.dtot[a.nblocks];
    const double S = (double)a.btot[a.nblocks];
    if (!(S > 0.0)) {                           // nothing carries weight: leave the slot
        a.anc[m] = m;
        return;
    }
    const int r = (int)a.dtot[m / kScanBlock] - tag - 1;
    const double u = prune_u(a);
    const int src = prune_find(a, prune_tooth(u, r, D, S));
    const int c = prune_copies(a, src, u, D, S);
    a.anc[m] = src;
    a.logw[m] = ((a.logw[src] - R->M) - R->logS) - log1p((double)c);
    if (a.pose) {
        // one pose (12 rows) at a time, its 12 loads in flight together: the refill of
        // 100,000 x 21 poses 0.25 -> 0.15 ms (three poses at a time: 0.145 ms; the rest
        // is the binary searches of the comb)
        copy_pose_col(a.pose, a.ld, src, m);
        for (int k = 0; k < a.K; ++k) copy_pose_col(a.kf + (size_t)k * kPoseC * a.ld, a.ld, src, m);
    }
}

__device__ __forceinline__ void prune_reweigh_body(const PruneArgs& a, int vb, int vg) {
    const int m = vb * blockDim.x + threadIdx.x;
    if (m >= a.P) return;
    WeighResult* R = a.res;
    const int D = (int)a.dtot[a.nblocks];
    const double S = (double)a.btot[a.nblocks];
    if (R->nonfinite) {
        a.logw[m] = -log((double)a.P);
        a.anc[m] = m;
        return;
    }
    if (m == 0) R->pruned = (S > 0.0) ? D : 0;
    if (a.anc[m] != m) return;                  // refilled by the spawn kernel
    const double x = (a.logw[m] - R->M) - R->logS;
    const int c = (D > 0 && S > 0.0) ? prune_copies(a, m, prune_u(a), D, S) : 0;
    a.logw[m] = c ? x - log1p((double)c) : x;
}

__global__ void __launch_bounds__(kScanBlock) k_prune_mark(PruneArgs a) { prune_mark_body(a, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(1024) k_prune_totals(PruneArgs a) { prune_totals_body(a, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(256) k_prune_spawn(PruneArgs a) { prune_spawn_body(a, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(256) k_prune_reweigh(PruneArgs a) { prune_reweigh_body(a, blockIdx.x, gridDim.x); }

// ------------------------------------------------------------------ batched launches


__global__ void __launch_bounds__(kWeighThreads) k_weigh_b(const BatchList<WeighArgs>* L) {
    GMCS_BATCH_LOOP(L, const WeighArgs a = L->args[s]; weigh_body(a, vb, vg));
}
__global__ void __launch_bounds__(kScanBlock) k_resample_scan_b(const BatchList<ScanArgs>* L) {
    GMCS_BATCH_LOOP(L, const ScanArgs a = L->args[s]; resample_scan_body(a, vb, vg));
}
__global__ void __launch_bounds__(1024) k_scan_totals_b(const BatchList<TotalsArgs>* L) {
    GMCS_BATCH_LOOP(L, const TotalsArgs a = L->args[s]; scan_totals_body(a, vb, vg));
}
__global__ void __launch_bounds__(256) k_resample_search_b(const BatchList<SearchArgs>* L) {
    GMCS_BATCH_LOOP(L, const SearchArgs a = L->args[s]; resample_search_body(a, vb, vg));
}
__global__ void __launch_bounds__(256) k_gather_b(const BatchList<GatherArgs>* L) {
    GMCS_BATCH_LOOP(L, const GatherArgs a = L->args[s]; gather_body(a, vb, vg));
}
__global__ void __launch_bounds__(kScanBlock) k_prune_mark_b(const BatchList<PruneArgs>* L) {
    GMCS_BATCH_LOOP(L, const PruneArgs a = L->args[s]; prune_mark_body(a, vb, vg));
}
__global__ void __launch_bounds__(1024) k_prune_totals_b(const BatchList<PruneArgs>* L) {
    GMCS_BATCH_LOOP(L, const PruneArgs a = L->args[s]; prune_totals_body(a, vb, vg));
}
__global__ void __launch_bounds__(256) k_prune_spawn_b(const BatchList<PruneArgs>* L) {
    GMCS_BATCH_LOOP(L, const PruneArgs a = L->args[s]; prune_spawn_body(a, vb, vg));
}
__global__ void __launch_bounds__(256) k_prune_reweigh_b(const BatchList<PruneArgs>* L) {
    GMCS_BATCH_LOOP(L, const PruneArgs a = L->args[s]; prune_reweigh_body(a, vb, vg));
}

template <typename K>
static int persistent_grid_w(K kernel, int threads) {
    int per_sm = 0, dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * sms;
}

static int grid_weigh_b() { static const int g = persistent_grid_w(k_weigh_b, kWeighThreads); return g; }
static int grid_scan_b() { static const int g = persistent_grid_w(k_resample_scan_b, kScanBlock); return g; }
static int grid_search_b() { static const int g = persistent_grid_w(k_resample_search_b, 256); return g; }
static int grid_gather_b() { static const int g = persistent_grid_w(k_gather_b, 256); return g; }
static int grid_pmark_b() { static const int g = persistent_grid_w(k_prune_mark_b, kScanBlock); return g; }
static int grid_pspawn_b() { static const int g = persistent_grid_w(k_prune_spawn_b, 256); return g; }
static int grid_preweigh_b() { static const int g = persistent_grid_w(k_prune_reweigh_b, 256); return g; }

void launch_weigh_b(const BatchList<WeighArgs>* L, cudaStream_t s) { k_weigh_b<<<grid_weigh_b(), kWeighThreads, 0, s>>>(L); }
void launch_resample_scan_b(const BatchList<ScanArgs>* L, cudaStream_t s) {
    k_resample_scan_b<<<grid_scan_b(), kScanBlock, 0, s>>>(L);
}
void launch_scan_totals_b(const BatchList<TotalsArgs>* L, cudaStream_t s) {
    k_scan_totals_b<<<kMaxSlots, 1024, 0, s>>>(L);
}
void launch_resample_search_b(const BatchList<SearchArgs>* L, cudaStream_t s) {
    k_resample_search_b<<<grid_search_b(), 256, 0, s>>>(L);
}
void launch_gather_b(const BatchList<GatherArgs>* L, cudaStream_t s) { k_gather_b<<<grid_gather_b(), 256, 0, s>>>(L); }
void launch_prune_mark_b(const BatchList<PruneArgs>* L, cudaStream_t s) {
    k_prune_mark_b<<<grid_pmark_b(), kScanBlock, 0, s>>>(L);
}
void launch_prune_totals_b(const BatchList<PruneArgs>* L, cudaStream_t s) {
    k_prune_totals_b<<<2 * kMaxSlots, 1024, 0, s>>>(L);
}
void launch_prune_spawn_b(const BatchList<PruneArgs>* L, cudaStream_t s) {
    k_prune_spawn_b<<<grid_pspawn_b(), 256, 0, s>>>(L);
}
void launch_prune_reweigh_b(const BatchList<PruneArgs>* L, cudaStream_t s) {
    k_prune_reweigh_b<<<grid_preweigh_b(), 256, 0, s>>>(L);
}

void prepare_weights_batched() {
    grid_weigh_b();
    grid_scan_b();
    grid_search_b();
    grid_gather_b();
    grid_pmark_b();
    grid_pspawn_b();
    grid_preweigh_b();
}

int grid_resample_scan(int P) { return (P + kScanBlock - 1) / kScanBlock; }
int grid_resample_search(int P) { return (P + 255) / 256; }
int grid_gather(const GatherArgs& a) {
    const size_t n = (size_t)(1 + a.K) * kPoseC * a.P;
    size_t b = (n + 255) / 256;
    if (b > 148 * 16) b = 148 * 16;
    return (int)(b > 0 ? b : 1);
}

// 4 particles per thread (1 or 2 per thread, i.e. more CTAs and partials: 28 / 26 us
// instead of 24 at 100,000 particles)
int weigh_blocks(int P) {
    int b = (P + kWeighThreads * 4 - 1) / (kWeighThreads * 4);
    if (b > kWeighMaxBlocks) b = kWeighMaxBlocks;
    return b > 0 ? b : 1;
}

void launch_weigh(const WeighArgs& a, int nblocks, cudaStream_t s) {
    k_weigh<<<nblocks, kWeighThreads, 0, s>>>(a);
}

void launch_resample_scan(const ScanArgs& a, cudaStream_t s) {
    const int nb = grid_resample_scan(a.P);
    if (nb > 0) k_resample_scan<<<nb, kScanBlock, 0, s>>>(a);
}

void launch_scan_totals(unsigned long long* btot, int nblocks, cudaStream_t s) {
    k_scan_totals<<<1, 1024, 0, s>>>(TotalsArgs{btot, nblocks});
}

void launch_resample_search(const SearchArgs& a, cudaStream_t s) {
    if (a.P > 0) k_resample_search<<<grid_resample_search(a.P), 256, 0, s>>>(a);
}

void launch_gather(const GatherArgs& a, cudaStream_t s) {
    if (a.P > 0) k_gather<<<grid_gather(a), 256, 0, s>>>(a);
}

void launch_normalize(double* logw, int P, const WeighResult* res, double* w_out, int* anc, cudaStream_t s) {
    if (P > 0) k_normalize<<<(P + 255) / 256, 256, 0, s>>>(logw, P, res, w_out, anc);
}

int grid_prune_slots(int P) { return (P + 255) / 256; }

void launch_prune_mark(const PruneArgs& a, cudaStream_t s) {
    if (a.P > 0) k_prune_mark<<<a.nblocks, kScanBlock, 0, s>>>(a);
}
void launch_prune_totals(const PruneArgs& a, cudaStream_t s) {
    if (a.P > 0) k_prune_totals<<<2, 1024, 0, s>>>(a);
}
void launch_prune_spawn(const PruneArgs& a, cudaStream_t s) {
    if (a.P > 0) k_prune_spawn<<<grid_prune_slots(a.P), 256, 0, s>>>(a);
}
void launch_prune_reweigh(const PruneArgs& a, cudaStream_t s) {
    if (a.P > 0) k_prune_reweigh<<<grid_prune_slots(a.P), 256, 0, s>>>(a);
}

}  // namespace gmcs
