"""ctypes binding of the FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline / reference arm. The CUDA product path never imports
it. Function names follow oracle.h; arrays are numpy, poses are (..., 12)
row-major [R | t].
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)
_u32p = C.POINTER(C.c_uint32)


class Grid(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("h", C.c_double), ("n", C.c_int * 3), ("coef", C.c_int)]


class EvalParams(C.Structure):
    _fields_ = [("eps", C.c_double), ("face_delta", C.c_double)]


class MoveParams(C.Structure):
    _fields_ = [("sigma", C.c_double), ("lambda_", C.c_double), ("theta_max", C.c_double),
                ("t_max", C.c_double), ("w_min", C.c_double)]


class StepParams(C.Structure):
    _fields_ = [("sigma", C.c_double), ("eps", C.c_double), ("lambda_", C.c_double),
                ("theta_max", C.c_double), ("t_max", C.c_double), ("w_min", C.c_double),
                ("face_delta", C.c_double), ("k_nb", C.c_int), ("steps", C.c_int),
                ("resample", C.c_int), ("propagate", C.c_int), ("loop_recent", C.c_int), ("model", C.c_int),
                ("gicp_tau", C.c_double), ("prune_w", C.c_double), ("ll_cut", C.c_double), ("seed", C.c_uint64)]


class StepOut(C.Structure):
    _fields_ = [("estimate", C.c_double * 12), ("ess", C.c_double), ("max_w", C.c_double),
                ("argmax", C.c_int), ("resampled", C.c_int), ("pruned", C.c_int), ("pad", C.c_int)]


DEFAULTS = dict(sigma=0.2, eps=1e-3, lambda_=1e-3, theta_max=np.deg2rad(2.0), t_max=0.1,
                w_min=1e-6, face_delta=1e-3, k_nb=3, steps=3, resample=0, propagate=0, loop_recent=0, model=0,
                gicp_tau=20.0, prune_w=1e-8, ll_cut=float(np.log(1e-16)), seed=0)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        L.ora_systematic_u.restype = C.c_double
        L.ora_cell_eval.restype = C.c_int
        _LIB = L
    return _LIB


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_fp)


def make_grid(g, table=None):
    """ora_grid of a lattice dict; a 4-D table (cells x 8 coefficients) marks a
    coefficient table."""
    gr = Grid()
    for a in range(3):
        gr.origin[a] = float(g["origin"][a])
        gr.n[a] = int(g["dims"][a])
    gr.h = float(g["h"])
    gr.coef = 1 if (table is not None and np.ndim(table) == 4) else 0
    return gr


# ---------------------------------------------------------------- SE(3)
def pose_mul(A, B):
    A, pa = _d(A); B, pb = _d(B)
    out = np.zeros(12)
    lib().ora_pose_mul(pa, pb, out.ctypes.data_as(_dp))
    return out


def pose_inv(A):
    A, pa = _d(A)
    out = np.zeros(12)
    lib().ora_pose_inv(pa, out.ctypes.data_as(_dp))
    return out


def se3_exp(xi):
    xi, px = _d(xi)
    out = np.zeros(12)
    lib().ora_se3_exp(px, out.ctypes.data_as(_dp))
    return out


def se3_log(T):
    T, pt = _d(T)
    out = np.zeros(6)
    lib().ora_se3_log(pt, out.ctypes.data_as(_dp))
    return out


def se3_jr(xi):
    xi, px = _d(xi)
    J = np.zeros(36)
    lib().ora_se3_jr(px, J.ctypes.data_as(_dp))
    return J.reshape(6, 6)


def loglik_grad_xi(T0, xi, Tk, tables, grids, scan, eps=1e-3, face_delta=1e-3):
    """l(T0 exp(xi)) and its derivative in xi: Jr(xi)^T times the right-perturbation
    gradient at T0 exp(xi); slack and gradient mass are mapped the same way."""
    T = pose_mul(T0, se3_exp(xi))
    o = eval_particle(T, Tk, tables, grids, scan, eps, face_delta)
    J = se3_jr(xi)
    o["g_xi"] = J.T @ o["g"]
    o["jr_norm"] = float(np.linalg.norm(J, 2))
    return o


# ---------------------------------------------------------------- random draws
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normal6(seed, i, t):
    z = np.zeros(6)
    lib().ora_normal6(C.c_uint64(seed), C.c_uint32(i), C.c_uint32(t), z.ctypes.data_as(_dp))
    return z


def systematic_u(seed, t):
    return float(lib().ora_systematic_u(C.c_uint64(seed), C.c_uint32(t)))


# ---------------------------------------------------------------- tables
def build_table(pts, grid, sigma=0.2, r_t=1.0, brute=False):
    pts, pp = _f(pts)
    gr = make_grid(grid)
    nx, ny, nz = grid["dims"]
    vals = np.zeros((nz, ny, nx))
    fn = lib().ora_build_table_brute if brute else lib().ora_build_table
    fn(pp, C.c_int(pts.shape[0]), C.byref(gr), C.c_double(sigma), C.c_double(r_t), vals.ctypes.data_as(_dp))
    return vals


def quantize(vals, dtype):
    """dtype 1 = bfloat16, 2 = float16, both round-to-nearest-even."""
    v, pv = _d(vals)
    out = np.zeros_like(v)
    lib().ora_quantize(pv, C.c_size_t(v.size), C.c_int(dtype), out.ctypes.data_as(_dp))
    return out


def coef_table(vals):
    """Per-cell coefficients c0..c7 (FP64) of the trilinear interpolation of a
    vertex table (nz, ny, nx): array (nz-1, ny-1, nx-1, 8) with
      L = c0 + c1 x + c2 y + c3 z + c4 xy + c5 xz + c6 yz + c7 xyz
    in the in-cell fraction, by inclusion-exclusion over the corners."""
    v = np.asarray(vals, np.float64)
    V = {(dx, dy, dz): v[dz:v.shape[0] - 1 + dz, dy:v.shape[1] - 1 + dy, dx:v.shape[2] - 1 + dx]
         for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)}
    c = np.empty(v[:-1, :-1, :-1].shape + (8,))
    c[..., 0] = V[0, 0, 0]
    c[..., 1] = V[1, 0, 0] - V[0, 0, 0]
    c[..., 2] = V[0, 1, 0] - V[0, 0, 0]
    c[..., 3] = V[0, 0, 1] - V[0, 0, 0]
    c[..., 4] = V[1, 1, 0] - V[1, 0, 0] - V[0, 1, 0] + V[0, 0, 0]
    c[..., 5] = V[1, 0, 1] - V[1, 0, 0] - V[0, 0, 1] + V[0, 0, 0]
    c[..., 6] = V[0, 1, 1] - V[0, 1, 0] - V[0, 0, 1] + V[0, 0, 0]
    c[..., 7] = (V[1, 1, 1] - V[1, 1, 0] - V[1, 0, 1] - V[0, 1, 1]
                 + V[1, 0, 0] + V[0, 1, 0] + V[0, 0, 1] - V[0, 0, 0])
    return c


# Storage of the 16-bit coefficient records (the library's table format, not the
# paper's): the coefficients are taken in FP32; the record's word e (e = 0..3)
# holds HI[e] in its high half and LO[e] in its low half.
_REC_HI = (4, 2, 7, 6)
_REC_LO = (1, 0, 5, 3)


def _bf16_rn_bits(x32):
    """bfloat16 bits (uint32, in the low half) of float32 values, rounded to nearest even."""
    b = x32.view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return r.astype(np.uint32)


def quantize_coef(coef, dtype):
    """The coefficients (..., 8) as a 16-bit record stores them, widened to FP64.
    FP16 (dtype 2): each rounded to nearest even. BF16 (dtype 1): LO[e] rounded to
    bfloat16; HI[e] becomes the FP32 number whose low 16 bits are those bfloat16
    bits and whose value is nearest to HI[e] (ties to the candidate that keeps
    HI[e]'s own high half)."""
    c32 = np.asarray(coef, np.float64).astype(np.float32)
    out = c32.astype(np.float64)
    if dtype == 2:
        return c32.astype(np.float16).astype(np.float64)
    assert dtype == 1
    for hi, lo in zip(_REC_HI, _REC_LO):
        lo16 = _bf16_rn_bits(np.ascontiguousarray(c32[..., lo]))
        out[..., lo] = (lo16 << np.uint32(16)).view(np.float32).astype(np.float64)
        A = c32[..., hi]
        base = (A.view(np.uint32) & np.uint32(0xFFFF0000)) | lo16
        mag = (base >> np.uint32(16)) & np.uint32(0x7FFF)
        best = base.copy()
        a64 = A.astype(np.float64)
        err = np.abs(a64 - base.view(np.float32).astype(np.float64))
        with np.errstate(invalid="ignore", over="ignore"):
            for cand, ok in ((base - np.uint32(0x10000), mag > 0), (base + np.uint32(0x10000), mag < 0x7F7F)):
                e = np.abs(a64 - cand.view(np.float32).astype(np.float64))
                take = ok & (e < err)
                best = np.where(take, cand, best)
                err = np.where(take, e, err)
        out[..., hi] = best.view(np.float32).astype(np.float64)
    return out


def stored_table(vals, dtype):
    """What the lookups of a table with storage type dtype evaluate, from the FP64
    vertex table: FP32 (0) the vertex table itself (the FP32 coefficients are
    differences of the float corners, within ~2.4e-7 of it); BF16 (1) and FP16 (2)
    the cell coefficients as the 16-bit records store them (quantize_coef)."""
    if dtype == 0:
        return np.asarray(vals, np.float64)
    return quantize_coef(coef_table(vals), dtype)


def cell_eval(vals, grid, c, u):
    gr = make_grid(grid, vals)
    v, pv = _d(vals)
    ci = (C.c_int * 3)(*[int(x) for x in c])
    uu = (C.c_double * 3)(*[float(x) for x in u])
    L = C.c_double()
    d = (C.c_double * 3)()
    ok = lib().ora_cell_eval(pv, C.byref(gr), ci, uu, C.byref(L), d)
    return ok, L.value, np.array(list(d))


# ---------------------------------------------------------------- evaluation
def eval_particle(Tt, Tk, tables, grids, scan, eps=1e-3, face_delta=1e-3, cells=None, frozen=False,
                  want_cells=False):
    """Tk: (n_nb, 12); tables: list of (nz, ny, nx) arrays; grids: list of dicts."""
    Tt, pt = _d(Tt)
    Tk = np.ascontiguousarray(np.asarray(Tk, np.float64).reshape(-1, 12))
    n_nb = Tk.shape[0]
    tabs = [np.ascontiguousarray(t, np.float64) for t in tables]
    tab_ptrs = (_dp * max(n_nb, 1))(*[t.ctypes.data_as(_dp) for t in tabs])
    grs = (Grid * max(n_nb, 1))(*[make_grid(g, t) for g, t in zip(grids, tabs)])
    scan, ps = _f(scan)
    N = scan.shape[0]
    prm = EvalParams(eps, face_delta)
    ll = C.c_double()
    g = np.zeros(6)
    mom = np.zeros(10)
    slack = C.c_double()
    gabs = C.c_double()
    if cells is None and (want_cells or frozen):
        cells = np.zeros((n_nb, N, 3), np.int32)
    cp = None
    if cells is not None:
        cells = np.ascontiguousarray(cells, np.int32)
        cp = cells.ctypes.data_as(_ip)
    lib().ora_eval_particle(pt, C.c_int(n_nb), Tk.ctypes.data_as(_dp), tab_ptrs, grs, ps, C.c_int(N),
                            C.byref(prm), C.byref(ll), g.ctypes.data_as(_dp), mom.ctypes.data_as(_dp),
                            C.byref(slack), C.byref(gabs), cp, C.c_int(1 if frozen else 0))
    out = {"ll": ll.value, "g": g, "mom": mom, "slack": slack.value, "gabs": gabs.value}
    if cells is not None:
        out["cells"] = cells
    return out


def eval_batch(poses, nbr, kf_poses, tables, grids, scan, eps=1e-3, face_delta=1e-3, idx=None):
    """Per-particle evaluation over a set. kf_poses: (K, P, 12); nbr: (P, n_nb).
    idx restricts to a subset of particle indices."""
    poses = np.asarray(poses, np.float64).reshape(-1, 12)
    P = poses.shape[0]
    idx = np.arange(P) if idx is None else np.asarray(idx)
    res = {"ll": np.zeros(len(idx)), "g": np.zeros((len(idx), 6)), "mom": np.zeros((len(idx), 10)),
           "slack": np.zeros(len(idx)), "gabs": np.zeros(len(idx))}
    for r, i in enumerate(idx):
        ks = [int(k) for k in nbr[i] if k >= 0]
        o = eval_particle(poses[i], [kf_poses[k][i] for k in ks], [tables[k] for k in ks],
                          [grids[k] for k in ks], scan, eps, face_delta)
        res["ll"][r] = o["ll"]; res["g"][r] = o["g"]; res["mom"][r] = o["mom"]; res["slack"][r] = o["slack"]
        res["gabs"][r] = o["gabs"]
    return res


def h_from_moments(mom, sigma=0.2):
    m, pm = _d(mom)
    H = np.zeros(36)
    lib().ora_h_from_moments(pm, C.c_double(sigma), H.ctypes.data_as(_dp))
    return H.reshape(6, 6)


def h_explicit(scan, w, sigma=0.2):
    s, ps = _f(scan)
    w, pw = _d(w)
    H = np.zeros(36)
    lib().ora_h_explicit(ps, C.c_int(s.shape[0]), pw, C.c_double(sigma), H.ctypes.data_as(_dp))
    return H.reshape(6, 6)


def move(Tt, g, mom, sigma=0.2, lambda_=1e-3, theta_max=np.deg2rad(2.0), t_max=0.1, w_min=1e-6):
    Tt, pt = _d(Tt); g, pg = _d(g); mom, pm = _d(mom)
    mp = MoveParams(sigma, lambda_, theta_max, t_max, w_min)
    Tout = np.zeros(12)
    psi = np.zeros(6)
    lib().ora_move(pt, pg, pm, C.byref(mp), Tout.ctypes.data_as(_dp), psi.ctypes.data_as(_dp))
    return Tout, psi


def select_nbrs(Tt, kf_t, k_nb=3):
    Tt, pt = _d(Tt)
    kf_t, pk = _d(np.asarray(kf_t).reshape(-1, 3))
    idx = np.full(k_nb, -1, np.int32)
    lib().ora_select_nbrs(pt, pk, C.c_int(kf_t.shape[0]), C.c_int(k_nb), idx.ctypes.data_as(_ip))
    return idx


def predict(T, dT, cov, z):
    T, pt = _d(T); dT, pd = _d(dT); cov, pc = _d(np.asarray(cov).reshape(36)); z, pz = _d(z)
    out = np.zeros(12)
    lib().ora_predict(pt, pd, pc, pz, out.ctypes.data_as(_dp))
    return out


def propagate(psi, nbr, kf_path, path_now, kf_i):
    """Eq. 8-10 on one particle's keyframe poses kf_i (K x 12), returned updated."""
    psi, pp = _d(psi)
    nb = np.ascontiguousarray(nbr, np.int32)
    D, pd = _d(kf_path)
    kf = np.ascontiguousarray(np.asarray(kf_i, np.float64).reshape(-1, 12)).copy()
    lib().ora_propagate(pp, nb.ctypes.data_as(_ip), C.c_int(nb.size), C.c_int(kf.shape[0]), pd, C.c_double(path_now),
                        kf.ctypes.data_as(_dp))
    return kf


def loop(nbr, K, recent):
    nb = np.ascontiguousarray(nbr, np.int32)
    return bool(lib().ora_loop(nb.ctypes.data_as(_ip), C.c_int(nb.size), C.c_int(K), C.c_int(recent)))


def lse(logw, ll):
    logw, pl = _d(logw); ll, pll = _d(ll)
    P = logw.shape[0]
    lo = np.zeros(P); w = np.zeros(P)
    M = C.c_double(); lS = C.c_double(); am = C.c_int(); ess = C.c_double()
    lib().ora_lse(pl, pll, C.c_int(P), lo.ctypes.data_as(_dp), w.ctypes.data_as(_dp), C.byref(M), C.byref(lS),
                  C.byref(am), C.byref(ess))
    return {"logw": lo, "w": w, "M": M.value, "logS": lS.value, "argmax": am.value, "ess": ess.value}


def resample(w, u):
    w, pw = _d(w)
    P = w.shape[0]
    anc = np.zeros(P, np.int32)
    lib().ora_resample(pw, C.c_int(P), C.c_double(u), anc.ctypes.data_as(_ip))
    return anc


def prune(x, w, ll, argmax, prune_w=1e-8, ll_cut=float(np.log(1e-16)), u=0.5):
    """Dead-particle pruning (Sec. III-F): returns (anc, new log-weights, D)."""
    x, px = _d(x); w, pw = _d(w)
    pll = None
    if ll is not None:
        ll, pll = _d(ll)
    P = x.shape[0]
    anc = np.zeros(P, np.int32)
    lo = np.zeros(P)
    D = lib().ora_prune(px, pw, pll, C.c_int(P), C.c_int(argmax), C.c_double(prune_w), C.c_double(ll_cut),
                        C.c_double(u), anc.ctypes.data_as(_ip), lo.ctypes.data_as(_dp))
    return anc, lo, int(D)


def knn_cov(points, k=10, eps=1e-3):
    """Per-point covariances for GICP (Eq. 4's Sigma_j, Sigma'_j): the k nearest
    points of the same cloud (the point itself included) by squared distance
    formed in float32 as ((dx*dx + dy*dy) + dz*dz), each operation rounded,
    ties to the lower index; their FP64 covariance (1/k); then the plane
    regularisation of generalised ICP (Segal et al., RSS 2009): eigenvalues
    replaced by (eps, 1, 1) in ascending order. Returns (n, 6): xx xy xz yy yz zz."""
    P = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    n = P.shape[0]
    kk = min(k, n)
    out = np.zeros((n, 6))
    for i in range(n):
        d = P - P[i]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        nb = np.argsort(d2, kind="stable")[:kk]
        Q = P[nb].astype(np.float64)
        m = Q.sum(0) / kk
        D = Q - m
        Cv = D.T @ D / kk
        lam, V = np.linalg.eigh(Cv)
        S = V @ np.diag([eps, 1.0, 1.0]) @ V.T
        out[i] = [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]]
    return out


def gicp_voxel_map(points, covs, grid):
    """Dense GICP voxel map (the voxel-based correspondence of Sec. III-C1):
    voxel floor((p - origin) / h) in FP64; per non-empty voxel the mean of its
    points and the mean of their covariances. Returns (n2*n1*n0, 10):
    mean (3), count, covariance (6); x fastest."""
    P = np.asarray(points, np.float32).reshape(-1, 3).astype(np.float64)
    o = np.asarray(grid["origin"], np.float64)
    h = float(grid["h"])
    n = [int(v) for v in grid["dims"]]
    v = np.floor((P - o) / h).astype(np.int64)
    inside = np.all((v >= 0) & (v < np.array(n)), axis=1)
    rec = np.zeros((n[0] * n[1] * n[2], 10))
    for i in np.flatnonzero(inside):
        f = (v[i, 2] * n[1] + v[i, 1]) * n[0] + v[i, 0]
        rec[f, :3] += P[i]
        rec[f, 3] += 1.0
        rec[f, 4:] += covs[i]
    occ = rec[:, 3] > 0
    rec[occ, :3] /= rec[occ, 3:4]
    rec[occ, 4:] /= rec[occ, 3:4]
    return rec


def gicp_eval(T, kf_poses, maps, grids, scan, scov, tau=20.0, face_delta=1e-3, gate_delta=0.0):
    """ora_gicp_eval_particle: ll, b (6), H (6 x 6), slack (3), valid lookups."""
    n_nb = len(kf_poses)
    Tk = np.ascontiguousarray(np.asarray(kf_poses, np.float64).reshape(n_nb, 12))
    mps = [np.ascontiguousarray(m, np.float64) for m in maps]
    mp = (_dp * max(n_nb, 1))(*[m.ctypes.data_as(_dp) for m in mps])
    grs = (Grid * max(n_nb, 1))(*[make_grid(g) for g in grids])
    scan, ps = _f(scan)
    sc, psc = _d(np.asarray(scov).reshape(-1, 6))
    T, pT = _d(np.asarray(T).reshape(12))
    ll = C.c_double(); b = np.zeros(6); H = np.zeros(36); sl = np.zeros(3); nv = C.c_int()
    lib().ora_gicp_eval_particle(pT, C.c_int(n_nb), Tk.ctypes.data_as(_dp), mp, grs, ps, psc,
                                 C.c_int(scan.shape[0]), C.c_double(tau), C.c_double(face_delta),
                                 C.c_double(gate_delta), C.byref(ll),
                                 b.ctypes.data_as(_dp), H.ctypes.data_as(_dp), sl.ctypes.data_as(_dp), C.byref(nv))
    return {"ll": ll.value, "b": b, "H": H.reshape(6, 6), "slack": sl, "nvalid": nv.value}


def move_h(T, b, H, sigma=0.2, lambda_=1e-3, theta_max=np.deg2rad(2.0), t_max=0.1):
    """ora_move_h: (new pose, psi)."""
    T, pT = _d(np.asarray(T).reshape(12))
    b, pb = _d(b)
    H, pH = _d(np.asarray(H).reshape(36))
    mp = MoveParams(sigma, lambda_, theta_max, t_max, 0.0)
    out = np.zeros(12); psi = np.zeros(6)
    lib().ora_move_h(pT, pb, pH, C.byref(mp), out.ctypes.data_as(_dp), psi.ctypes.data_as(_dp))
    return out, psi


def occupancy_grid(pts, h):
    """ora_occupancy_grid: the overlap lattice of a cloud as a grid dict."""
    pts, pp = _f(np.asarray(pts).reshape(-1, 3))
    g = Grid()
    lib().ora_occupancy_grid(pp, C.c_int(pts.shape[0]), C.c_double(h), C.byref(g))
    return {"origin": np.array(list(g.origin)), "h": g.h, "dims": tuple(int(v) for v in g.n)}


def overlap(kf_pts, scan, T_rel, h=1.0):
    """ora_overlap: share of scan points, moved by T_rel, in occupied voxels of kf_pts."""
    kf, pk = _f(np.asarray(kf_pts).reshape(-1, 3))
    sc, ps = _f(np.asarray(scan).reshape(-1, 3))
    T, pT = _d(np.asarray(T_rel).reshape(12))
    g = make_grid(occupancy_grid(kf, h))
    lib().ora_overlap.restype = C.c_double
    return lib().ora_overlap(pk, C.c_int(kf.shape[0]), C.byref(g), ps, C.c_int(sc.shape[0]), pT)


class State:
    """Particle set held by the oracle in FP64: poses (P, 12), keyframe poses
    (K, P, 12), log-weights (P,), plus the shared keyframe tables."""

    def __init__(self, poses, kf_poses, tables, grids, logw=None, kf_path=None, path_now=0.0):
        self.kf_path = None if kf_path is None else np.ascontiguousarray(kf_path, np.float64)
        self.path_now = float(path_now)
        self.poses = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 12))
        self.kf_poses = np.ascontiguousarray(np.asarray(kf_poses, np.float64))
        P = self.poses.shape[0]
        self.logw = np.full(P, -np.log(P)) if logw is None else np.ascontiguousarray(logw, np.float64)
        self.tables = [np.ascontiguousarray(t, np.float64) for t in tables]
        self.grids = list(grids)

    def step(self, scan, dT, cov, frame, z=None, u=None, scov=None, **params):
        """One frame (ora_step). For the GICP model (model=1) the tables are voxel
        maps (gicp_voxel_map) and scov the scan's point covariances (knn_cov)."""
        prm = dict(DEFAULTS)
        prm.update(params)
        sp = StepParams(prm["sigma"], prm["eps"], prm["lambda_"], prm["theta_max"], prm["t_max"], prm["w_min"],
                        prm["face_delta"], prm["k_nb"], prm["steps"], prm["resample"], prm["propagate"],
                        prm["loop_recent"], prm["model"], prm["gicp_tau"], prm["prune_w"], prm["ll_cut"], prm["seed"])
        # odometry path length of this frame (Eq. 9 along the odometry trajectory)
        self.path_now += float(np.linalg.norm(np.asarray(dT, np.float64).reshape(12)[[3, 7, 11]]))
        kp = None if self.kf_path is None else self.kf_path.ctypes.data_as(_dp)
        P = self.poses.shape[0]
        K = len(self.tables)
        tab_ptrs = (_dp * max(K, 1))(*[t.ctypes.data_as(_dp) for t in self.tables])
        grs = (Grid * max(K, 1))(*[make_grid(g, t) for g, t in zip(self.grids, self.tables)])
        scan, ps = _f(scan)
        psc = None
        if scov is not None:
            scov, psc = _d(np.asarray(scov).reshape(-1, 6))
        dT, pd = _d(dT)
        cov, pc = _d(np.asarray(cov).reshape(36))
        zp = None
        if z is not None:
            z, zp = _d(z)
        up = None
        if u is not None:
            uu = C.c_double(u)
            up = C.byref(uu)
        out = StepOut()
        k_nb = min(prm["k_nb"], K)
        ll = np.zeros(P); w = np.zeros(P); anc = np.zeros(P, np.int32); nbr = np.zeros((P, max(k_nb, 1)), np.int32)
        lib().ora_step(C.c_int(P), C.c_int(K), self.poses.ctypes.data_as(_dp), self.kf_poses.ctypes.data_as(_dp),
                       self.logw.ctypes.data_as(_dp), tab_ptrs, grs, ps, psc, C.c_int(scan.shape[0]), pd, pc,
                       C.c_uint32(frame), zp, up, C.byref(sp), kp, C.c_double(self.path_now),
                       C.byref(out), ll.ctypes.data_as(_dp),
                       w.ctypes.data_as(_dp), anc.ctypes.data_as(_ip), nbr.ctypes.data_as(_ip))
        return {"estimate": np.array(list(out.estimate)), "ess": out.ess, "max_w": out.max_w,
                "argmax": out.argmax, "resampled": bool(out.resampled), "pruned": out.pruned, "ll": ll, "w": w, "anc": anc,
                "nbr": nbr[:, :k_nb]}
