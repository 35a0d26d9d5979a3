"""Pins of the oracle's GICP likelihood (Eq. 2-6): per-point covariances from
k nearest neighbours with the plane regularisation, the voxel map, and the
distribution-to-distribution terms checked against closed forms -- identity
covariances reduce it to point-to-point ICP, one Gauss-Newton step recovers a
pure translation exactly, and b is half the derivative of the log-likelihood
where Omega does not depend on the pose. CPU only."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
import synth

EPS = 1e-3


@pytest.fixture(scope="module")
def small_forest():
    return synth.forest_workload(seed=0, n_particles=16, n_points=256, n_keyframes=4, kf_points=2048, n_frames=2)


def _h44(T):
    M = np.eye(4)
    M[:3] = np.asarray(T, np.float64).reshape(3, 4)
    return M


def _orthonormal(T):
    T = np.asarray(T, np.float64).reshape(3, 4).copy()
    U, _, Vt = np.linalg.svd(T[:, :3])
    T[:, :3] = U @ Vt
    return T.reshape(12)


def _sym(v):
    return np.array([[v[0], v[1], v[2]], [v[1], v[3], v[4]], [v[2], v[4], v[5]]])


def test_plane_points_get_the_plane_normal():
    rng = np.random.default_rng(0)
    xy = rng.uniform(-1, 1, (300, 2))
    z = 0.3 * xy[:, 0] - 0.1 * xy[:, 1] + 0.5
    pts = np.c_[xy, z].astype(np.float32)
    S = oracle.knn_cov(pts, k=10, eps=EPS)
    n = np.array([-0.3, 0.1, 1.0])
    n /= np.linalg.norm(n)
    expect = np.eye(3) - (1 - EPS) * np.outer(n, n)
    for i in range(0, 300, 7):
        np.testing.assert_allclose(_sym(S[i]), expect, atol=2e-5)   # float32 inputs: plane to ~1e-7


def test_neighbours_agree_with_a_kd_tree():
    """The regularised covariance's normal equals the smallest-eigenvalue
    direction of the neighbourhood a k-d tree (scipy) returns, and its
    eigenvalues are (eps, 1, 1)."""
    rng = np.random.default_rng(1)
    pts = rng.normal(0, 1, (400, 3)).astype(np.float32) * np.array([3.0, 2.0, 0.5], np.float32)
    S = oracle.knn_cov(pts, k=10, eps=EPS)
    tree = cKDTree(pts.astype(np.float64))
    _, nb = tree.query(pts.astype(np.float64), k=10)
    for i in range(400):
        lam_s, V_s = np.linalg.eigh(_sym(S[i]))
        np.testing.assert_allclose(lam_s, [EPS, 1, 1], atol=1e-12)
        Q = pts[nb[i]].astype(np.float64)
        lam, V = np.linalg.eigh(np.cov(Q.T, bias=True))
        if lam[1] - lam[0] < 1e-6 * lam[2]:
            continue                                   # normal undefined
        assert abs(abs(V[:, 0] @ V_s[:, 0]) - 1) < 1e-9, i


def test_neighbour_ties_go_to_the_lower_index():
    g = np.stack(np.meshgrid(np.arange(6), np.arange(6), np.arange(2), indexing="ij"), -1).reshape(-1, 3)
    pts = g.astype(np.float32)
    S = oracle.knn_cov(pts, k=7, eps=EPS)
    for i in [0, 13, 40, 71]:
        d2 = ((g - g[i]) ** 2).sum(1)
        nb = sorted(range(len(g)), key=lambda j: (d2[j], j))[:7]
        Q = g[nb].astype(np.float64)
        lam, V = np.linalg.eigh(np.cov(Q.T, bias=True))
        if lam[1] - lam[0] < 1e-9:
            continue
        n = V[:, 0]
        np.testing.assert_allclose(_sym(S[i]), np.eye(3) - (1 - EPS) * np.outer(n, n), atol=1e-12)


def test_voxel_map_matches_grouping():
    rng = np.random.default_rng(2)
    pts = rng.uniform(-3, 3, (500, 3)).astype(np.float32)
    covs = rng.normal(0, 1, (500, 6))
    grid = {"origin": np.array([-2.0, -2.5, -3.0]), "h": 0.7, "dims": (6, 7, 9)}
    rec = oracle.gicp_voxel_map(pts, covs, grid)
    groups = {}
    for i, p in enumerate(pts.astype(np.float64)):
        v = tuple(int(np.floor((p[a] - grid["origin"][a]) / grid["h"])) for a in range(3))
        if all(0 <= v[a] < grid["dims"][a] for a in range(3)):
            groups.setdefault(v, []).append(i)
    assert rec[:, 3].sum() == sum(len(m) for m in groups.values())
    for v, members in groups.items():
        f = (v[2] * 7 + v[1]) * 6 + v[0]
        assert rec[f, 3] == len(members)
        np.testing.assert_allclose(rec[f, :3], pts[members].astype(np.float64).mean(0), rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(rec[f, 4:], covs[members].mean(0), rtol=1e-13, atol=1e-14)
    assert np.all(rec[rec[:, 3] == 0] == 0)


def _kf_map(kf, h=1.0, k=10):
    grid = synth.grid_for_points(kf["points"], h, 1.0)
    covs = oracle.knn_cov(kf["points"], k=k, eps=EPS)
    return oracle.gicp_voxel_map(kf["points"], covs, grid), grid


def test_identity_covariances_reduce_to_point_to_point(small_forest):
    """Sigma' = Sigma_j = I/2 gives Omega = I: l = -sum min(|e|^2, tau) over
    all lookups (tau where there is no distribution) and H = sum B^T B over the
    inliers, B = [-[mu]x | I] (the field path's explicit matrix with unit
    weights)."""
    w = small_forest
    kf = w["keyframes"][0]
    rec, grid = _kf_map(kf)
    rec[:, 4:] = np.where(rec[:, 3:4] > 0, [0.5, 0, 0, 0.5, 0, 0.5], 0)
    scan = w["scans"][0]
    scov = np.tile([0.5, 0, 0, 0.5, 0, 0.5], (scan.shape[0], 1))
    Tt = _orthonormal(w["particles"][3])                 # R R^T = I to rounding, so Omega = I
    Tk = _orthonormal(w["kf_particle_poses"][0][3])
    o = oracle.gicp_eval(Tt, [Tk], [rec], [grid], scan, scov)
    Rk, tk = Tk.reshape(3, 4)[:, :3], Tk.reshape(3, 4)[:, 3]
    inv = np.eye(4)
    inv[:3, :3], inv[:3, 3] = Rk.T, -Rk.T @ tk           # rigid inverse (the float32 R is not exactly orthonormal)
    rel = (inv @ _h44(Tt))[:3]
    x = scan.astype(np.float64) @ rel[:, :3].T + rel[:, 3]
    v = np.floor((x - grid["origin"]) / grid["h"]).astype(int)
    dims = np.array(grid["dims"])
    inside = np.all((v >= 0) & (v < dims), 1)
    f = (v[:, 2] * dims[1] + v[:, 1]) * dims[0] + v[:, 0]
    tau = 20.0
    d2 = np.full(len(x), np.inf)
    has = inside.copy()
    has[inside] = rec[f[inside], 3] > 0
    e = rec[f[has], :3] - x[has]
    d2[has] = (e * e).sum(1)
    ok = d2 < tau
    assert o["nvalid"] == ok.sum() > 50 and (~ok).sum() > 0
    np.testing.assert_allclose(o["ll"], -(d2[ok].sum() + tau * (~ok).sum()), rtol=1e-12)
    H_icp = oracle.h_explicit(scan[ok], np.ones(ok.sum()), 1.0)
    np.testing.assert_allclose(o["H"], H_icp, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(o["H"], o["H"].T, rtol=0, atol=1e-9)


def test_one_step_recovers_a_translation_exactly():
    """Scan points at voxel means, particle displaced by a pure translation that
    keeps every point in its voxel: e = -delta for every correspondence, so the
    undamped Gauss-Newton step psi = H^-1 b is [0, -delta] for any Omega."""
    rng = np.random.default_rng(3)
    h = 1.0
    cells = rng.choice(8 * 8 * 4, 60, replace=False)
    c = np.stack([cells % 8, (cells // 8) % 8, cells // 64], 1)
    mu = (c + 0.5 + rng.uniform(-0.2, 0.2, (60, 3))).astype(np.float32)
    grid = {"origin": np.zeros(3), "h": h, "dims": (8, 8, 4)}
    covs = oracle.knn_cov(mu, k=6, eps=EPS)
    rec = oracle.gicp_voxel_map(mu, covs, grid)
    scov = oracle.knn_cov(mu, k=5, eps=EPS)
    delta = np.array([0.04, -0.03, 0.05])
    Tt = np.eye(3, 4).reshape(12).copy()
    Tt[[3, 7, 11]] = delta
    o = oracle.gicp_eval(Tt, [np.eye(3, 4).reshape(12)], [rec], [grid], mu, scov)
    assert o["nvalid"] == 60
    T1, psi = oracle.move_h(Tt, o["b"], o["H"], lambda_=0.0, theta_max=10.0, t_max=10.0)
    np.testing.assert_allclose(psi, [0, 0, 0, -0.04, 0.03, -0.05], atol=1e-12)
    np.testing.assert_allclose(T1, np.eye(3, 4).reshape(12), atol=1e-12)


def _fd(T, kfs, maps, grids, scan, scov, d, step):
    e = np.zeros(6)
    e[d] = step
    out = []
    for sgn in (1, -1):
        Tp = (_h44(T) @ _h44(oracle.se3_exp(sgn * e)))[:3].reshape(12)
        out.append(oracle.gicp_eval(Tp, kfs, maps, grids, scan, scov, tau=1e3)["ll"])
    return (out[0] - out[1]) / (2 * step)


@pytest.mark.parametrize("isotropic", [True, False])
def test_b_is_half_the_log_likelihood_gradient(small_forest, isotropic):
    """dl/dxi = 2 b wherever Omega does not move with the pose: every direction
    with isotropic covariances, the translation directions always (Omega
    depends on the rotation only). Central differences at step 1e-6 from a pose
    whose lookups are all more than 1e-3 voxel from a face, with the cap high
    enough (1e3) that every lookup with a distribution is an inlier."""
    w = small_forest
    maps, grids = [], []
    for kf in w["keyframes"][:2]:
        rec, grid = _kf_map(kf)
        if isotropic:
            rec[:, 4:] = np.where(rec[:, 3:4] > 0, [0.3, 0, 0, 0.3, 0, 0.3], 0)
        maps.append(rec)
        grids.append(grid)
    scan = w["scans"][0][:128]
    scov = np.tile([0.2, 0, 0, 0.2, 0, 0.2], (128, 1)) if isotropic else oracle.knn_cov(scan, k=10, eps=EPS)
    checked = 0
    for i in range(16):
        Tt = w["particles"][i].astype(np.float64)
        kfs = [w["kf_particle_poses"][k][i].astype(np.float64) for k in range(2)]
        o = oracle.gicp_eval(Tt, kfs, maps, grids, scan, scov, tau=1e3, face_delta=1e-3)
        if np.any(o["slack"] > 0) or o["nvalid"] < 20:
            continue
        dirs = range(6) if isotropic else range(3, 6)
        for d in dirs:
            fd = _fd(Tt, kfs, maps, grids, scan, scov, d, 1e-6)
            assert abs(fd - 2 * o["b"][d]) <= 1e-5 * max(abs(fd), 1.0) + 1e-6 * np.abs(o["H"]).max(), (i, d, fd, o["b"][d])
        checked += 1
    assert checked >= 3


def test_gicp_frame_tracks_truth(small_forest):
    w = small_forest
    maps, grids = [], []
    for kf in w["keyframes"]:
        rec, grid = _kf_map(kf)
        maps.append(rec)
        grids.append(grid)
    st = oracle.State(w["particles"], np.stack(w["kf_particle_poses"]), maps, grids)
    for fr in range(2):
        scov = oracle.knn_cov(w["scans"][fr], k=10, eps=EPS)
        o = st.step(w["scans"][fr], w["odometry"][fr], w["cov"], frame=fr, scov=scov, model=1)
        assert abs(o["w"].sum() - 1) < 1e-12 and np.all(o["ll"] <= 0)
        err = np.linalg.norm(o["estimate"][[3, 7, 11]] - w["truth"][fr + 1][[3, 7, 11]])
        assert err < 0.3, (fr, err)


def _rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w_, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w_), 2 * (x * z + y * w_)],
                     [2 * (x * y + z * w_), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w_)],
                     [2 * (x * z - y * w_), 2 * (y * z + x * w_), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("along", [True, False])
def test_aligned_planes_closed_form(along):
    """One voxel holding a plane with normal n (Sigma' = I - (1-eps) n n^T) and a
    scan point whose plane normal m maps onto n under the relative rotation
    (R m = n): C = 2 (I - (1-eps) n n^T), so an error alpha n costs
    alpha^2 / (2 eps) and an error beta t (t perpendicular to n) costs beta^2 / 2."""
    rng = np.random.default_rng(11)
    R = _rot(rng)
    n = np.array([0.2, -0.5, 0.84])
    n /= np.linalg.norm(n)
    m = R.T @ n
    tang = np.cross(n, [1.0, 0, 0])
    tang /= np.linalg.norm(tang)
    Sv = np.eye(3) - (1 - EPS) * np.outer(n, n)
    Sm = np.eye(3) - (1 - EPS) * np.outer(m, m)
    grid = {"origin": np.zeros(3), "h": 1.0, "dims": (1, 1, 1)}
    mu_v = np.array([0.5, 0.5, 0.5])
    rec = np.zeros((1, 10))
    rec[0, :3] = mu_v
    rec[0, 3] = 1
    rec[0, 4:] = [Sv[0, 0], Sv[0, 1], Sv[0, 2], Sv[1, 1], Sv[1, 2], Sv[2, 2]]
    mu = np.array([0.25, -0.5, 1.0], np.float32)
    err = 0.005 * n if along else 0.3 * tang
    t = mu_v - err - R @ mu.astype(np.float64)           # so that e = mu' - (R mu + t) = err
    T = np.c_[R, t].reshape(12)
    scov = np.array([[Sm[0, 0], Sm[0, 1], Sm[0, 2], Sm[1, 1], Sm[1, 2], Sm[2, 2]]])
    o = oracle.gicp_eval(T, [np.eye(3, 4).reshape(12)], [rec], [grid], mu[None], scov)
    expect = 0.005 ** 2 / (2 * EPS) if along else 0.3 ** 2 / 2
    assert o["nvalid"] == 1
    np.testing.assert_allclose(-o["ll"], expect, rtol=1e-9)


def test_translation_block_is_half_the_hessian(small_forest):
    """Within fixed voxels l is quadratic in the translation and Omega does not
    depend on it, so H_vv = -1/2 d2 l / dv2 (second differences, step 1e-4)."""
    w = small_forest
    rec, grid = _kf_map(w["keyframes"][1])
    scan = w["scans"][1][:128]
    scov = oracle.knn_cov(scan, k=10, eps=EPS)
    for i in range(16):
        Tt = w["particles"][i].astype(np.float64)
        kfs = [w["kf_particle_poses"][1][i].astype(np.float64)]
        o = oracle.gicp_eval(Tt, kfs, [rec], [grid], scan, scov, tau=1e3, face_delta=1e-2)
        if np.any(o["slack"] > 0) or o["nvalid"] < 20:
            continue
        h = 1e-4
        Hn = np.zeros((3, 3))
        def ll(dv):
            xi = np.r_[0, 0, 0, dv]
            Tp = (_h44(Tt) @ _h44(oracle.se3_exp(xi)))[:3].reshape(12)
            return oracle.gicp_eval(Tp, kfs, [rec], [grid], scan, scov, tau=1e3)["ll"]
        for a in range(3):
            for b in range(3):
                ea, eb = np.eye(3)[a] * h, np.eye(3)[b] * h
                Hn[a, b] = -(ll(ea + eb) - ll(ea - eb) - ll(-ea + eb) + ll(-ea - eb)) / (4 * h * h) / 2
        np.testing.assert_allclose(o["H"][3:, 3:], Hn, rtol=1e-5, atol=1e-6 * np.abs(Hn).max())
        return
    pytest.fail("no particle away from voxel faces")
