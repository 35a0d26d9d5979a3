"""Pins of the FP64 oracle against things other than itself: published test
vectors, library routines (scipy expm / map_coordinates / rotation vectors,
numpy half conversion, torch bfloat16), closed forms, brute force and
invariants. CPU only."""
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.ndimage
from scipy.spatial.transform import Rotation

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def twist(xi):
    """4x4 twist matrix of xi = [omega; v]."""
    w, v = xi[:3], xi[3:]
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    X[:3, 3] = v
    return X


def expm_pose(xi):
    return scipy.linalg.expm(twist(np.asarray(xi, np.float64)))[:3, :].reshape(12)


def to44(T):
    M = np.eye(4)
    M[:3, :] = np.asarray(T).reshape(3, 4)
    return M


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_normal_draws_are_standard():
    z = np.array([oracle.normal6(7, i, 3) for i in range(20000)]).reshape(-1)
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.02
    # independent across particles and frames
    assert not np.allclose(oracle.normal6(7, 0, 3), oracle.normal6(7, 1, 3))
    assert not np.allclose(oracle.normal6(7, 0, 3), oracle.normal6(7, 0, 4))
    u = [oracle.systematic_u(5, t) for t in range(2000)]
    assert min(u) >= 0.0 and max(u) < 1.0 and abs(np.mean(u) - 0.5) < 0.03


# ----------------------------------------------------------------- SE(3)
@pytest.mark.parametrize("scale", [0.0, 1e-7, 1e-5, 9.9e-5, 1.01e-4, 1e-3, 0.3, 2.5])
def test_se3_exp_matches_matrix_exponential(scale):
    rng = np.random.default_rng(int(scale * 1e7) + 1)
    for _ in range(5):
        w = rng.normal(size=3)
        w = w / np.linalg.norm(w) * scale
        xi = np.concatenate([w, rng.normal(size=3)])
        np.testing.assert_allclose(oracle.se3_exp(xi), expm_pose(xi), atol=1e-14, rtol=0)


def test_se3_exp_rotation_matches_scipy_and_log_roundtrip():
    rng = np.random.default_rng(3)
    for _ in range(20):
        xi = rng.normal(size=6) * [0.7, 0.7, 0.7, 3, 3, 3]
        T = oracle.se3_exp(xi)
        R = T.reshape(3, 4)[:, :3]
        np.testing.assert_allclose(R, Rotation.from_rotvec(xi[:3]).as_matrix(), atol=1e-14)
        np.testing.assert_allclose(oracle.se3_log(T), xi, atol=1e-12)
        I = oracle.pose_mul(T, oracle.se3_exp(-xi))
        np.testing.assert_allclose(I, np.eye(4)[:3].reshape(12), atol=1e-14)
    np.testing.assert_array_equal(oracle.se3_exp(np.zeros(6)), np.eye(4)[:3].reshape(12))


def test_pose_mul_inv():
    rng = np.random.default_rng(4)
    A = expm_pose(rng.normal(size=6))
    B = expm_pose(rng.normal(size=6))
    np.testing.assert_allclose(to44(oracle.pose_mul(A, B)), to44(A) @ to44(B), atol=1e-14)
    np.testing.assert_allclose(to44(oracle.pose_inv(A)), np.linalg.inv(to44(A)), atol=1e-13)


# ----------------------------------------------------------------- tables
def test_table_splat_equals_brute_force():
    rng = np.random.default_rng(5)
    pts = (rng.normal(size=(60, 3)) * [1.0, 0.8, 0.5]).astype(np.float32)
    grid = synth.grid_for_points(pts, 0.2, 1.0)
    a = oracle.build_table(pts, grid, 0.2, 1.0)
    b = oracle.build_table(pts, grid, 0.2, 1.0, brute=True)
    assert a.shape == tuple(reversed(grid["dims"]))
    np.testing.assert_array_equal(a, b)
    # the margin makes every boundary vertex farther than r_t from all points
    assert a[0].max() == 0 and a[-1].max() == 0 and a[:, 0].max() == 0 and a[:, :, -1].max() == 0


def test_table_closed_form_single_point():
    grid = {"origin": np.array([-1.0, -1.0, -1.0]), "h": 0.25, "dims": (9, 9, 9)}
    p = np.array([[0.0, 0.0, 0.1]], np.float32)
    t = oracle.build_table(p, grid, 0.2, 1.0)
    for (ix, iy, iz) in [(4, 4, 4), (5, 4, 4), (4, 6, 3), (8, 8, 8), (0, 4, 4)]:
        x = np.array([-1 + 0.25 * ix, -1 + 0.25 * iy, -1 + 0.25 * iz])
        d2 = float(((x - p[0].astype(np.float64)) ** 2).sum())
        exp = np.exp(-d2 / (2 * 0.04)) if d2 <= 1.0 else 0.0
        assert t[iz, iy, ix] == pytest.approx(exp, rel=1e-15, abs=0)


def test_quantize_matches_library_conversions():
    import torch
    rng = np.random.default_rng(6)
    v32 = np.concatenate([rng.random(5000), np.exp(-rng.uniform(0, 12.5, 5000)), [0.0, 1.0]]).astype(np.float32)
    v = v32.astype(np.float64)
    np.testing.assert_array_equal(oracle.quantize(v, 2), v32.astype(np.float16).astype(np.float64))
    bf = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.quantize(v, 1), bf)
    # double inputs straight to half, rounded once
    vd = rng.random(5000) * 1e-3
    np.testing.assert_array_equal(oracle.quantize(vd, 2), vd.astype(np.float16).astype(np.float64))


def test_coef_table_is_the_trilinear_interpolation():
    """A coefficient table evaluates to the same function as the vertex table it
    came from (the trilinear polynomial, every cell, inside and on its faces), and
    c0 is the cell's lower corner: a swapped or transposed coefficient fails."""
    grid = {"origin": np.array([0.5, -1.0, 2.0]), "h": 0.5, "dims": (6, 5, 4)}
    rng = np.random.default_rng(12)
    vals = rng.random((4, 5, 6))
    coef = oracle.coef_table(vals)
    assert coef.shape == (3, 4, 5, 8)
    np.testing.assert_array_equal(coef[..., 0], vals[:-1, :-1, :-1])
    for _ in range(200):
        c = [rng.integers(0, 5), rng.integers(0, 4), rng.integers(0, 3)]
        u = np.array(c, np.float64) + rng.random(3) * rng.choice([1.0, 0.0, 0.999999], 3)
        ok_v, Lv, dv = oracle.cell_eval(vals, grid, c, u)
        ok_c, Lc, dc = oracle.cell_eval(coef, grid, c, u)
        assert ok_v and ok_c
        assert Lc == pytest.approx(Lv, abs=1e-14)
        np.testing.assert_allclose(dc, dv, atol=1e-14)
    ok, L, d = oracle.cell_eval(coef, grid, [5, 0, 0], [5.2, 0.1, 0.1])
    assert not ok and L == 0.0 and not d.any()


def test_record_quantisation_fp16_and_bf16():
    """16-bit coefficient records. FP16: each coefficient rounded to nearest (numpy's
    conversion). BF16: the low-half coefficients equal torch's bfloat16 rounding; each
    high-half coefficient is, of all FP32 numbers whose low 16 bits are its partner's
    bfloat16 bits, the one nearest to it (checked against an exhaustive search of
    the 65,536 candidates), hence within half a bfloat16 spacing."""
    import torch
    rng = np.random.default_rng(13)
    c = np.concatenate([rng.normal(0, 0.3, (400, 8)), np.exp(-rng.uniform(0, 20, (400, 8))) * rng.choice([-1, 1], (400, 8)),
                        np.zeros((4, 8)), np.eye(8)[:4]])
    c32 = c.astype(np.float32)
    q16 = oracle.quantize_coef(c, 2)
    np.testing.assert_array_equal(q16, c32.astype(np.float16).astype(np.float64))
    qb = oracle.quantize_coef(c, 1)
    hi, lo = [4, 2, 7, 6], [1, 0, 5, 3]
    bf = torch.from_numpy(np.ascontiguousarray(c32[:, lo])).to(torch.bfloat16)
    np.testing.assert_array_equal(qb[:, lo], bf.to(torch.float64).numpy())
    lo_bits = bf.view(torch.int16).numpy().astype(np.uint16).astype(np.uint32)
    highs = np.arange(1 << 16, dtype=np.uint32) << np.uint32(16)
    for r in range(0, c.shape[0], 7):
        for e in range(4):
            with np.errstate(invalid="ignore"):
                cand = (highs | lo_bits[r, e]).view(np.float32).astype(np.float64)
            A = float(c32[r, hi[e]])
            err = np.abs(np.where(np.isfinite(cand), cand, np.inf) - A)
            assert abs(qb[r, hi[e]] - A) == err.min()
            if A != 0.0:
                assert abs(qb[r, hi[e]] - A) <= 2.0 ** -8 * abs(A)


def test_stored_tables_keep_the_field_within_storage_precision(box_room_tables):
    t = box_room_tables[0]
    assert oracle.stored_table(t, 0) is not None and np.array_equal(oracle.stored_table(t, 0), t)
    exact = oracle.coef_table(t)
    for dt, u in ((1, 2.0 ** -8), (2, 2.0 ** -11)):
        q = oracle.stored_table(t, dt)
        assert q.shape == exact.shape
        assert np.all(np.abs(q - exact) <= u * np.abs(exact) + 1e-7)


# ----------------------------------------------------------------- lookup
def test_cell_eval_vertices_constant_and_affine():
    grid = {"origin": np.zeros(3), "h": 0.5, "dims": (6, 5, 4)}
    rng = np.random.default_rng(8)
    vals = rng.random((4, 5, 6))
    for _ in range(30):
        c = [rng.integers(0, 5), rng.integers(0, 4), rng.integers(0, 3)]
        ok, L, d = oracle.cell_eval(vals, grid, c, np.array(c, np.float64))
        assert ok and L == vals[c[2], c[1], c[0]]
    ok, L, d = oracle.cell_eval(np.full((4, 5, 6), 0.7), grid, [1, 2, 1], [1.3, 2.9, 1.5])
    assert L == pytest.approx(0.7, abs=1e-15) and np.abs(d).max() < 1e-15
    a = np.array([0.3, -0.2, 0.05])
    iz, iy, ix = np.meshgrid(np.arange(4), np.arange(5), np.arange(6), indexing="ij")
    aff = a[0] * ix + a[1] * iy + a[2] * iz + 0.4
    for _ in range(30):
        u = rng.random(3) * [4.99, 3.99, 2.99]
        c = np.floor(u).astype(int)
        ok, L, d = oracle.cell_eval(aff, grid, c, u)
        assert L == pytest.approx(a @ u + 0.4, abs=1e-14)
        np.testing.assert_allclose(d, a, atol=1e-14)
    ok, L, d = oracle.cell_eval(aff, grid, [5, 0, 0], [5.1, 0.0, 0.0])
    assert not ok and L == 0.0


def _particle_case(box_room, box_room_tables, i=3, seed=11):
    rng = np.random.default_rng(seed)
    kfs = box_room["keyframes"]
    Tt = synth.perturb_poses(box_room["truth"][1], 1, 0.05, np.deg2rad(1.0), rng)[0]
    nb = [0, 1, 2]
    Tk = np.stack([kfs[k]["pose"] for k in nb])
    return Tt, Tk, [box_room_tables[k] for k in nb], [kfs[k]["grid"] for k in nb], box_room["scans"][0]


def test_loglik_matches_scipy_trilinear(box_room, box_room_tables):
    Tt, Tk, tabs, grids, scan = _particle_case(box_room, box_room_tables)
    o = oracle.eval_particle(Tt, Tk, tabs, grids, scan)
    ll = 0.0
    mom = np.zeros(10)
    p = scan.astype(np.float64)
    for s in range(3):
        rel = np.linalg.inv(to44(Tk[s])) @ to44(Tt)
        x = p @ rel[:3, :3].T + rel[:3, 3]
        u = (x - grids[s]["origin"]) / grids[s]["h"]
        L = scipy.ndimage.map_coordinates(tabs[s], [u[:, 2], u[:, 1], u[:, 0]], order=1, mode="constant", cval=0.0)
        ll += np.log(L + 1e-3).sum()
        w = L / (L + 1e-3)
        mom += np.concatenate([[w.sum()], (w[:, None] * p).sum(0),
                               [(w * p[:, a] * p[:, b]).sum() for a, b in [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]]])
    assert o["ll"] == pytest.approx(ll, rel=1e-12)
    np.testing.assert_allclose(o["mom"], mom, rtol=1e-11, atol=1e-9)


def test_gradient_matches_frozen_cell_central_differences(box_room, box_room_tables):
    """FD in the Lie algebra with step 1e-5, each lookup kept in the cell it uses
    at the base pose. The central difference at 1e-5 carries an O(step^2)
    truncation term from the curvature of log(L + eps); extrapolating it with
    the 2e-5 difference (Richardson) removes that term, and the result must be
    within 1e-6 relative of the analytic gradient."""
    Tt, Tk, tabs, grids, scan = _particle_case(box_room, box_room_tables)
    base = oracle.eval_particle(Tt, Tk, tabs, grids, scan, want_cells=True)
    cells = base["cells"]

    def central(step):
        fd = np.zeros(6)
        for d in range(6):
            e = np.zeros(6)
            e[d] = step
            Tp = (to44(Tt) @ to44(expm_pose(e)))[:3].reshape(12)
            Tm = (to44(Tt) @ to44(expm_pose(-e)))[:3].reshape(12)
            lp = oracle.eval_particle(Tp, Tk, tabs, grids, scan, cells=cells.copy(), frozen=True)["ll"]
            lm = oracle.eval_particle(Tm, Tk, tabs, grids, scan, cells=cells.copy(), frozen=True)["ll"]
            fd[d] = (lp - lm) / (2 * step)
        return fd

    g = base["g"]
    assert np.linalg.norm(g) > 1.0
    f1, f2 = central(1e-5), central(2e-5)
    rich = (4 * f1 - f2) / 3
    assert np.linalg.norm(rich - g) / np.linalg.norm(g) <= 1e-6
    for d in range(6):
        assert abs(rich[d] - g[d]) <= 1e-6 * np.abs(g).max()
    # the plain central difference converges to it at second order
    e1 = np.linalg.norm(f1 - g)
    e2 = np.linalg.norm(f2 - g)
    assert e1 / np.linalg.norm(g) <= 1e-5
    assert 3.0 < e2 / e1 < 5.0


def test_h_from_moments_matches_explicit_sum():
    rng = np.random.default_rng(12)
    p = (rng.normal(size=(300, 3)) * [5, 5, 1]).astype(np.float32)
    w = rng.random(300)
    pd = p.astype(np.float64)
    mom = np.concatenate([[w.sum()], (w[:, None] * pd).sum(0),
                          [(w * pd[:, a] * pd[:, b]).sum() for a, b in [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]]])
    H_ref = np.zeros((6, 6))
    for j in range(300):
        B = np.hstack([-twist(np.concatenate([pd[j], np.zeros(3)]))[:3, :3], np.eye(3)])
        H_ref += w[j] * B.T @ B / 0.04
    np.testing.assert_allclose(oracle.h_from_moments(mom, 0.2), H_ref, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(oracle.h_explicit(p, w, 0.2), H_ref, rtol=1e-12, atol=1e-9)


# ----------------------------------------------------------------- lattice-plane cases
def _plane_case(z_plane):
    h = 0.25
    grid = {"origin": np.array([-5.0, -5.0, -2.0]), "h": h, "dims": (41, 41, 17)}
    xs = np.arange(-4.0, 4.0 + 1e-9, h)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z_plane)], 1).astype(np.float32)
    tab = oracle.build_table(pts, grid, 0.2, 1.0)
    g1 = np.arange(-1.5, 1.5 + 1e-9, 0.5)
    SX, SY = np.meshgrid(g1, g1, indexing="ij")
    scan = np.stack([SX.ravel(), SY.ravel(), np.full(SX.size, z_plane)], 1).astype(np.float32)
    return grid, tab, scan


def test_zero_gradient_at_true_pose_on_midplane_scene():
    """Noise-free scan of a plane lying on a cell mid-plane, sampled on the
    lattice columns: the field is symmetric about the plane and constant along
    it, so the gradient at the true pose vanishes."""
    grid, tab, scan = _plane_case(0.125)
    I = np.eye(4)[:3].reshape(12)
    o = oracle.eval_particle(I, I[None], [tab], [grid], scan)
    assert np.abs(o["g"]).max() < 1e-12
    # a particle displaced past the flat central cell sees a restoring gradient
    # (within one cell of the mid-plane the two bracketing vertex layers are equal)
    o2 = oracle.eval_particle(expm_pose([0, 0, 0, 0.3, 0, 0.2]), I[None], [tab], [grid], scan)
    assert o2["g"][5] < -1.0


def test_one_move_closed_form_on_vertex_plane():
    """Plane through a vertex layer, particle displaced by dz along the normal:
    trilinear field L = (1-f) + f v1 with f = dz/h, v1 = exp(-h^2/2 sigma^2);
    one damped Gauss-Newton step is psi_z = sigma^2 (v1-1) / (h L (1+lambda))."""
    grid, tab, scan = _plane_case(0.0)
    h, sigma, lam, eps = 0.25, 0.2, 1e-3, 1e-3
    I = np.eye(4)[:3].reshape(12)
    for dz in [0.01, 0.05, 0.12]:
        Tt = I.copy()
        Tt[11] = dz
        o = oracle.eval_particle(Tt, I[None], [tab], [grid], scan, eps=eps)
        v1 = np.exp(-h * h / (2 * sigma * sigma))
        f = dz / h
        L = (1 - f) + f * v1
        N = scan.shape[0]
        assert o["ll"] == pytest.approx(N * np.log(L + eps), rel=1e-13)
        np.testing.assert_allclose(o["g"], [0, 0, 0, 0, 0, N * (v1 - 1) / h / (L + eps)], atol=1e-9)
        Tout, psi = oracle.move(Tt, o["g"], o["mom"], sigma=sigma, lambda_=lam)
        pz = sigma ** 2 * (v1 - 1) / (h * L * (1 + lam))
        pz = max(pz, -0.1)       # translation step clamped at t_max = 0.1 m
        np.testing.assert_allclose(psi, [0, 0, 0, 0, 0, pz], atol=1e-12)
        exp = I.copy()
        exp[11] = dz + pz
        np.testing.assert_allclose(Tout, exp, atol=1e-12)


def test_move_clamps_and_skips_without_contact():
    g = np.array([50.0, -20, 5, 400, 0, 0])
    mom = np.array([10.0, 0, 0, 0, 100, 0, 0, 100, 0, 1])
    Tout, psi = oracle.move(np.eye(4)[:3].reshape(12), g, mom)
    assert np.linalg.norm(psi[3:]) == pytest.approx(0.1, rel=1e-12)
    assert np.linalg.norm(psi[:3]) <= np.deg2rad(2.0) * (1 + 1e-12)
    Tout, psi = oracle.move(np.eye(4)[:3].reshape(12), g, np.zeros(10))
    assert np.all(psi == 0)


# ----------------------------------------------------------------- prediction, neighbours
def test_predict_matches_matrix_exponential():
    rng = np.random.default_rng(13)
    T = expm_pose(rng.normal(size=6))
    dT = expm_pose(rng.normal(size=6) * 0.1)
    A = rng.normal(size=(6, 6))
    cov = A @ A.T * 1e-3 + np.eye(6) * 1e-4
    z = rng.normal(size=6)
    Lc = np.linalg.cholesky(cov)
    exp = (to44(T) @ to44(dT) @ to44(expm_pose(Lc @ z)))[:3].reshape(12)
    np.testing.assert_allclose(oracle.predict(T, dT, cov, z), exp, atol=1e-13)
    # zero covariance: deterministic composition
    np.testing.assert_allclose(oracle.predict(T, dT, np.zeros((6, 6)), z), (to44(T) @ to44(dT))[:3].reshape(12),
                               atol=1e-14)


def test_predict_noise_covariance():
    cov = np.diag([1e-4, 2e-4, 3e-4, 1e-3, 2e-3, 4e-3])
    cov[3, 4] = cov[4, 3] = 5e-4
    I = np.eye(4)[:3].reshape(12)
    d = np.array([oracle.se3_log(oracle.predict(I, I, cov, oracle.normal6(1, i, 0))) for i in range(20000)])
    np.testing.assert_allclose(np.cov(d.T), cov, atol=8e-5 * np.sqrt(np.outer(np.diag(cov), np.diag(cov))).max() / 1e-3)


def test_select_nbrs_brute_force():
    rng = np.random.default_rng(14)
    for K in [1, 2, 3, 5, 20]:
        kt = rng.normal(size=(K, 3)) * 5
        if K >= 5:
            kt[3] = kt[1]          # exact tie: lower index first
        T = np.eye(4)[:3].reshape(12).copy()
        T[[3, 7, 11]] = rng.normal(size=3)
        t32 = T[[3, 7, 11]].astype(np.float32)
        k32 = kt.astype(np.float32)
        dx = k32 - t32
        d2 = (dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1]) + dx[:, 2] * dx[:, 2]
        exp = np.argsort(d2, kind="stable")[:3]
        got = oracle.select_nbrs(T, kt, 3)
        np.testing.assert_array_equal(got[:min(K, 3)], exp[:min(K, 3)])
        assert np.all(got[min(K, 3):] == -1)


# ----------------------------------------------------------------- weights, resampling
def test_lse_normalises_and_is_shift_invariant():
    rng = np.random.default_rng(15)
    lw = rng.normal(size=1000) * 50 - 1e4
    ll = rng.normal(size=1000) * 30
    a = oracle.lse(lw, ll)
    assert abs(a["w"].sum() - 1.0) < 1e-13
    b = oracle.lse(lw + 12345.678, ll)
    np.testing.assert_allclose(a["w"], b["w"], rtol=1e-9, atol=1e-300)
    assert a["argmax"] == int(np.argmax(lw + ll))
    assert a["ess"] == pytest.approx(1.0 / (a["w"] ** 2).sum(), rel=1e-15)
    two = oracle.lse(np.array([0.0, 0.0]), np.array([-1.0, -3.0]))
    assert two["w"][0] == pytest.approx(1 / (1 + np.exp(-2.0)), rel=1e-15)
    tie = oracle.lse(np.zeros(5), np.array([1.0, 3.0, 3.0, 2.0, 3.0]))
    assert tie["argmax"] == 1
    uni = oracle.lse(np.zeros(64), np.zeros(64))
    assert uni["ess"] == pytest.approx(64.0, rel=1e-13)


def test_resample_invariants():
    rng = np.random.default_rng(16)
    for P in [1, 2, 7, 100, 1000]:
        w = rng.random(P) ** 4
        w /= w.sum()
        u = rng.random()
        anc = oracle.resample(w, P and u)
        assert anc.shape == (P,) and anc.min() >= 0 and anc.max() < P
        assert np.all(np.diff(anc) >= 0)
        q = np.rint(w * 2.0 ** 52)
        counts = np.bincount(anc, minlength=P)
        exp = P * q / q.sum()
        assert np.all(counts >= np.floor(exp) - 1e-9) and np.all(counts <= np.ceil(exp) + 1e-9)
        assert counts.sum() == P
    np.testing.assert_array_equal(oracle.resample(np.full(50, 1 / 50), 0.0), np.arange(50))
    oh = np.zeros(40)
    oh[17] = 1.0
    np.testing.assert_array_equal(oracle.resample(oh, 0.3), np.full(40, 17))


def test_resample_exact_rational_definition():
    """a_m = min{i : C_i > (u+m)/P * S}, evaluated in exact rationals where the
    rounding of (u+m)/P*S cannot change a comparison."""
    from fractions import Fraction
    rng = np.random.default_rng(17)
    P = 300
    w = rng.random(P)
    w /= w.sum()
    u = float(rng.random())
    q = [int(x) for x in np.rint(w * 2.0 ** 52)]
    C = np.cumsum(q, dtype=object)
    S = C[-1]
    anc = oracle.resample(w, u)
    for m in range(P):
        tau = (Fraction(u) + m) / P * S
        a = next(i for i in range(P) if C[i] > tau)
        if abs(float(tau) - float(C[a - 1] if a > 0 else 0)) > 1e-3 * float(S) / P:
            assert anc[m] == a


def test_paper_memory_claim():
    P, K, b, mib = [int(x) for x in open(os.path.join(GOLDEN, "paper_memory_claim.txt")).read().split("\n")[-2].split()]
    assert round(P * K * b / 2 ** 20) == mib


# ----------------------------------------------------------------- SE(3) right Jacobian
@pytest.mark.parametrize("scale", [0.0, 1e-6, 0.05, 0.099, 0.101, 0.7, 2.0])
def test_se3_right_jacobian_matches_matrix_exponential(scale):
    """Column d of Jr(xi) is log(exp(xi)^-1 exp(xi + h e_d)) / h, from scipy's
    expm and logm (central differences, h = 1e-6)."""
    rng = np.random.default_rng(int(scale * 1000) + 7)
    for _ in range(3):
        w = rng.normal(size=3)
        w = w / np.linalg.norm(w) * scale
        xi = np.concatenate([w, rng.normal(size=3)])
        J = oracle.se3_jr(xi)
        h = 1e-6
        E0inv = np.linalg.inv(scipy.linalg.expm(twist(xi)))
        num = np.zeros((6, 6))
        for d in range(6):
            e = np.zeros(6)
            e[d] = h
            Lp = scipy.linalg.logm(E0inv @ scipy.linalg.expm(twist(xi + e))).real
            Lm = scipy.linalg.logm(E0inv @ scipy.linalg.expm(twist(xi - e))).real
            D = (Lp - Lm) / (2 * h)
            num[:, d] = [D[2, 1], D[0, 2], D[1, 0], D[0, 3], D[1, 3], D[2, 3]]
        np.testing.assert_allclose(J, num, atol=2e-7)
    np.testing.assert_array_equal(oracle.se3_jr(np.zeros(6)), np.eye(6))


# ----------------------------------------------------------------- keyframe propagation, Eq. 8-10
def test_propagation_closed_form():
    """Oldest neighbour o keeps its pose (ratio 0), keyframes before it are not
    touched, keyframe k > o moves by expm(r_k psi) with r_k = (D_k - D_o)/(Dt - D_o),
    a keyframe at the current path length moves like the current pose (ratio 1)."""
    rng = np.random.default_rng(21)
    K = 7
    kf = np.stack([expm_pose(rng.normal(size=6)) for _ in range(K)])
    psi = np.array([0.01, -0.02, 0.015, 0.05, -0.03, 0.02])
    D = np.array([0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 9.0])
    out = oracle.propagate(psi, [3, 5, 4], D, 9.0, kf)
    for k in range(K):
        if k <= 3:
            np.testing.assert_array_equal(out[k], kf[k])
        else:
            r = (D[k] - 3.0) / 6.0
            np.testing.assert_allclose(to44(out[k]), to44(kf[k]) @ to44(expm_pose(r * psi)), atol=1e-14)
    np.testing.assert_allclose(to44(out[6]), to44(kf[6]) @ to44(expm_pose(psi)), atol=1e-14)
    # no path travelled since the oldest neighbour: nothing moves
    np.testing.assert_array_equal(oracle.propagate(psi, [3, 5, 4], D, 3.0, kf), kf)
    # ratios clamp to [0, 1]
    D2 = D.copy()
    D2[5] = 20.0
    out2 = oracle.propagate(psi, [3, 5, 4], D2, 9.0, kf)
    np.testing.assert_allclose(to44(out2[5]), to44(kf[5]) @ to44(expm_pose(psi)), atol=1e-14)


def test_loop_condition():
    assert oracle.loop([5, 6, 7], 8, 0)
    assert oracle.loop([5, 6, 7], 8, 2)          # oldest neighbour 5 < 8 - 2
    assert not oracle.loop([6, 7, 5], 8, 3)      # 5 is among the 3 newest
    assert oracle.loop([6, 7, 4], 8, 3)
    assert not oracle.loop([-1, -1, -1], 8, 1)
