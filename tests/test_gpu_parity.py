"""Stage-by-stage parity of the CUDA path (through the C ABI) with the FP64
oracle on the same seeded inputs: tables, neighbour selection, prediction,
lookup/gradient/moments, the move, weighting and resampling."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import (grad_tolerance, gpu_eval, gpu_nbr, make_filter, moment_scales, oracle_nbr,
                        torch_cuda)

pytestmark = pytest.mark.gpu

P_SMALL = 1000          # not a multiple of 32: the last particle tile is ragged


@pytest.fixture(scope="module")
def quantised_tables(box_room_tables):
    """The oracle's own tables as the 16-bit records store them (cell coefficients)."""
    return {dt: [oracle.stored_table(t, dt) for t in box_room_tables] for dt in (1, 2)}


# --------------------------------------------------------------------------- tables
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_tables_match_oracle(box_room, box_room_tables, quantised_tables, dtype, layout):
    """The stored tables read back (vertex values and cell coefficients) against
    the oracle's, for the dense and the column-sparse layout (which reads as zero
    every cell it does not store)."""
    f = make_filter(box_room, 64, dtype, table_layout=layout)
    ulp = {1: 2.0 ** -7, 2: 2.0 ** -10}
    for k, kf in enumerate(box_room["keyframes"]):
        nx, ny, nz = kf["grid"]["dims"]
        vals = np.zeros((nz, ny, nx), np.float32)
        f.get_table(k, vals)
        ref = box_room_tables[k]
        assert ref.max() > 0.99 and (ref > 0).mean() > 0.05
        if dtype == 0:
            assert np.abs(vals - ref).max() <= 5e-6
        else:
            # every cell's stored coefficients against the oracle's quantisation of its own
            # table: the GPU rounds coefficients it formed in float from float corners (each
            # within ~2.4e-7 of its exact value), the oracle the FP32 rounding of its double
            # coefficients, so a small coefficient can land one storage unit apart (measured:
            # 0.26 % of them)
            q = quantised_tables[dtype][k]
            got = np.zeros((q.shape[0] * q.shape[1] * q.shape[2], 8), np.float32)
            f.get_records(k, 0, got.shape[0], got)
            got = got.reshape(q.shape).astype(np.float64)
            bad = got != q
            assert bad.mean() <= 1e-2, bad.mean()
            assert np.all(np.abs(got[bad] - q[bad]) <= ulp[dtype] * np.abs(q[bad]) + 1e-6)
            # vertex read-back: the corner sums of the stored coefficients
            corner = q[..., 0]
            assert np.abs(vals[:-1, :-1, :-1] - corner).max() <= 2 * ulp[dtype] * corner.max() + 4e-6
    f.close()


# --------------------------------------------------------------------------- neighbours
def test_select_matches_oracle(box_room):
    f = make_filter(box_room, P_SMALL)
    nbr = gpu_nbr(f, P_SMALL, 3)
    ref = oracle_nbr(box_room["particles"][:P_SMALL], box_room["kf_particle_poses"])
    np.testing.assert_array_equal(nbr, ref)
    f.close()


def test_select_ties_and_few_keyframes(box_room):
    w = dict(box_room)
    kfp = [p.copy() for p in box_room["kf_particle_poses"]]
    kfp[3][:, [3, 7, 11]] = kfp[1][:, [3, 7, 11]]          # exact ties: keyframe 1 must win
    w["kf_particle_poses"] = kfp
    f = make_filter(w, 100)
    nbr = gpu_nbr(f, 100, 3)
    np.testing.assert_array_equal(nbr, oracle_nbr(w["particles"][:100], kfp))
    f.close()
    f2 = make_filter(box_room, 40, keyframes=box_room["keyframes"][:2])
    nbr2 = gpu_nbr(f2, 40, 2)
    np.testing.assert_array_equal(nbr2, oracle_nbr(box_room["particles"][:40], box_room["kf_particle_poses"][:2]))
    f2.close()


# --------------------------------------------------------------------------- prediction
@pytest.mark.parametrize("given_noise", [True, False])
def test_predict_matches_oracle(box_room, given_noise):
    P = P_SMALL
    f = make_filter(box_room, P, seed=1234)
    rng = np.random.default_rng(3)
    dT = box_room["odometry"][2]
    cov = box_room["cov"] * 4.0
    cov[0, 3] = cov[3, 0] = 0.5 * np.sqrt(cov[0, 0] * cov[3, 3])
    z = rng.normal(size=(P, 6)).astype(np.float32) if given_noise else None
    f.predict(dT, cov, z, frame=7)
    got, _ = f.particles()
    for i in range(P):
        zi = z[i].astype(np.float64) if given_noise else oracle.normal6(1234, i, 7)
        ref = oracle.predict(box_room["particles"][i].astype(np.float64), dT, cov, zi)
        t = np.abs(ref[[3, 7, 11]]).max()
        assert np.abs(got[i] - ref).max() <= 2e-6 * (1 + t), i
    f.close()


# --------------------------------------------------------------------------- lookups
def _check_eval(ll, g, mom, o, scan, label):
    rel_ll = np.abs(ll - o["ll"]) / np.abs(o["ll"])
    assert rel_ll.max() <= 1e-4, (label, rel_ll.max())
    err = np.linalg.norm(g - o["g"], axis=1)
    tol = grad_tolerance(o)
    worst = int(np.argmax(err / tol))
    assert np.all(err <= tol), (label, worst, err[worst], tol[worst], o["slack"][worst])
    sc = moment_scales(o["mom"], scan)
    assert np.all(np.abs(mom - o["mom"]) <= 1e-4 * sc), label
    # almost every particle is within the strict bound without any face slack
    strict = err <= 1e-3 * np.maximum(np.linalg.norm(o["g"], axis=1), 1e-2 * o["gabs"])
    assert strict.mean() >= 0.8, (label, strict.mean())


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_eval_matches_oracle(box_room, box_room_tables, quantised_tables, dtype, layout):
    P = P_SMALL
    f = make_filter(box_room, P, dtype, table_layout=layout)
    scan = box_room["scans"][0]
    nbr = gpu_nbr(f, P, 3)
    ref_nbr = oracle_nbr(box_room["particles"][:P], box_room["kf_particle_poses"])
    np.testing.assert_array_equal(nbr, ref_nbr)
    ll, g, mom = gpu_eval(f, scan, P)
    tabs = box_room_tables if dtype == 0 else quantised_tables[dtype]
    o = oracle.eval_batch(box_room["particles"][:P], ref_nbr, box_room["kf_particle_poses"], tabs,
                          [kf["grid"] for kf in box_room["keyframes"]], scan)
    _check_eval(ll, g, mom, o, scan, f"dtype{dtype}")
    # value-only pass agrees with the gradient pass
    ll2, _, _ = gpu_eval(f, scan, P, grad=False)
    np.testing.assert_allclose(ll2, ll, rtol=2e-6)
    f.close()


def test_eval_device_buffers_match_host_buffers(box_room):
    torch = torch_cuda()
    P = 300
    f = make_filter(box_room, P)
    f.select()
    scan = box_room["scans"][1]
    ll_h, g_h, m_h = gpu_eval(f, scan, P)
    scan_d = torch.from_numpy(scan).cuda()
    ll_d = torch.zeros(P, device="cuda")
    g_d = torch.zeros(P, 6, device="cuda")
    m_d = torch.zeros(P, 10, device="cuda")
    f.eval(scan_d, ll_d, g_d, m_d)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ll_d.cpu().numpy(), ll_h)
    np.testing.assert_array_equal(g_d.cpu().numpy(), g_h)
    np.testing.assert_array_equal(m_d.cpu().numpy(), m_h)
    f.close()


# --------------------------------------------------------------------------- move
def test_move_matches_oracle(box_room, box_room_tables):
    P = P_SMALL
    f = make_filter(box_room, P)
    scan = box_room["scans"][0]
    nbr = gpu_nbr(f, P, 3)
    f.move(scan)
    got, _ = f.particles()
    grids = [kf["grid"] for kf in box_room["keyframes"]]
    o = oracle.eval_batch(box_room["particles"][:P], nbr, box_room["kf_particle_poses"], box_room_tables, grids, scan)
    tol_g = grad_tolerance(o)
    errs, bounds = [], []
    for i in range(P):
        T0 = box_room["particles"][i].astype(np.float64)
        Tref, psi = oracle.move(T0, o["g"][i], o["mom"][i])
        H = oracle.h_from_moments(o["mom"][i])
        Hd = H + np.diag(np.diag(H)) * 1e-3        # lambda diag(H)
        inv_norm = 1.0 / np.linalg.eigvalsh(Hd).min()
        dH = 1e-4 * np.abs(H).max()
        bound = inv_norm * (tol_g[i] + dH * np.linalg.norm(psi)) * 1.1 + 2e-5
        xi = oracle.se3_log(oracle.pose_mul(oracle.pose_inv(Tref), got[i].astype(np.float64)))
        errs.append(np.linalg.norm(xi))
        bounds.append(bound)
    errs, bounds = np.array(errs), np.array(bounds)
    worst = int(np.argmax(errs / bounds))
    assert np.all(errs <= bounds), (worst, errs[worst], bounds[worst])
    assert np.median(errs) < 1e-4
    f.close()


# --------------------------------------------------------------------------- weights
def test_weigh_matches_oracle(box_room):
    import paper_2504_18056_b300 as gm
    torch_cuda()
    P = 5000
    f = gm.Filter(P, 1, 16)
    rng = np.random.default_rng(9)
    logw = rng.normal(size=P) * 20 - 3e3
    logw[4000] = logw[17]
    f.init_particles(np.ascontiguousarray(np.repeat(box_room["particles"][:1], P, 0)), logw)
    ll = (rng.normal(size=P) * 40 - 5e3).astype(np.float32)
    ll[17] = ll[4000] = ll.max() + 7.0        # tie: the lower index is the argmax
    w = np.zeros(P)
    res = f.weigh(ll, w)
    ref = oracle.lse(logw, ll.astype(np.float64))
    assert res["argmax"] == ref["argmax"] == 17
    np.testing.assert_allclose(w, ref["w"], rtol=1e-12, atol=1e-300)
    assert res["ess"] == pytest.approx(ref["ess"], rel=1e-12)
    assert res["log_norm"] == pytest.approx(ref["M"] + ref["logS"], rel=1e-14)
    assert abs(w.sum() - 1) < 1e-12
    f.close()


# --------------------------------------------------------------------------- resampling
@pytest.mark.parametrize("P", [1, 2, 1023, 1025, 4096, 70001])
def test_resample_bit_exact(P):
    import paper_2504_18056_b300 as g
    torch_cuda()
    f = g.Filter(70001, 1, 16)
    rng = np.random.default_rng(P)
    cases = [np.full(P, 1.0 / P), rng.random(P) ** 8, np.exp(rng.normal(size=P) * 5)]
    oh = np.zeros(P)
    oh[P // 3] = 1.0
    cases.append(oh)
    z = rng.random(P)
    z[rng.random(P) < 0.5] = 0.0
    z[0] = 1.0
    cases.append(z)
    for w in cases:
        w = w / w.sum()
        for u in [0.0, 0.5, float(rng.random()), 1.0 - 2.0 ** -53]:
            anc = np.zeros(P, np.int32)
            f.resample(np.ascontiguousarray(w), u, anc)
            np.testing.assert_array_equal(anc, oracle.resample(w, u))
    f.close()
