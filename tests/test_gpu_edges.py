"""Edge cases of the C ABI on the GPU: degenerate sizes, particles outside
every table, empty scans, capacity and ordering errors, degenerate weights,
resampling policies."""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_eval, gpu_nbr, grad_tolerance, make_filter, oracle_nbr, torch_cuda

pytestmark = pytest.mark.gpu


# with K >= 3 the three-neighbour pass runs; P, N chosen so that its warps get point
# chunks of 1 (N = 1, 3), 9 (N = 97) and 10 points with a last chunk of 1 (N = 301):
# odd and even chunks end the software-pipelined loop at either of its two exits
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("P,N,K", [(1, 1, 1), (1, 512, 4), (33, 7, 2), (65, 300, 3), (40, 1, 4), (40, 3, 4),
                                   (65, 301, 4), (130, 97, 4)])
def test_small_shapes_match_oracle(box_room, box_room_tables, P, N, K, dtype, layout):
    """FP32, BF16 and FP16 coefficient records, dense and column-sparse tables,
    through the software-pipelined passes, against the oracle on the same stored
    values."""
    kfs = box_room["keyframes"][:K]
    f = make_filter(box_room, P, dtype=dtype, keyframes=kfs, table_layout=layout)
    tables = [oracle.stored_table(t, dtype) for t in box_room_tables[:K]]
    scan = box_room["scans"][2][:N]
    nbr = gpu_nbr(f, P, min(3, K))
    ref_nbr = oracle_nbr(box_room["particles"][:P], box_room["kf_particle_poses"][:K])
    np.testing.assert_array_equal(nbr, ref_nbr)
    ll, g, mom = gpu_eval(f, scan, P)
    o = oracle.eval_batch(box_room["particles"][:P], ref_nbr, box_room["kf_particle_poses"][:K],
                          tables, [kf["grid"] for kf in kfs], scan)
    assert np.all(np.abs(ll - o["ll"]) <= 1e-4 * np.abs(o["ll"]))
    assert np.all(np.linalg.norm(g - o["g"], axis=1) <= grad_tolerance(o))
    llv, _, _ = gpu_eval(f, scan, P, grad=False)     # the value-only pass
    assert np.all(np.abs(llv - o["ll"]) <= 1e-4 * np.abs(o["ll"]))
    f.close()


def test_passes_refuse_before_neighbour_selection(box_room):
    """The neighbour sets start empty (-1): evaluation, a move and the
    differentiable log-likelihood refuse to run (GMCS_E_STATE) until a selection or
    a step has filled them, and run once one has."""
    import paper_2504_18056_b300 as g
    P = 64
    f = make_filter(box_room, P)
    scan = np.ascontiguousarray(box_room["scans"][0])
    xi = np.zeros((P, 6), np.float32)
    ll = np.zeros(P, np.float32)
    calls = [lambda: gpu_eval(f, scan, P), lambda: f.move(scan), lambda: f.loglik(xi, scan, ll),
             lambda: f.loglik_backward(xi, scan, np.ones(P, np.float32), np.zeros((P, 6), np.float32))]
    for call in calls:
        with pytest.raises(g.GmcsError) as e:
            call()
        assert e.value.code == g.E_STATE
    f.select()
    ll1, _, _ = gpu_eval(f, scan, P)
    f.loglik(xi, scan, ll)
    np.testing.assert_allclose(ll, ll1, rtol=1e-6)
    f.close()


def test_particles_outside_every_table(box_room):
    P = 64
    w = dict(box_room)
    far = box_room["particles"][:P].copy()
    far[:, [3, 7, 11]] += 1e4
    w["particles"] = far
    f = make_filter(w, P)
    f.select()
    scan = box_room["scans"][0]
    ll, g, mom = gpu_eval(f, scan, P)
    np.testing.assert_allclose(ll, scan.shape[0] * 3 * np.log(np.float32(1e-3)), rtol=1e-5)
    assert np.all(g == 0) and np.all(mom == 0)
    before, _ = f.particles()
    f.move(scan)
    after, _ = f.particles()
    np.testing.assert_array_equal(before, after)     # no contact: no move
    f.close()


def test_empty_scan_step_only_predicts(box_room):
    P = 100
    f = make_filter(box_room, P, seed=3, resample=2)
    dT, cov = box_room["odometry"][0], box_room["cov"]
    out = f.step(np.zeros((0, 3), np.float32), dT, cov)
    assert out["status"] == 0 and not out["resampled"]
    got, logw = f.particles()
    for i in range(P):
        ref = oracle.predict(box_room["particles"][i].astype(np.float64), dT, cov, oracle.normal6(3, i, 0))
        assert np.abs(got[i] - ref).max() < 1e-5
    np.testing.assert_allclose(logw, -np.log(P), rtol=1e-12)
    f.close()


def test_capacity_and_order_errors(box_room):
    import paper_2504_18056_b300 as g
    torch_cuda()
    f = g.Filter(10, 1, 8)
    scan = box_room["scans"][0][:8]
    with pytest.raises(g.GmcsError) as e:
        f.step(scan, box_room["odometry"][0], box_room["cov"])
    assert e.value.code == g.E_STATE
    with pytest.raises(g.GmcsError) as e:
        f.init_particles(np.ascontiguousarray(box_room["particles"][:11]))
    assert e.value.code == g.E_CAPACITY
    f.init_particles(np.ascontiguousarray(box_room["particles"][:10]))
    kf = box_room["keyframes"][0]
    f.add_keyframe(kf["points"], kf["grid"])
    with pytest.raises(g.GmcsError) as e:
        f.add_keyframe(kf["points"], kf["grid"])
    assert e.value.code == g.E_CAPACITY
    with pytest.raises(g.GmcsError) as e:
        f.step(box_room["scans"][0][:9], box_room["odometry"][0], box_room["cov"])
    assert e.value.code == g.E_CAPACITY
    out = f.step(scan, box_room["odometry"][0], box_room["cov"])     # exactly max_points
    assert out["status"] == 0
    bad = dict(kf["grid"])
    bad["dims"] = (1, 5, 5)
    f2 = g.Filter(10, 2, 8)
    f2.init_particles(np.ascontiguousarray(box_room["particles"][:10]))
    with pytest.raises(g.GmcsError) as e:
        f2.add_keyframe(kf["points"], bad)
    assert e.value.code == g.E_INVALID
    with pytest.raises(g.GmcsError) as e:
        f.step(scan, box_room["odometry"][0], box_room["cov"], u=1.5)
    assert e.value.code == g.E_INVALID
    f.close()
    f2.close()


def test_degenerate_weights_reset_to_uniform(box_room):
    P = 50
    f = make_filter(box_room, P)
    f.init_particles(np.ascontiguousarray(box_room["particles"][:P]), np.full(P, -np.inf))
    out = f.step(box_room["scans"][0], box_room["odometry"][0], box_room["cov"])
    assert out["status"] == -6 and not out["resampled"]
    _, logw = f.particles()
    np.testing.assert_allclose(logw, -np.log(P))
    f.close()


@pytest.mark.parametrize("policy", [1, 2])
def test_resample_policies(box_room, policy):
    P = 256
    f = make_filter(box_room, P, resample=policy)
    out = f.step(box_room["scans"][0], box_room["odometry"][0], box_room["cov"])
    w = np.zeros(P)
    anc = np.zeros(P, np.int32)
    f.frame_diag(None, w, anc, None)
    _, logw = f.particles()
    if policy == 2 or out["ess"] >= P / 2:
        assert not out["resampled"]
        np.testing.assert_array_equal(anc, np.arange(P))
        np.testing.assert_allclose(np.exp(logw), w, rtol=1e-12, atol=1e-300)
    else:
        assert out["resampled"]
        np.testing.assert_allclose(logw, -np.log(P))
        np.testing.assert_array_equal(anc, oracle.resample(w, oracle.systematic_u(0, 0)))
    f.close()


def test_given_offset_and_stats(box_room):
    P = 128
    f = make_filter(box_room, P)
    f.set_profiling(True)
    f.reset_stats()
    f.step(box_room["scans"][0], box_room["odometry"][0], box_room["cov"], u=0.25)
    w = np.zeros(P)
    anc = np.zeros(P, np.int32)
    f.frame_diag(None, w, anc, None)
    np.testing.assert_array_equal(anc, oracle.resample(w, 0.25))
    s = f.stats()
    assert s["frames"] == 1 and s["launches"] >= 12
    assert s["kinds"]["pass_grad"]["ms"] > 0 and s["kinds"]["pass_grad"]["launches"] == 3
    assert f.device_bytes() > 0
    f.close()


def test_non_finite_scan_points_are_misses(box_room):
    """NaN / inf scan points (a dropped lidar return) do not poison the frame: the
    normalised weights, the estimate and the moved particles equal those of the
    same frame with the points removed (up to the float summation order)."""
    P = 1024
    w = box_room
    scan = w["scans"][0].copy()
    bad = np.array([3, 100, 257, 511])
    dirty = scan.copy()
    dirty[bad[0], 0] = np.nan
    dirty[bad[1]] = np.inf
    dirty[bad[2], 2] = -np.inf
    dirty[bad[3], 1] = np.nan
    clean = np.delete(scan, bad, axis=0)
    outs, parts, ws = [], [], []
    for s in (dirty, clean):
        f = make_filter(w, P, seed=2, resample=2)      # no resampling: compare the moved particles
        outs.append(f.step(np.ascontiguousarray(s), w["odometry"][0], w["cov"]))
        wg = np.zeros(P)
        f.frame_diag(None, wg, None, None)
        ws.append(wg)
        parts.append(f.particles()[0])
        f.close()
    assert outs[0]["status"] == 0 and np.isfinite(ws[0]).all()
    np.testing.assert_allclose(ws[0], ws[1], rtol=1e-2, atol=1e-12)
    assert outs[0]["argmax"] == outs[1]["argmax"]
    np.testing.assert_allclose(outs[0]["estimate"], outs[1]["estimate"], atol=1e-5)
    np.testing.assert_allclose(parts[0], parts[1], atol=1e-4)
