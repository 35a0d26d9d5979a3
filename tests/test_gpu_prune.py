"""Dead-particle pruning (Sec. III-F) on the GPU against the oracle's pruning:
the stand-alone hook on given weights (bit-exact dead set and ancestors, split
log-weights to rounding), the whole frame under the pruning policy against the
same frame without resampling (survivors untouched, dead slots hold their
ancestor's state), tracking over several frames, and a served session equal
to the plain step under the same policy."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_common import make_filter, torch_cuda

pytestmark = pytest.mark.gpu

LL_CUT32 = math.log(float(np.float32(1e-16)))   # the context's prune_lr is a float


def _weights(rng, P, dead_frac):
    lw = rng.normal(0.0, 1.0, P)
    dead = rng.random(P) < dead_frac
    lw[dead] = np.log(1e-12) + rng.normal(0.0, 3.0, dead.sum())
    lw -= lw.max()
    lw -= np.log(np.exp(lw).sum())
    return lw, np.exp(lw)


def _hook(f, x, w, ll, am, u):
    P = x.shape[0]
    anc = np.zeros(P, np.int32)
    lo = np.zeros(P)
    D = f.prune(np.ascontiguousarray(x), np.ascontiguousarray(w), ll, am, u, anc, lo)
    return anc, lo, D


def _check(anc, lo, D, ref):
    ra, rl, rD = ref
    assert D == rD
    np.testing.assert_array_equal(anc, ra)
    np.testing.assert_allclose(lo, rl, rtol=4e-16, atol=0)


@pytest.mark.parametrize("P,dead_frac,u", [(3 * 1024 + 517, 0.3, 0.37), (1024, 0.0, 0.5), (100_000, 0.6, 0.999),
                                           (1, 0.0, 0.2), (2048, 0.95, 0.0)])
def test_hook_matches_oracle(P, dead_frac, u):
    torch_cuda()
    import paper_2504_18056_b300 as g
    rng = np.random.default_rng(P)
    x, w = _weights(rng, P, dead_frac)
    am = int(np.argmax(w))
    ll = (rng.normal(-400.0, 10.0, P)).astype(np.float32)
    ll[rng.random(P) < 0.05] -= 50.0
    f = g.Filter(P, 1, 16, resample=g.RESAMPLE_PRUNE)
    got = _hook(f, x, w, ll, am, u)
    ref = oracle.prune(x, w, ll.astype(np.float64), am, float(np.float32(1e-8)), LL_CUT32, u)
    _check(*got, ref)
    got2 = _hook(f, x, w, None, am, u)             # posterior criterion only
    ref2 = oracle.prune(x, w, None, am, float(np.float32(1e-8)), -np.inf, u)
    _check(*got2, ref2)
    f.close()


def test_hook_edge_cases():
    torch_cuda()
    import paper_2504_18056_b300 as g
    P = 5000
    f = g.Filter(P, 1, 16, resample=g.RESAMPLE_PRUNE)
    # one survivor: every other slot copies it and the weight splits P ways
    x = np.full(P, np.log(1e-30))
    x[4321] = 0.0
    anc, lo, D = _hook(f, x, np.exp(x), None, 4321, 0.5)
    assert D == P - 1 and np.all(anc == 4321)
    np.testing.assert_allclose(lo, -np.log(P), rtol=1e-15)
    # NaN weights are dead; -inf log-weights too
    rng = np.random.default_rng(9)
    x, w = _weights(rng, P, 0.0)
    x[[3, 1500]] = np.nan
    w[[3, 1500]] = np.nan
    x[7] = -np.inf
    w[7] = 0.0
    am = int(np.nanargmax(w))
    anc, lo, D = _hook(f, x, w, None, am, 0.25)
    ref = oracle.prune(x, w, None, am, float(np.float32(1e-8)), -np.inf, 0.25)
    assert D == 3 == ref[2]
    np.testing.assert_array_equal(anc, ref[0])
    assert np.isfinite(lo).all()
    # no dead particle: log-weights come back bit for bit
    x, w = _weights(rng, P, 0.0)
    anc, lo, D = _hook(f, x, w, None, int(np.argmax(w)), 0.5)
    assert D == 0
    np.testing.assert_array_equal(anc, np.arange(P))
    np.testing.assert_array_equal(lo, x)
    f.close()


def test_frame_under_pruning_equals_frame_without_resampling_plus_refill():
    """Same seed, same inputs: the pruning context's frame equals the
    no-resampling context's frame up to the weighting, then its dead slots (as
    the oracle's pruning decides them from the GPU's own weights and
    log-likelihoods) hold their ancestors' current and keyframe poses."""
    P = 2000
    w = synth.box_room_workload(seed=0, n_particles=P, n_frames=3)
    fa = make_filter(w, P, max_points=1024, seed=11, resample=2)
    fb = make_filter(w, P, max_points=1024, seed=11, resample=3)
    K = len(w["keyframes"])
    for fr in range(3):
        oa = fa.step(w["scans"][fr], w["odometry"][fr], w["cov"], u=0.3)
        ob = fb.step(w["scans"][fr], w["odometry"][fr], w["cov"], u=0.3)
        assert not ob["resampled"]
        ll = np.zeros(P, np.float32)
        wa = np.zeros(P)
        wb = np.zeros(P)
        anc = np.zeros(P, np.int32)
        fa.frame_diag(ll, wa, None, None)
        fb.frame_diag(None, wb, anc, None)
        pa, la = fa.particles()
        pb, lb = fb.particles()
        if fr == 0:
            np.testing.assert_array_equal(wa, wb)
            assert oa["argmax"] == ob["argmax"]
            ref_anc, ref_lo, D = oracle.prune(la, wa, ll.astype(np.float64), oa["argmax"], float(np.float32(1e-8)),
                                              LL_CUT32, 0.3)
            assert ob["pruned"] == D and D > 0
            np.testing.assert_array_equal(anc, ref_anc)
            np.testing.assert_allclose(lb, ref_lo, rtol=4e-16, atol=0)
            dead = anc != np.arange(P)
            np.testing.assert_array_equal(pb[~dead], pa[~dead])
            np.testing.assert_array_equal(pb[dead], pa[anc[dead]])
            for k in range(K):
                ka = np.zeros((P, 12), np.float32)
                kb = np.zeros((P, 12), np.float32)
                fa.get_kf_poses(k, ka)
                fb.get_kf_poses(k, kb)
                np.testing.assert_array_equal(kb, ka[anc])
            # the survivors' weighted measure is kept
            surv = ~dead
            per = np.bincount(anc, weights=np.exp(lb), minlength=P)
            np.testing.assert_allclose(per[surv], wa[surv], rtol=1e-13)
        else:
            # free-running afterwards: weights stay normalised over the survivors' mass
            assert 0.999 < np.exp(lb).sum() <= 1.0 + 1e-12
        err = np.linalg.norm(ob["estimate"][[3, 7, 11]] - w["truth"][fr + 1][[3, 7, 11]])
        assert err < w["h"], (fr, err)
    fa.close()
    fb.close()


def test_served_session_under_pruning_equals_plain_step():
    import paper_2504_18056_b300 as g
    torch_cuda()
    w = synth.box_room_workload(seed=4, n_particles=3000, n_frames=3)
    P, K = w["particles"].shape[0], len(w["keyframes"])
    srv = g.Server(budget_bytes=8 << 30, max_sessions=4, background=True, resample=g.RESAMPLE_PRUNE)
    sid = srv.open(P, K, 1024, table_bytes=0, seed=21)
    s = srv.session(sid)
    s.init_particles(np.ascontiguousarray(w["particles"]))
    for k, kf in enumerate(w["keyframes"]):
        s.add_keyframe(kf["points"], kf["grid"], np.ascontiguousarray(w["kf_particle_poses"][k]))
    srv.ready(sid)
    tickets = [srv.submit(sid, w["scans"][fr], w["odometry"][fr], w["cov"]) for fr in range(3)]
    srv.drain()
    served = []
    for t in tickets:
        r = None
        while r is None:
            r = srv.poll(t)
        served.append(r[0])
    sp, sl = s.particles()
    srv.close()
    f = make_filter(w, P, max_points=1024, seed=21, resample=g.RESAMPLE_PRUNE)
    plain = [f.step(w["scans"][fr], w["odometry"][fr], w["cov"]) for fr in range(3)]
    pp, pl = f.particles()
    f.close()
    for a, b in zip(served, plain):
        np.testing.assert_array_equal(a["estimate"], b["estimate"])
        assert a["pruned"] == b["pruned"] and a["ess"] == b["ess"]
    assert plain[0]["pruned"] > 0
    np.testing.assert_array_equal(sp, pp)
    np.testing.assert_array_equal(sl, pl)
