"""Pins of the oracle's dead-particle pruning (Sec. III-F): the dead set from
the two criteria the section names (posterior below 1e-8, likelihood below
1e-16 of the best particle), the refill of dead slots by one systematic comb
over the survivors, checked against exact rational arithmetic, and the weight
split that keeps the survivors' weighted measure. CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

LL_CUT = float(np.log(1e-16))


def _weights(rng, P, dead_frac, tiny=1e-12):
    """Normalised log-weights x (and w = exp x) with about dead_frac of the
    particles below the posterior threshold."""
    lw = rng.normal(0.0, 1.0, P)
    dead = rng.random(P) < dead_frac
    lw[dead] = np.log(tiny) + rng.normal(0.0, 1.0, dead.sum())
    lw -= lw.max()
    lw -= np.log(np.exp(lw).sum())
    return lw, np.exp(lw), dead


def _comb_exact(w, dead, u):
    """The comb with exact rationals: q_i = rint(w_i 2^52) on survivors, tooth r
    at min((u + r) / D * S, S - 1), ancestor = first i with C_i > tooth. Also
    returns, per tooth, how far the exact tooth is from the nearest C_i (FP64
    evaluation of the tooth may differ from the exact one by a few units)."""
    q = [0 if d else int(np.rint(x * 2.0 ** 52)) for x, d in zip(w, dead)]
    C, run = [], 0
    for v in q:
        run += v
        C.append(run)
    S = run
    D = int(sum(dead))
    out, margin = [], []
    for r in range(D):
        tau = (Fraction(u) + r) / D * S
        tau = min(tau, Fraction(S - 1))
        a = next(i for i, c in enumerate(C) if c > tau)
        out.append(a)
        margin.append(min(abs(Fraction(c) - tau) for c in C))
    return out, margin, q, S


def test_no_dead_particle_changes_nothing():
    rng = np.random.default_rng(1)
    x, w, _ = _weights(rng, 300, 0.0)
    assert w.min() > 1e-8
    anc, lo, D = oracle.prune(x, w, None, int(np.argmax(w)))
    assert D == 0
    np.testing.assert_array_equal(anc, np.arange(300))
    np.testing.assert_array_equal(lo, x)


def test_dead_set_from_both_criteria():
    rng = np.random.default_rng(2)
    P = 400
    x, w, dead_w = _weights(rng, P, 0.2)
    ll = rng.normal(-50.0, 3.0, P)
    bad_ll = rng.random(P) < 0.1
    ll[bad_ll] -= 60.0                      # more than 36.84 below the best
    am = int(np.argmax(w))
    ll[am] = ll.min() - 100.0               # the largest weight survives regardless
    expect = (w < 1e-8) | (ll - ll.max() < LL_CUT)
    expect[am] = False
    anc, lo, D = oracle.prune(x, w, ll, am, 1e-8, LL_CUT, 0.3)
    assert D == expect.sum() and D > 40
    moved = anc != np.arange(P)
    np.testing.assert_array_equal(moved, expect)
    assert not expect[anc].any()            # ancestors are survivors
    # likelihood criterion off: only the posterior one
    anc2, _, D2 = oracle.prune(x, w, ll, am, 1e-8, -np.inf, 0.3)
    e2 = w < 1e-8
    e2[am] = False
    assert D2 == e2.sum()
    np.testing.assert_array_equal(anc2 != np.arange(P), e2)


@pytest.mark.parametrize("seed,u", [(3, 0.0), (4, 0.37), (5, 0.999999)])
def test_refill_matches_exact_comb(seed, u):
    rng = np.random.default_rng(seed)
    P = 257
    x, w, _ = _weights(rng, P, 0.3)
    am = int(np.argmax(w))
    anc, lo, D = oracle.prune(x, w, None, am, 1e-8, -np.inf, u)
    dead = (w < 1e-8)
    dead[am] = False
    ref, margin, q, S = _comb_exact(w, dead, u)
    got = anc[np.flatnonzero(dead)]
    assert len(ref) == D == dead.sum()
    for r, (a, b, m) in enumerate(zip(got, ref, margin)):
        if m > 8:                            # FP64 tooth cannot cross a boundary
            assert a == b, (r, a, b)
    # systematic comb: copies of each survivor within one of D q_a / S
    cnt = np.bincount(got, minlength=P)
    qa = np.array(q, dtype=object)
    lo_c = np.array([int(Fraction(int(v) * D, S)) for v in qa])
    assert np.all((cnt >= lo_c) & (cnt <= lo_c + 1))
    assert cnt.sum() == D


def test_weight_split_keeps_the_survivors_measure():
    rng = np.random.default_rng(6)
    P = 500
    x, w, _ = _weights(rng, P, 0.4)
    am = int(np.argmax(w))
    anc, lo, D = oracle.prune(x, w, None, am, 1e-8, -np.inf, 0.61)
    surv = ~((w < 1e-8) & (np.arange(P) != am))
    per_anc = np.bincount(anc, weights=np.exp(lo), minlength=P)
    np.testing.assert_allclose(per_anc[surv], w[surv], rtol=1e-13)
    assert np.all(per_anc[~surv] == 0)
    np.testing.assert_allclose(np.exp(lo).sum(), w[surv].sum(), rtol=1e-13)
    # every slot that shares an ancestor has the same log-weight
    for a in np.unique(anc):
        assert np.ptp(lo[anc == a]) == 0.0


def test_single_survivor_fills_every_slot():
    P = 64
    x = np.full(P, np.log(1e-20))
    x[17] = 0.0
    w = np.exp(x)
    anc, lo, D = oracle.prune(x, w, None, 17, 1e-8, -np.inf, 0.5)
    assert D == P - 1
    assert np.all(anc == 17)
    np.testing.assert_allclose(lo, -np.log(P), rtol=1e-15)


def test_nan_weight_is_dead():
    rng = np.random.default_rng(7)
    x, w, _ = _weights(rng, 50, 0.0)
    w[5] = np.nan
    x[5] = np.nan
    am = int(np.nanargmax(w))
    anc, lo, D = oracle.prune(x, w, None, am, 1e-8, -np.inf, 0.5)
    assert D == 1 and anc[5] != 5 and np.isfinite(lo).all()


def test_frame_with_pruning_policy(box_room_tables):
    """A whole oracle frame with policy 3: dead slots take their ancestor's
    current and keyframe poses, survivors keep theirs, and the weights keep
    the survivors' measure."""
    w = synth.box_room_workload(seed=0, n_particles=256)
    grids = [kf["grid"] for kf in w["keyframes"]]
    kfp = np.stack(w["kf_particle_poses"])
    ref = oracle.State(w["particles"], kfp, box_room_tables, grids)
    st = oracle.State(w["particles"], kfp, box_room_tables, grids)
    o_ref = ref.step(w["scans"][0], w["odometry"][0], w["cov"], frame=0, resample=2)
    o = st.step(w["scans"][0], w["odometry"][0], w["cov"], frame=0, resample=3, u=0.25)
    P = 256
    assert o["pruned"] > 0 and not o["resampled"]
    np.testing.assert_array_equal(o["w"], o_ref["w"])
    anc = o["anc"]
    dead = anc != np.arange(P)
    assert dead.sum() == o["pruned"]
    np.testing.assert_array_equal(st.poses[~dead], ref.poses[~dead])
    np.testing.assert_array_equal(st.poses[dead], ref.poses[anc[dead]])
    np.testing.assert_array_equal(st.kf_poses[:, dead], ref.kf_poses[:, anc[dead]])
    a2, lo2, D2 = oracle.prune(ref.logw, o_ref["w"], o_ref["ll"], o_ref["argmax"], 1e-8, LL_CUT, 0.25)
    assert D2 == o["pruned"]
    np.testing.assert_array_equal(a2, anc)
    np.testing.assert_array_equal(lo2, st.logw)
