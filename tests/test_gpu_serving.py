"""Serving: continuous batching of frames from several sessions into graph
launches. A session's frames must give the same result whether it is served
alone, mixed with other sessions of different sizes, or run through the plain
single-session gmcs_step (same kernels and block decomposition: bit-identical),
and sessions are admitted by the device-memory budget."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import check_moved_frame, make_filter, set_state, torch_cuda

pytestmark = pytest.mark.gpu

FRAMES = 4
SEEDS = {"A": 100, "B": 101, "C": 102, "D": 103}


@pytest.fixture(scope="module")
def worlds():
    # session A (the one compared) and three others of different sizes
    return {"A": synth.box_room_workload(seed=0, n_particles=1024, n_frames=FRAMES),
            "B": synth.box_room_workload(seed=1, n_particles=3000, n_frames=FRAMES),
            "C": synth.box_room_workload(seed=2, n_particles=257, n_frames=FRAMES),
            "D": synth.box_room_workload(seed=3, n_particles=5000, n_frames=FRAMES)}


def _open(srv, w, seed, N=None):
    P = w["particles"].shape[0]
    K = len(w["keyframes"])
    sid = srv.open(P, K, 1024, table_bytes=0, seed=seed)
    assert sid is not None
    f = srv.session(sid)
    f.init_particles(np.ascontiguousarray(w["particles"]))
    for k, kf in enumerate(w["keyframes"]):
        f.add_keyframe(kf["points"], kf["grid"], np.ascontiguousarray(w["kf_particle_poses"][k]))
    srv.ready(sid)
    return sid, f


def _serve(names, worlds, interleave=True, table_dtype=0):
    import paper_2504_18056_b300 as g
    torch_cuda()
    srv = g.Server(budget_bytes=40 << 30, max_sessions=8, background=True, table_dtype=table_dtype)
    sids = {n: _open(srv, worlds[n], seed=SEEDS[n]) for n in names}
    tickets = {n: [] for n in names}
    for fr in range(FRAMES):
        for n in (names if interleave else names[:1]):
            w = worlds[n]
            tickets[n].append(srv.submit(sids[n][0], w["scans"][fr], w["odometry"][fr], w["cov"]))
    srv.drain()
    out = {}
    for n in names:
        res = []
        for t in tickets[n]:
            r = None
            while r is None:
                r = srv.poll(t)
            res.append(r)
        poses, logw = sids[n][1].particles()
        out[n] = (res, poses, logw)
    stats = srv.stats()
    srv.close()
    return out, stats


# FP32 tables (pipelined lookup bodies) and BF16 tables (unrolled bodies) in the batched kernels
@pytest.mark.parametrize("dtype", [0, 1])
def test_served_session_equals_plain_step(worlds, dtype):
    served, stats = _serve(["A"], worlds, table_dtype=dtype)
    w = worlds["A"]
    f = make_filter(w, w["particles"].shape[0], dtype=dtype, max_points=1024, seed=100)
    plain = [f.step(w["scans"][fr], w["odometry"][fr], w["cov"]) for fr in range(FRAMES)]
    poses, logw = f.particles()
    f.close()
    res, sposes, slogw = served["A"]
    for fr in range(FRAMES):
        a, b = res[fr][0], plain[fr]
        np.testing.assert_array_equal(a["estimate"], b["estimate"])
        assert a["ess"] == b["ess"] and a["argmax"] == b["argmax"] and a["frame"] == b["frame"] == fr
    np.testing.assert_array_equal(sposes, poses)
    np.testing.assert_array_equal(slogw, logw)
    assert stats["frames"] == FRAMES and stats["latency_p50_s"] > 0


def test_session_same_alone_and_in_the_mix(worlds):
    alone, _ = _serve(["A"], worlds)
    mixed, stats = _serve(["B", "A", "C", "D"], worlds)
    ra, pa, la = alone["A"]
    rm, pm, lm = mixed["A"]
    for fr in range(FRAMES):
        np.testing.assert_array_equal(ra[fr][0]["estimate"], rm[fr][0]["estimate"])
        assert ra[fr][0]["ess"] == rm[fr][0]["ess"]
    np.testing.assert_array_equal(pa, pm)
    np.testing.assert_array_equal(la, lm)
    assert stats["frames"] == 4 * FRAMES
    assert stats["mean_sessions_per_tick"] > 1.0          # frames of several sessions shared ticks
    for n in "BCD":
        err = np.linalg.norm(mixed[n][0][-1][0]["estimate"][[3, 7, 11]] - worlds[n]["truth"][FRAMES][[3, 7, 11]])
        assert err < 0.25, (n, err)


def test_admission_by_budget(worlds):
    import paper_2504_18056_b300 as g
    torch_cuda()
    w = worlds["D"]
    P, K = w["particles"].shape[0], len(w["keyframes"])
    probe = g.Server(budget_bytes=1 << 40, max_sessions=4, background=False)
    sid, f = _open(probe, w, 1)
    one = probe.stats()["used_bytes"]
    probe.close()
    srv = g.Server(budget_bytes=int(one * 1.5), max_sessions=4, background=False)
    s1, _ = _open(srv, w, 1)
    assert abs(srv.stats()["used_bytes"] - one) <= 0.01 * one
    assert srv.open(P, K, 1024, table_bytes=one, seed=2) is None        # the second one does not fit
    t = srv.submit(s1, w["scans"][0], w["odometry"][0], w["cov"])
    srv.drain()
    assert srv.poll(t) is not None
    srv.close_session(s1)
    assert srv.stats()["used_bytes"] == 0
    s2 = srv.open(P, K, 1024, table_bytes=one, seed=2)                 # admitted once memory is back
    assert s2 is not None
    srv.close()


def test_served_mix_of_uneven_sessions_matches_oracle():
    """Three sessions of different particle counts (1,000, 2,500, 257) and scan
    sizes (512, 1,024, 3,000 points) served together in every tick, each compared
    with the FP64 oracle frame by frame: before every frame each session is set to
    its oracle state (rounded to float32), then the three frames share a tick and
    every session's neighbours, moved poses and log-likelihoods must meet the
    whole-frame bound of the plain path (check_moved_frame)."""
    import paper_2504_18056_b300 as g
    torch_cuda()
    specs = {"A": (0, 1000, (16, 32)), "B": (1, 2500, (16, 64)), "C": (2, 257, (30, 100))}
    worlds, tables, grids, states = {}, {}, {}, {}
    for n, (seed, P, lidar) in specs.items():
        w = synth.box_room_workload(seed=seed, n_particles=P, n_frames=3, lidar=lidar)
        worlds[n] = w
        grids[n] = [kf["grid"] for kf in w["keyframes"]]
        tables[n] = [oracle.build_table(kf["points"], kf["grid"], 0.2, 1.0) for kf in w["keyframes"]]
        states[n] = oracle.State(w["particles"], np.stack(w["kf_particle_poses"]), tables[n], grids[n])
    assert [worlds[n]["scans"][0].shape[0] for n in "ABC"] == [512, 1024, 3000]
    srv = g.Server(budget_bytes=40 << 30, max_sessions=4, background=False, resample=g.RESAMPLE_NEVER)
    sids = {}
    for n, w in worlds.items():
        P, K = w["particles"].shape[0], len(w["keyframes"])
        sid = srv.open(P, K, 4096, table_bytes=0, seed=0)
        f = srv.session(sid)
        f.init_particles(np.ascontiguousarray(w["particles"]))
        for k, kf in enumerate(w["keyframes"]):
            f.add_keyframe(kf["points"], kf["grid"], np.ascontiguousarray(w["kf_particle_poses"][k]))
        srv.ready(sid)
        sids[n] = (sid, f)
    for fr in range(3):
        tickets = {}
        for n in "ABC":
            set_state(sids[n][1], states[n])
        for n in "ABC":
            w = worlds[n]
            tickets[n] = srv.submit(sids[n][0], w["scans"][fr], w["odometry"][fr], w["cov"])
        srv.drain()
        st = srv.stats()
        assert st["mean_sessions_per_tick"] > 1.0
        for n in "ABC":
            w, (sid, f) = worlds[n], sids[n]
            assert srv.poll(tickets[n]) is not None
            P = w["particles"].shape[0]
            ll = np.zeros(P, np.float32)
            nbr = np.zeros((P, 3), np.int32)
            f.frame_diag(ll, None, None, nbr)
            moved, _ = f.particles()
            ref = states[n].step(w["scans"][fr], w["odometry"][fr], w["cov"], frame=0, resample=2)
            check_moved_frame(ll, moved, nbr, ref, states[n].poses, states[n], w["scans"][fr], grids[n], tables[n],
                              f"session {n} frame {fr}")
    srv.close()
