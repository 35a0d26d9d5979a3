"""Keyframe pose propagation (Eq. 8-10) and the loop condition (Sec. III-C2) on
the GPU against the oracle: one move step, and whole frames."""
import numpy as np
import pytest

import oracle
from gpu_common import grad_tolerance, gpu_nbr, make_filter, rel_pose_error

pytestmark = pytest.mark.gpu

P = 1000


def _move_bound(o, i, psi):
    H = oracle.h_from_moments(o["mom"][i])
    Hd = H + np.diag(np.diag(H)) * 1e-3
    return 1.1 / np.linalg.eigvalsh(Hd).min() * (grad_tolerance(o)[i] + 1e-4 * np.abs(H).max() * np.linalg.norm(psi)) + 2e-5


@pytest.mark.parametrize("loop_recent", [0, 3])
def test_move_with_propagation_matches_oracle(box_room, box_room_tables, loop_recent):
    w = box_room
    K = len(w["keyframes"])
    D = np.array([0.0, 0.7, 1.9, 2.6])
    now = 4.1
    f = make_filter(w, P, propagate=1, loop_recent=loop_recent)
    f.set_path(now, D)
    scan = w["scans"][0]
    nbr = gpu_nbr(f, P, 3)
    f.move(scan)
    got, _ = f.particles()
    got_kf = [np.zeros((P, 12), np.float32) for _ in range(K)]
    for k in range(K):
        f.get_kf_poses(k, got_kf[k])
    grids = [kf["grid"] for kf in w["keyframes"]]
    o = oracle.eval_batch(w["particles"][:P], nbr, w["kf_particle_poses"], box_room_tables, grids, scan)
    moved = 0
    for i in range(P):
        T0 = w["particles"][i].astype(np.float64)
        kfi = np.stack([w["kf_particle_poses"][k][i] for k in range(K)]).astype(np.float64)
        if oracle.loop(nbr[i], K, loop_recent):
            Tref, psi = oracle.move(T0, o["g"][i], o["mom"][i])
            kref = oracle.propagate(psi, nbr[i], D, now, kfi)
            bound = _move_bound(o, i, psi)
            moved += 1
        else:
            Tref, kref, bound = T0, kfi, 1e-12
        xi = oracle.se3_log(oracle.pose_mul(oracle.pose_inv(Tref), got[i].astype(np.float64)))
        assert np.linalg.norm(xi) <= bound, (i, np.linalg.norm(xi), bound)
        for k in range(K):
            xk = oracle.se3_log(oracle.pose_mul(oracle.pose_inv(kref[k]), got_kf[k][i].astype(np.float64)))
            assert np.linalg.norm(xk) <= bound + 1e-6, (i, k, np.linalg.norm(xk), bound)
    if loop_recent == 0:
        assert moved == P
    else:
        assert 0 < moved < P
    f.close()


def test_step_with_propagation_matches_oracle(box_room, box_room_tables):
    """Whole frames with propagation: both sides start every frame from the same
    float state and path lengths; the current and keyframe poses of the
    representative particle agree."""
    w = box_room
    K = len(w["keyframes"])
    D = np.array([0.0, 0.4, 0.8, 1.2])
    f = make_filter(w, P, propagate=1)
    f.set_path(1.2, D)
    grids = [kf["grid"] for kf in w["keyframes"]]
    st = oracle.State(w["particles"][:P], np.stack([p[:P] for p in w["kf_particle_poses"]]), box_room_tables, grids,
                      kf_path=D, path_now=1.2)
    for fr in range(3):
        st.poses[:] = st.poses.astype(np.float32)
        st.kf_poses[:] = st.kf_poses.astype(np.float32)
        f.init_particles(st.poses.astype(np.float32), st.logw.copy())
        for k in range(K):
            f.set_kf_poses(k, np.ascontiguousarray(st.kf_poses[k].astype(np.float32)))
        f.set_path(st.path_now, D)
        out = f.step(w["scans"][fr], w["odometry"][fr], w["cov"])
        ref = st.step(w["scans"][fr], w["odometry"][fr], w["cov"], frame=0, propagate=1)
        anc = np.zeros(P, np.int32)
        f.frame_diag(None, None, anc, None)
        assert (anc == ref["anc"]).mean() >= 0.9
        if out["argmax"] == ref["argmax"]:
            ang, tr = rel_pose_error(out["estimate"], ref["estimate"])
            assert ang[0] < 1e-3 and tr[0] < 1e-3
        got_kf = np.zeros((P, 12), np.float32)
        for k in range(K):
            f.get_kf_poses(k, got_kf)
            same = anc == ref["anc"]
            a, t = rel_pose_error(got_kf[same], st.kf_poses[k][same])
            assert np.median(t) < 1e-4 and np.percentile(t, 99) < 5e-3, (fr, k, np.median(t), t.max())
    f.close()
