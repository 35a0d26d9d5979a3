"""End-to-end behaviour of the FP64 oracle's whole frame on the plain box-room
case: with true odometry the representative particle (largest weight, as in
Sec. IV-A) stays within one voxel of the true pose. CPU only."""
import numpy as np

import oracle
import synth


def test_box_room_filter_tracks_truth(box_room_tables):
    w = synth.box_room_workload(seed=0, n_particles=512)
    st = oracle.State(w["particles"], np.stack(w["kf_particle_poses"]), box_room_tables,
                      [kf["grid"] for kf in w["keyframes"]])
    for f in range(len(w["scans"])):
        o = st.step(w["scans"][f], w["odometry"][f], w["cov"], frame=f)
        tr = w["truth"][f + 1]
        err = np.linalg.norm(o["estimate"][[3, 7, 11]] - tr[[3, 7, 11]])
        assert err < w["h"], (f, err)
        assert abs(o["w"].sum() - 1.0) < 1e-12
        assert o["resampled"] and np.all(np.diff(o["anc"]) >= 0)
        assert np.all(st.logw == -np.log(512))
        R = st.poses[:, [0, 1, 2, 4, 5, 6, 8, 9, 10]].reshape(-1, 3, 3)
        # inputs are float32 poses; the FP64 updates add no further drift
        assert np.abs(R @ R.transpose(0, 2, 1) - np.eye(3)).max() < 1e-6


def test_resample_policy_and_given_offset(box_room_tables):
    w = synth.box_room_workload(seed=0, n_particles=64)
    st = oracle.State(w["particles"], np.stack(w["kf_particle_poses"]), box_room_tables,
                      [kf["grid"] for kf in w["keyframes"]])
    o = st.step(w["scans"][0], w["odometry"][0], w["cov"], frame=0, resample=2)
    assert not o["resampled"] and np.all(o["anc"] == np.arange(64))
    np.testing.assert_allclose(np.exp(st.logw), o["w"], rtol=1e-12)
    z = np.zeros((64, 6))
    st2 = oracle.State(w["particles"], np.stack(w["kf_particle_poses"]), box_room_tables,
                       [kf["grid"] for kf in w["keyframes"]])
    o2 = st2.step(w["scans"][0], w["odometry"][0], w["cov"], frame=0, z=z, u=0.5)
    np.testing.assert_array_equal(o2["anc"], oracle.resample(o2["w"], 0.5))
