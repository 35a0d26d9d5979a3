"""Precision of the likelihood tables: FP32, BF16 and FP16 storage with FP32
arithmetic and FP64 weights, on the paper-scale session (100,000 particles x
2,048 points x 20 keyframes). Each result is compared (a) with the oracle fed
the same quantised table (parity, the usual tolerances) and (b) with the FP64
oracle on the unquantised field (the storage error, reported and bounded),
and whole frames are compared with the all-FP32 run on the same seeds."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_common import grad_tolerance, gpu_eval, gpu_nbr, make_filter, moment_scales, rel_pose_error

pytestmark = pytest.mark.gpu

P = 100_000
DT_NAME = {0: "f32", 1: "bf16", 2: "f16"}


@pytest.fixture(scope="module")
def forest():
    return synth.forest_workload(seed=0, n_particles=P, n_frames=4)


@pytest.fixture(scope="module")
def sample(forest):
    idx = np.unique(np.concatenate([np.linspace(0, P - 1, 48).astype(int), [1, 33, 99_998]]))
    return idx


def _rel_g(g, o):
    return np.linalg.norm(g - o["g"], axis=1) / np.maximum(np.linalg.norm(o["g"], axis=1), 1e-2 * o["gabs"])


def test_table_precision_per_result(forest, sample):
    scan = forest["scans"][0]
    grids = [kf["grid"] for kf in forest["keyframes"]]
    f32 = make_filter(forest, P, 0, max_points=2048)
    nbr = gpu_nbr(f32, P, 3)
    res32 = gpu_eval(f32, scan, P)
    f32.close()
    need = sorted(set(int(k) for k in nbr[sample].ravel()))
    exact = {k: oracle.build_table(forest["keyframes"][k]["points"], grids[k], 0.2, 1.0) for k in need}
    K = len(grids)
    o64 = oracle.eval_batch(forest["particles"], nbr, forest["kf_particle_poses"],
                            [exact.get(k) for k in range(K)], grids, scan, idx=sample)
    report = {}
    for dt in (0, 1, 2):
        if dt == 0:
            ll, g, mom = res32
            oq = o64
        else:
            f = make_filter(forest, P, dt, max_points=2048)
            np.testing.assert_array_equal(gpu_nbr(f, P, 3), nbr)
            ll, g, mom = gpu_eval(f, scan, P)
            f.close()
            quant = {k: oracle.stored_table(exact[k], dt) for k in need}
            oq = oracle.eval_batch(forest["particles"], nbr, forest["kf_particle_poses"],
                                   [quant.get(k) for k in range(K)], grids, scan, idx=sample)
        # (a) parity with the oracle on the same stored values
        assert np.all(np.abs(ll[sample] - oq["ll"]) <= 1e-4 * np.abs(oq["ll"])), DT_NAME[dt]
        assert np.all(np.linalg.norm(g[sample] - oq["g"], axis=1) <= grad_tolerance(oq)), DT_NAME[dt]
        assert np.all(np.abs(mom[sample] - oq["mom"]) <= 1e-4 * moment_scales(oq["mom"], scan)), DT_NAME[dt]
        # (b) error of the stored precision against the FP64 oracle on the exact field
        e_ll = np.abs(ll[sample] - o64["ll"]) / np.abs(o64["ll"])
        e_g = _rel_g(g[sample], o64)
        e_w = np.abs(mom[sample, 0] - o64["mom"][:, 0]) / np.maximum(o64["mom"][:, 0], 1e-6)
        e_vs32 = np.abs(ll - res32[0]) / np.abs(res32[0])
        report[DT_NAME[dt]] = {
            "ll_rel_err_max": float(e_ll.max()), "ll_rel_err_median": float(np.median(e_ll)),
            "grad_rel_err_max": float(e_g.max()), "grad_rel_err_median": float(np.median(e_g)),
            "W_rel_err_max": float(e_w.max()),
            "ll_rel_diff_vs_f32_max_all_particles": float(e_vs32.max()),
        }
    print("\nPRECISION_PER_RESULT " + json.dumps(report))
    out = os.environ.get("GMCS_REPORT_DIR")
    if out:
        with open(os.path.join(out, "precision_per_result.json"), "w") as fh:
            json.dump(report, fh, indent=1)
    assert report["f32"]["ll_rel_err_max"] <= 1e-4
    for name in ("bf16", "f16"):
        assert report[name]["ll_rel_err_max"] <= 2e-3
        assert report[name]["grad_rel_err_median"] <= 0.05


def test_whole_frames_per_table_type(forest):
    """Three frames from the same state and seeds with each table type: the
    reduced-precision runs track the FP32 run's estimate and the truth."""
    runs = {}
    for dt in (0, 1, 2):
        f = make_filter(forest, P, dt, max_points=2048, seed=11)
        outs = [f.step(forest["scans"][fr], forest["odometry"][fr], forest["cov"]) for fr in range(3)]
        ll = np.zeros(P, np.float32)
        w = np.zeros(P)
        f.frame_diag(ll, w, None, None)
        runs[dt] = (outs, ll, w)
        f.close()
    report = {}
    for dt in (1, 2):
        outs, ll, w = runs[dt]
        ang, tr = rel_pose_error(np.stack([o["estimate"] for o in outs]), np.stack([o["estimate"] for o in runs[0][0]]))
        err_truth = [float(np.linalg.norm(o["estimate"][[3, 7, 11]] - forest["truth"][fr + 1][[3, 7, 11]]))
                     for fr, o in enumerate(outs)]
        report[DT_NAME[dt]] = {"estimate_vs_f32_m": tr.tolist(), "estimate_vs_f32_rad": ang.tolist(),
                               "estimate_vs_truth_m": err_truth,
                               "ess": [o["ess"] for o in outs], "ess_f32": [o["ess"] for o in runs[0][0]]}
        assert max(err_truth) < 0.2
        assert np.all(tr < 0.2)
    print("\nPRECISION_FRAMES " + json.dumps(report))
    out = os.environ.get("GMCS_REPORT_DIR")
    if out:
        with open(os.path.join(out, "precision_frames.json"), "w") as fh:
            json.dump(report, fh, indent=1)
