"""bench.py's reference arm on the CPU: the FP64 oracle as the reference
implementation, run by a pool of forked workers (one per host core) on disjoint
particle blocks of a small session; the JSON line carries the keys of the
benchmark contract."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2", "--warmup", "1",
           "--particles", "2000", "--points", "256", "--keyframes", "4"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "evals/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "evals/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_pool_blocks_cover_the_sample():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    w = synth.forest_workload(seed=1, n_particles=300, n_points=128, n_keyframes=4, n_frames=1)
    pool = bench.OraclePool(w, 96, max_workers=3)
    try:
        wall, per = pool.frame(0)
    finally:
        pool.close()
    assert pool.workers == min(3, bench.host_cores())
    assert pool.per_worker * pool.workers <= 96 + pool.workers
    # the workers' blocks are disjoint slices of the same particle set
    starts = [np.asarray(st.poses)[0] for st in bench._POOL_STATES]
    for i, st in enumerate(bench._POOL_STATES):
        np.testing.assert_array_equal(st.poses, w["particles"][i * pool.per_worker:(i + 1) * pool.per_worker])
    assert len({tuple(s) for s in starts}) == pool.workers
    assert wall > 0 and len(per) == pool.workers and all(t > 0 for t in per)
