"""Checkpoint / resume (gmcs_save, gmcs_load): a session saved after two frames
and restored into a fresh context continues bit for bit like the original, for
the voxel-field and the GICP models; restoring into a context that already has
keyframes, or from a file that is not a checkpoint of this format version, is
refused."""
import numpy as np
import pytest

import synth
from gpu_common import make_filter, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,dtype", [(0, 0), (0, 1), (1, 0)])
def test_resume_is_bit_identical(tmp_path, model, dtype):
    import paper_2504_18056_b300 as g
    torch_cuda()
    w = synth.box_room_workload(seed=6, n_particles=1500, n_frames=5)
    P, K = 1500, len(w["keyframes"])
    cfg = dict(seed=9, model=model, resample=g.RESAMPLE_PRUNE if model else g.RESAMPLE_ALWAYS)
    if model == 1:
        grids = [synth.grid_for_points(kf["points"], 1.0, 1.0) for kf in w["keyframes"]]
        kfs = [dict(kf, grid=gr) for kf, gr in zip(w["keyframes"], grids)]
        a = make_filter(w, P, max_points=1024, keyframes=kfs, **cfg)
    else:
        a = make_filter(w, P, dtype=dtype, max_points=1024, **cfg)
    for fr in range(2):
        a.step(w["scans"][fr], w["odometry"][fr], w["cov"])
    path = str(tmp_path / "session.ckpt")
    a.save(path)
    b = g.Filter(P, K + 2, 1024)          # default config: the checkpoint's replaces it
    b.load(path)
    assert b.sizes() == a.sizes()
    for fr in range(2, 5):
        oa = a.step(w["scans"][fr], w["odometry"][fr], w["cov"])
        ob = b.step(w["scans"][fr], w["odometry"][fr], w["cov"])
        np.testing.assert_array_equal(oa["estimate"], ob["estimate"])
        assert oa["ess"] == ob["ess"] and oa["frame"] == ob["frame"] and oa["pruned"] == ob["pruned"]
    pa, la = a.particles()
    pb, lb = b.particles()
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(la, lb)
    a.close()
    b.close()


def test_refusals(tmp_path, box_room):
    import paper_2504_18056_b300 as g
    torch_cuda()
    a = make_filter(box_room, 256, max_points=1024)
    path = str(tmp_path / "s.ckpt")
    a.save(path)
    with pytest.raises(g.GmcsError) as e:
        a.load(path)                        # already has keyframes
    assert e.value.code == g.E_STATE
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint" * 16)
    b = g.Filter(256, 8, 1024)
    with pytest.raises(g.GmcsError) as e:
        b.load(str(bad))
    assert e.value.code == g.E_IO
    old = tmp_path / "v2.ckpt"             # a file of the earlier format (16-bit tables as corners)
    raw = bytearray(open(path, "rb").read())
    assert raw[:8] == b"GMCSCKPT" and int.from_bytes(raw[8:12], "little") == 3
    raw[8:12] = (2).to_bytes(4, "little")
    old.write_bytes(bytes(raw))
    with pytest.raises(g.GmcsError) as e:
        b.load(str(old))
    assert e.value.code == g.E_IO
    # a table block cut short: refused on the host, before any device state changes
    cut = tmp_path / "cut.ckpt"
    cut.write_bytes(open(path, "rb").read()[:-4096])
    with pytest.raises(g.GmcsError) as e:
        b.load(str(cut))
    assert e.value.code == g.E_IO
    assert b.sizes()[1] == 0                # b is still empty and usable
    b.load(path)
    assert b.sizes()[:2] == a.sizes()[:2]
    b.close()
    b = g.Filter(256, 8, 1024)
    small = g.Filter(128, 8, 1024)
    with pytest.raises(g.GmcsError) as e:
        small.load(path)                    # 256 particles do not fit 128
    assert e.value.code == g.E_CAPACITY
    for f in (a, b, small):
        f.close()
