"""Pins of the oracle's keyframe-insertion overlap rate (Sec. III-E): the share
of the current scan's points that, moved into the last keyframe's frame by the
odometry, land in a voxel holding keyframe points. CPU only."""
import numpy as np
import pytest

import oracle


def _pose(R, t):
    return np.c_[R, t].reshape(12)


def _rot(rng):
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(rng.normal(0, 0.5, 3)).as_matrix()


def test_grid_puts_every_point_a_voxel_inside():
    rng = np.random.default_rng(0)
    pts = rng.uniform(-7.3, 12.1, (500, 3)).astype(np.float32)
    g = oracle.occupancy_grid(pts, 0.75)
    v = np.floor((pts.astype(np.float64) - g["origin"]) / g["h"])
    assert v.min() >= 1 and np.all(v.max(0) <= np.array(g["dims"]) - 2)
    assert np.allclose(g["origin"] / 0.75, np.round(g["origin"] / 0.75))


def test_self_overlap_is_one_and_far_is_zero():
    rng = np.random.default_rng(1)
    pts = rng.uniform(-5, 5, (800, 3)).astype(np.float32)
    assert oracle.overlap(pts, pts, _pose(np.eye(3), np.zeros(3)), 1.0) == 1.0
    assert oracle.overlap(pts, pts, _pose(np.eye(3), [1000.0, 0, 0]), 1.0) == 0.0


@pytest.mark.parametrize("k", [0, 1, 3, 7])
def test_slab_shifted_by_whole_voxels(k):
    """Points at voxel centres of a 10 x 4 x 4 block; shifting by k voxels along
    x leaves (10 - k) / 10 of them over occupied voxels."""
    c = np.stack(np.meshgrid(np.arange(10), np.arange(4), np.arange(4), indexing="ij"), -1).reshape(-1, 3)
    pts = (c + 0.5).astype(np.float32)
    ov = oracle.overlap(pts, pts, _pose(np.eye(3), [float(k), 0, 0]), 1.0)
    assert ov == (10 - k) / 10


def test_matches_a_set_of_voxels():
    rng = np.random.default_rng(2)
    kf = rng.normal(0, 4, (1500, 3)).astype(np.float32)
    scan = rng.normal(0, 4, (700, 3)).astype(np.float32)
    T = _pose(_rot(rng), rng.normal(0, 1, 3))
    h = 0.8
    g = oracle.occupancy_grid(kf, h)
    occ = {tuple(v) for v in np.floor((kf.astype(np.float64) - g["origin"]) / h).astype(int)}
    M = np.asarray(T).reshape(3, 4)
    x = scan.astype(np.float64) @ M[:, :3].T + M[:, 3]
    vs = np.floor((x - g["origin"]) / h).astype(int)
    expect = sum(tuple(v) in occ for v in vs) / len(scan)
    assert 0.05 < expect < 0.95
    assert oracle.overlap(kf, scan, T, h) == pytest.approx(expect, abs=1.5 / len(scan))
