"""Helpers shared by the GPU parity tests: building filter sessions from the
seeded workloads and the tolerance rules the comparisons use."""
import numpy as np

import oracle


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    return torch


def make_filter(w, P, dtype=0, max_points=4096, keyframes=None, **cfg):
    """Filter session holding the first P particles of workload w and its keyframes."""
    import paper_2504_18056_b300 as g
    torch_cuda()
    kfs = w["keyframes"] if keyframes is None else keyframes
    f = g.Filter(P, max(len(kfs), 1), max_points, table_dtype=dtype, **cfg)
    f.init_particles(np.ascontiguousarray(w["particles"][:P]))
    for k, kf in enumerate(kfs):
        f.add_keyframe(kf["points"], kf["grid"], np.ascontiguousarray(w["kf_particle_poses"][k][:P]))
    return f


def gpu_eval(f, scan, P, grad=True):
    ll = np.zeros(P, np.float32)
    g = np.zeros((P, 6), np.float32) if grad else None
    mom = np.zeros((P, 10), np.float32) if grad else None
    f.eval(np.ascontiguousarray(scan, np.float32), ll, g, mom)
    return ll, g, mom


def gpu_nbr(f, P, k_nb):
    nbr = np.zeros((P, k_nb), np.int32)
    f.select(nbr)
    return nbr


def oracle_nbr(poses, kf_poses, k_nb=3):
    K = len(kf_poses)
    out = np.full((poses.shape[0], min(k_nb, K)), -1, np.int32)
    for i in range(poses.shape[0]):
        kt = np.array([kf_poses[k][i][[3, 7, 11]] for k in range(K)], np.float64)
        out[i] = oracle.select_nbrs(poses[i].astype(np.float64), kt, k_nb)[:min(k_nb, K)]
    return out


def grad_tolerance(o, rel=1e-3, floor=1e-2):
    """Per particle: rel * max(|g|, floor * sum |d l_jk / d xi|) plus the face
    slack (lookups whose cell a different rounding of u could change)."""
    gn = np.linalg.norm(o["g"], axis=1)
    return rel * np.maximum(gn, floor * o["gabs"]) + o["slack"]


def moment_scales(mom, scan):
    """Absolute scales for the 10 moments: W, W max|p|, W max|p|^2."""
    pm = float(np.abs(scan).max())
    W = np.maximum(mom[:, 0], 1e-6)
    return np.stack([W] + [W * pm] * 3 + [W * pm * pm] * 6, 1)


def rel_pose_error(A, B):
    """Rotation angle (rad) and translation distance between row-major 3x4 poses."""
    A = np.asarray(A, np.float64).reshape(-1, 3, 4)
    B = np.asarray(B, np.float64).reshape(-1, 3, 4)
    R = np.einsum("nji,njk->nik", A[:, :, :3], B[:, :, :3])
    c = np.clip((np.trace(R, axis1=1, axis2=2) - 1) / 2, -1, 1)
    ang = np.arccos(c)
    # arccos loses precision near 0; use the skew part there
    skew = np.stack([R[:, 2, 1] - R[:, 1, 2], R[:, 0, 2] - R[:, 2, 0], R[:, 1, 0] - R[:, 0, 1]], 1) / 2
    ang = np.where(ang < 1e-3, np.linalg.norm(skew, axis=1), ang)
    tr = np.linalg.norm(A[:, :, 3] - B[:, :, 3], axis=1)
    return ang, tr


def set_state(f, st):
    """Load the oracle state st (rounded to float32) into the filter: poses,
    log-weights and every keyframe's per-particle poses; frame counter 0."""
    st.poses[:] = st.poses.astype(np.float32)
    st.kf_poses[:] = st.kf_poses.astype(np.float32)
    f.init_particles(st.poses.astype(np.float32), st.logw.copy())
    for k in range(st.kf_poses.shape[0]):
        f.set_kf_poses(k, np.ascontiguousarray(st.kf_poses[k].astype(np.float32)))


def check_moved_frame(ll, poses, nbr, ref, ref_poses, st, scan, grids, tables, label=""):
    """One frame without resampling, GPU against oracle from the same state.
    The moved poses may diverge by the rounding of three moves (d_i, the norm of
    log(T_oracle^-1 T_gpu)); every particle's value-pass log-likelihood must then
    agree within 1e-4 relative plus what that divergence can change it by:
    1.5 * d_i * sum_jk |d l_jk / d xi| at the oracle's pose (a Lipschitz bound of
    l over the lookups). Returns the divergences."""
    P = ll.shape[0]
    same_nbr = (nbr == ref["nbr"]).all(axis=1)
    assert same_nbr.mean() >= 0.99, (label, same_nbr.mean())
    ang, tr = rel_pose_error(poses, ref_poses)
    d = np.hypot(ang, tr)
    assert np.median(d) <= 1e-5 and d.max() <= 1e-2, (label, np.median(d), d.max())
    lip = np.zeros(P)
    for i in range(P):
        ks = [int(k) for k in ref["nbr"][i] if k >= 0]
        o = oracle.eval_particle(ref_poses[i], [st.kf_poses[k][i] for k in ks], [tables[k] for k in ks],
                                 [grids[k] for k in ks], scan)
        lip[i] = o["gabs"]
    bound = 1e-4 * np.abs(ref["ll"]) + 1.5 * d * lip
    err = np.abs(ll - ref["ll"])
    ok = err <= bound
    # a particle whose neighbour set differs (a near-tie of keyframe distances) reads other tables
    assert np.all(ok | ~same_nbr), (label, np.nonzero(~ok & same_nbr)[0][:10], (err / bound)[~ok].max())
    return d
