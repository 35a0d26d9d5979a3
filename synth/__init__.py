"""Seeded synthetic inputs for the particle-update hot path.

This module is shared by the FP64 oracle tests, the CUDA parity tests and the
benchmark. It produces scenes, ray-cast lidar scans, trajectories, keyframe
point clouds, voxel-lattice geometry and particle sets. It holds none of the
filter's arithmetic: no likelihood field, no lookup, no gradient, no SE(3)
exponential of the method, no weighting and no resampling. Rotations for
perturbations come from scipy's rotation-vector conversion.

Poses are 3x4 row-major [R | t] matrices flattened to 12 numbers, mapping
sensor-frame points into the world frame: x_w = R p + t.

The workloads follow the paper's setting (Sec. III-A: a lidar scan, shared
keyframe clouds, particles holding a current pose plus one pose per keyframe)
with synthetic stand-ins for its recorded datasets (Sec. IV uses a Livox
MID-360 in a forest-like area; those recordings are not available here).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial.transform import Rotation

__all__ = [
    "Scene", "box_room", "corridor_forest", "lidar_dirs", "cast_scan",
    "pose_from_rt", "pose_mul", "pose_inv", "pose_apply", "perturb_poses",
    "grid_for_points", "sample_surfaces", "room_walk", "loop_walk",
    "box_room_workload", "forest_workload", "random_uniform_poses",
]


# ----------------------------------------------------------------------------
# pose helpers (plain composition; data generation only)
# ----------------------------------------------------------------------------

def pose_from_rt(R, t):
    T = np.zeros(12, dtype=np.float64)
    T.reshape(3, 4)[:, :3] = R
    T.reshape(3, 4)[:, 3] = t
    return T


def pose_mul(A, B):
    """Composition A*B of poses given as (..., 12) arrays."""
    A = np.asarray(A, dtype=np.float64).reshape(-1, 3, 4)
    B = np.asarray(B, dtype=np.float64).reshape(-1, 3, 4)
    R = A[:, :, :3] @ B[:, :, :3]
    t = (A[:, :, :3] @ B[:, :, 3:4])[..., 0] + A[:, :, 3]
    out = np.concatenate([R, t[..., None]], axis=2).reshape(-1, 12)
    return out


def pose_inv(A):
    A = np.asarray(A, dtype=np.float64).reshape(-1, 3, 4)
    Rt = np.transpose(A[:, :, :3], (0, 2, 1))
    t = -(Rt @ A[:, :, 3:4])[..., 0]
    return np.concatenate([Rt, t[..., None]], axis=2).reshape(-1, 12)


def pose_apply(T, pts):
    T = np.asarray(T, dtype=np.float64).reshape(3, 4)
    return pts @ T[:, :3].T + T[:, 3]


def perturb_poses(T, n, trans_std, rot_std, rng):
    """n copies of pose T, each right-multiplied by a random rigid motion with
    rotation vector ~ N(0, rot_std^2 I) and translation ~ N(0, trans_std^2 I)."""
    rv = rng.normal(0.0, rot_std, size=(n, 3))
    dt = rng.normal(0.0, trans_std, size=(n, 3))
    dR = Rotation.from_rotvec(rv).as_matrix()
    D = np.concatenate([dR, dt[..., None]], axis=2).reshape(n, 12)
    return pose_mul(np.repeat(np.asarray(T, np.float64).reshape(1, 12), n, 0), D)


def random_uniform_poses(n, rng, trans_box, rot_std):
    R = Rotation.from_rotvec(rng.normal(0, rot_std, size=(n, 3))).as_matrix()
    lo, hi = np.asarray(trans_box[0]), np.asarray(trans_box[1])
    t = lo + (hi - lo) * rng.random((n, 3))
    return np.concatenate([R, t[..., None]], axis=2).reshape(n, 12)


# ----------------------------------------------------------------------------
# scenes and ray casting
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    """Planes (n, d) with n.x = d, axis-aligned boxes (lo, hi), and vertical
    cylinders (cx, cy, r, z0, z1). Planes carry an optional rectangular extent
    used only for surface sampling."""
    planes: np.ndarray            # (Np, 4)  nx ny nz d
    plane_extent: np.ndarray      # (Np, 6)  lo xyz, hi xyz (sampling box)
    boxes: np.ndarray             # (Nb, 6)  lo xyz, hi xyz
    cylinders: np.ndarray         # (Nc, 5)  cx cy r z0 z1

    def raycast(self, o, d, max_range=np.inf):
        """Nearest hit distance along unit directions d from origins o; inf on miss."""
        o = np.asarray(o, np.float64).reshape(-1, 3)
        d = np.asarray(d, np.float64).reshape(-1, 3)
        M = d.shape[0]
        if o.shape[0] == 1:
            o = np.repeat(o, M, 0)
        best = np.full(M, np.inf)
        # planes
        for (nx, ny, nz, dd) in self.planes:
            n = np.array([nx, ny, nz])
            den = d @ n
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (dd - o @ n) / den
            ok = (np.abs(den) > 1e-12) & (t > 1e-9)
            best = np.where(ok & (t < best), t, best)
        # boxes: slab test, entry distance (rays start outside boxes)
        if len(self.boxes):
            lo = self.boxes[None, :, 0:3]
            hi = self.boxes[None, :, 3:6]
            with np.errstate(divide="ignore", invalid="ignore"):
                inv = 1.0 / d[:, None, :]
                t1 = (lo - o[:, None, :]) * inv
                t2 = (hi - o[:, None, :]) * inv
            tmin = np.nanmax(np.minimum(t1, t2), axis=2)
            tmax = np.nanmin(np.maximum(t1, t2), axis=2)
            hit = (tmax >= tmin) & (tmin > 1e-9)
            tb = np.where(hit, tmin, np.inf).min(axis=1)
            best = np.minimum(best, tb)
        # vertical cylinders: side surface only
        if len(self.cylinders):
            c = self.cylinders
            ox = o[:, 0:1] - c[None, :, 0]
            oy = o[:, 1:2] - c[None, :, 1]
            dx, dy = d[:, 0:1], d[:, 1:2]
            a = dx * dx + dy * dy
            b = ox * dx + oy * dy
            cc = ox * ox + oy * oy - c[None, :, 2] ** 2
            disc = b * b - a * cc
            with np.errstate(divide="ignore", invalid="ignore"):
                sq = np.sqrt(np.maximum(disc, 0.0))
                t = (-b - sq) / a
            z = o[:, 2:3] + t * d[:, 2:3]
            ok = (disc > 0) & (a > 1e-12) & (t > 1e-9) & (z >= c[None, :, 3]) & (z <= c[None, :, 4])
            tc = np.where(ok, t, np.inf).min(axis=1)
            best = np.minimum(best, tc)
        best[best > max_range] = np.inf
        return best


def box_room(seed=0, size=(20.0, 20.0, 5.0), n_boxes=8):
    """20 x 20 x 5 m room: floor, ceiling, four walls, plus random boxes."""
    rng = np.random.default_rng(seed)
    sx, sy, sz = size
    hx, hy = sx / 2, sy / 2
    planes = np.array([
        [0, 0, 1, 0.0], [0, 0, 1, sz],
        [1, 0, 0, -hx], [1, 0, 0, hx],
        [0, 1, 0, -hy], [0, 1, 0, hy],
    ], dtype=np.float64)
    ext = np.array([
        [-hx, -hy, 0, hx, hy, 0], [-hx, -hy, sz, hx, hy, sz],
        [-hx, -hy, 0, -hx, hy, sz], [hx, -hy, 0, hx, hy, sz],
        [-hx, -hy, 0, hx, -hy, sz], [-hx, hy, 0, hx, hy, sz],
    ], dtype=np.float64)
    boxes = []
    for _ in range(n_boxes):
        w = rng.uniform(0.5, 2.0, size=2)
        h = rng.uniform(0.5, 2.5)
        c = rng.uniform(-hx + 2.0, hx - 2.0, size=2)
        boxes.append([c[0] - w[0] / 2, c[1] - w[1] / 2, 0.0, c[0] + w[0] / 2, c[1] + w[1] / 2, h])
    return Scene(planes, ext, np.array(boxes, np.float64).reshape(-1, 6), np.zeros((0, 5)))


def corridor_forest(seed=0, half=60.0, n_cyl=400):
    """Ground plane, parallel corridor walls (thin boxes with doorway gaps),
    and vertical tree trunks of radius 0.1-0.4 m scattered between them."""
    rng = np.random.default_rng(seed)
    planes = np.array([[0, 0, 1, 0.0]], dtype=np.float64)
    ext = np.array([[-half, -half, 0, half, half, 0]], dtype=np.float64)
    boxes = []
    # corridor walls along x at these y offsets, broken by gaps every ~12 m
    for y in (-36.0, -30.0, 24.0, 30.0):
        x = -half
        while x < half:
            L = rng.uniform(6.0, 14.0)
            x1 = min(x + L, half)
            boxes.append([x, y - 0.1, 0.0, x1, y + 0.1, 3.0])
            x = x1 + rng.uniform(1.5, 3.0)
    for xw in (-42.0, 40.0):
        y = -20.0
        while y < 20.0:
            L = rng.uniform(5.0, 10.0)
            y1 = min(y + L, 20.0)
            boxes.append([xw - 0.1, y, 0.0, xw + 0.1, y1, 3.0])
            y = y1 + rng.uniform(1.5, 3.0)
    boxes = np.array(boxes, np.float64)
    cyl = []
    while len(cyl) < n_cyl:
        cx, cy = rng.uniform(-half, half, size=2)
        r = rng.uniform(0.1, 0.4)
        # keep trunks off the walls and off the central loop (|p| in 3..9 m band is clear)
        if np.any((cx > boxes[:, 0] - r - 0.3) & (cx < boxes[:, 3] + r + 0.3)
                  & (cy > boxes[:, 1] - r - 0.3) & (cy < boxes[:, 4] + r + 0.3)):
            continue
        if 3.5 < math.hypot(cx, cy) < 8.5:
            continue
        cyl.append([cx, cy, r, 0.0, rng.uniform(4.0, 8.0)])
    return Scene(planes, ext, boxes, np.array(cyl, np.float64))


def sample_surfaces(scene, spacing, noise, rng):
    """Points on the planes' sampling rectangles and on box faces, on a grid of
    the given spacing, each displaced by isotropic Gaussian noise."""
    pts = []

    def rect(lo, hi):
        lo = np.asarray(lo, np.float64)
        hi = np.asarray(hi, np.float64)
        axes = [np.arange(lo[a], hi[a] + 1e-9, spacing) if hi[a] > lo[a] else np.array([lo[a]])
                for a in range(3)]
        g = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
        pts.append(g)

    for e in scene.plane_extent:
        rect(e[:3], e[3:])
    for b in scene.boxes:
        lo, hi = b[:3], b[3:]
        for a in range(3):
            for side in (lo[a], hi[a]):
                l2, h2 = lo.copy(), hi.copy()
                l2[a] = h2[a] = side
                rect(l2, h2)
    P = np.concatenate(pts, 0)
    P = P + rng.normal(0.0, noise, size=P.shape)
    return P


def lidar_dirs(n_beams, n_az, elev_min_deg, elev_max_deg):
    """Unit ray directions of a spinning lidar in its own frame, beam-major."""
    el = np.deg2rad(np.linspace(elev_min_deg, elev_max_deg, n_beams))
    az = np.linspace(0.0, 2 * np.pi, n_az, endpoint=False)
    E, A = np.meshgrid(el, az, indexing="ij")
    d = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1)
    return d.reshape(-1, 3)


def cast_scan(scene, pose, dirs, rng, n_out=None, range_noise=0.01, rmin=0.5, rmax=80.0):
    """Ray-cast a scan from `pose` and return points in the sensor frame
    (float32, n_out x 3). When n_out is given, rays are drawn uniformly without
    replacement from `dirs` until n_out returns in [rmin, rmax] are found."""
    T = np.asarray(pose, np.float64).reshape(3, 4)
    R, t = T[:, :3], T[:, 3]
    if n_out is None:
        idx = np.arange(dirs.shape[0])
    else:
        idx = rng.permutation(dirs.shape[0])
    out = []
    have = 0
    pos = 0
    while pos < len(idx):
        take = idx[pos: pos + (len(idx) if n_out is None else max(2 * (n_out - have), 256))]
        pos += len(take)
        d_s = dirs[take]
        d_w = d_s @ R.T
        r = scene.raycast(t[None, :], d_w, max_range=rmax)
        ok = np.isfinite(r) & (r >= rmin)
        r = r[ok] + rng.normal(0.0, range_noise, size=int(ok.sum()))
        out.append(d_s[ok] * r[:, None])
        have += int(ok.sum())
        if n_out is not None and have >= n_out:
            break
    P = np.concatenate(out, 0)
    if n_out is not None:
        if P.shape[0] < n_out:
            raise ValueError("scene returned too few lidar points")
        P = P[:n_out]
    return P.astype(np.float32)


def grid_for_points(pts, h, margin):
    """Lattice covering the points' bounding box plus `margin` metres on every
    side: origin on a multiple of h, vertex counts (nx, ny, nz)."""
    pts = np.asarray(pts, np.float64)
    lo = pts.min(0) - margin
    hi = pts.max(0) + margin
    i0 = np.floor(lo / h)
    i1 = np.ceil(hi / h)
    origin = i0 * h
    dims = (i1 - i0 + 1).astype(np.int64)
    return {"origin": origin.astype(np.float64), "h": float(h), "dims": tuple(int(v) for v in dims)}


# ----------------------------------------------------------------------------
# trajectories
# ----------------------------------------------------------------------------

def room_walk(seed, n, start=(0.0, 0.0, 1.5), step=0.4, bound=6.0):
    """Seeded random walk in the horizontal plane with small roll/pitch, yawing
    back toward the centre when it nears `bound`."""
    rng = np.random.default_rng(seed)
    yaw = rng.uniform(-np.pi, np.pi)
    p = np.array(start, np.float64)
    out = []
    for _ in range(n):
        rp = rng.normal(0.0, np.deg2rad(1.0), size=2)
        R = Rotation.from_euler("zyx", [yaw, rp[1], rp[0]]).as_matrix()
        out.append(pose_from_rt(R, p))
        yaw += rng.normal(0.0, np.deg2rad(10.0))
        if np.hypot(p[0], p[1]) > bound:
            yaw = math.atan2(-p[1], -p[0]) + rng.normal(0.0, 0.2)
        p = p + step * np.array([math.cos(yaw), math.sin(yaw), 0.0])
        p[2] = start[2] + rng.normal(0.0, 0.02)
    return np.stack(out)


def loop_walk(seed, n, radius=6.0, step=0.4, z=1.5, phase0=0.0):
    """Closed loop of the given radius travelled at `step` metres per frame,
    with seeded lateral wobble and small roll/pitch."""
    rng = np.random.default_rng(seed)
    out = []
    ang = phase0
    for _ in range(n):
        rr = radius + rng.normal(0.0, 0.1)
        p = np.array([rr * math.cos(ang), rr * math.sin(ang), z + rng.normal(0, 0.02)])
        yaw = ang + np.pi / 2 + rng.normal(0.0, np.deg2rad(2.0))
        rp = rng.normal(0.0, np.deg2rad(1.0), size=2)
        R = Rotation.from_euler("zyx", [yaw, rp[1], rp[0]]).as_matrix()
        out.append(pose_from_rt(R, p))
        ang += step / radius
    return np.stack(out)


# ----------------------------------------------------------------------------
# complete workloads
# ----------------------------------------------------------------------------

def _odometry(traj):
    """Relative motions dT_t = (T_{t-1})^-1 T_t of a trajectory."""
    return [pose_mul(pose_inv(traj[i - 1]), traj[i])[0] for i in range(1, len(traj))]


def box_room_workload(seed=0, n_particles=1024, n_frames=10, n_keyframes=4, h=0.25,
                      surface_spacing=0.05, kf_radius=10.0, init_trans=0.3, init_rot_deg=5.0,
                      motion_std=(0.02, np.deg2rad(0.5)), kf_pert=(0.0, 0.0), lidar=(16, 32)):
    """Plain tiny case: box room, 4 keyframe grids at 0.25 m built from surface
    samples (5 cm spacing, 1 cm noise), 512-point scans from a 16 x 32 lidar
    (lidar = (beams, azimuths) for other scan sizes; the room is closed, so every
    ray returns) with 1 cm range noise, particles spread N(0, 0.3 m / 5 deg)."""
    rng = np.random.default_rng(seed)
    scene = box_room(seed)
    world = sample_surfaces(scene, surface_spacing, 0.01, rng)
    traj = room_walk(seed + 1, n_keyframes + n_frames + 1)
    kf_poses = traj[:n_keyframes]
    frames = traj[n_keyframes:]
    dirs = lidar_dirs(lidar[0], lidar[1], -15.0, 15.0)
    keyframes = []
    for k in range(n_keyframes):
        Tk = kf_poses[k]
        near = world[np.linalg.norm(world[:, :2] - Tk[[3, 7]], axis=1) < kf_radius]
        local = pose_apply(pose_inv(Tk)[0], near).astype(np.float32)
        keyframes.append({"points": local, "pose": Tk, "grid": grid_for_points(local, h, 1.0)})
    scans = [cast_scan(scene, frames[i], dirs, rng) for i in range(1, len(frames))]
    odom = _odometry(frames)
    st, sr = motion_std
    cov = np.diag([sr ** 2] * 3 + [st ** 2] * 3)
    particles = perturb_poses(frames[0], n_particles, init_trans, np.deg2rad(init_rot_deg), rng)
    kf_particle_poses = [perturb_poses(kf_poses[k], n_particles, kf_pert[0], kf_pert[1], rng)
                         for k in range(n_keyframes)]
    return {"scene": scene, "truth": frames, "keyframes": keyframes, "scans": scans,
            "odometry": odom, "cov": cov, "particles": particles.astype(np.float32),
            "kf_particle_poses": [p.astype(np.float32) for p in kf_particle_poses],
            "h": h, "sigma": 0.2}


def forest_workload(seed=0, n_particles=100_000, n_points=2048, n_keyframes=20,
                    kf_points=8192, n_frames=100, h=0.2, init_trans=0.3, init_rot_deg=5.0,
                    kf_pert=(0.05, np.deg2rad(0.5)), motion_std=(0.02, np.deg2rad(0.3)),
                    step=0.4, radius=6.0):
    """Paper-scale session: corridors plus 400 trunks, a 64 x 1024 lidar
    (elevation -22.5..22.5 deg, 0.5-80 m, 1 cm range noise) subsampled to
    n_points, keyframes of kf_points each placed every 2 m around a closed
    loop, particles spread N(0, 0.3 m / 5 deg), per-particle keyframe poses
    perturbed N(0, 5 cm / 0.5 deg)."""
    rng = np.random.default_rng(seed)
    scene = corridor_forest(seed)
    dirs = lidar_dirs(64, 1024, -22.5, 22.5)
    kf_traj = loop_walk(seed + 1, n_keyframes, radius=radius, step=2.0 * np.pi * radius / n_keyframes)
    keyframes = []
    for k in range(n_keyframes):
        pts = cast_scan(scene, kf_traj[k], dirs, rng, n_out=kf_points)
        keyframes.append({"points": pts, "pose": kf_traj[k], "grid": grid_for_points(pts, h, 1.0)})
    frames = loop_walk(seed + 2, n_frames + 1, radius=radius, step=step, phase0=0.05)
    scans = [cast_scan(scene, frames[i], dirs, rng, n_out=n_points) for i in range(1, n_frames + 1)]
    odom = _odometry(frames)
    st, sr = motion_std
    cov = np.diag([sr ** 2] * 3 + [st ** 2] * 3)
    particles = perturb_poses(frames[0], n_particles, init_trans, np.deg2rad(init_rot_deg), rng)
    kf_particle_poses = [perturb_poses(kf_traj[k], n_particles, kf_pert[0], kf_pert[1], rng).astype(np.float32)
                         for k in range(n_keyframes)]
    return {"scene": scene, "truth": frames, "keyframes": keyframes, "scans": scans,
            "odometry": odom, "cov": cov, "particles": particles.astype(np.float32),
            "kf_particle_poses": kf_particle_poses, "h": h, "sigma": 0.2}


def serving_pool(seed=0, n_kf=300, kf_points=2048, n_scans=40, scan_points=8192, rmax=25.0, h=0.2, radius=6.0):
    """Shared material for many serving sessions: n_kf keyframe clouds placed
    around a loop in the corridor-and-trunk scene (ranges up to rmax), n_scans
    scans of scan_points along the same loop, and their odometry."""
    rng = np.random.default_rng(seed)
    scene = corridor_forest(seed)
    dirs = lidar_dirs(64, 1024, -22.5, 22.5)
    kf_traj = loop_walk(seed + 1, n_kf, radius=radius, step=2.0 * np.pi * radius / n_kf)
    keyframes = []
    for k in range(n_kf):
        pts = cast_scan(scene, kf_traj[k], dirs, rng, n_out=kf_points, rmax=rmax)
        keyframes.append({"points": pts, "pose": kf_traj[k], "grid": grid_for_points(pts, h, 1.0)})
    frames = loop_walk(seed + 2, n_scans + 1, radius=radius, step=0.4, phase0=0.05)
    scans = [cast_scan(scene, frames[i], dirs, rng, n_out=scan_points, rmax=rmax) for i in range(1, n_scans + 1)]
    return {"keyframes": keyframes, "truth": frames, "scans": scans, "odometry": _odometry(frames),
            "cov": np.diag([np.deg2rad(0.3) ** 2] * 3 + [0.02 ** 2] * 3), "h": h}


def serving_sessions(seed, n_sessions=32, p_range=(4096, 200_000), n_range=(1024, 8192), k_range=(10, 300),
                     n_frames=20, rate_hz=10.0):
    """Session specs: particle count, scan size and keyframe count drawn uniformly,
    Poisson frame arrivals (offsets in seconds from admission)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_sessions):
        arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_frames))
        out.append({"P": int(rng.integers(p_range[0], p_range[1] + 1)), "N": int(rng.integers(n_range[0], n_range[1] + 1)),
                    "K": int(rng.integers(k_range[0], k_range[1] + 1)), "arrivals": arrivals, "seed": 1000 + s,
                    "frame0": int(rng.integers(0, 8))})
    return out


def session_particles(pool, spec, init_trans=0.3, init_rot_deg=5.0):
    """Initial particles of a serving session around its first frame's true pose."""
    rng = np.random.default_rng(spec["seed"])
    return perturb_poses(pool["truth"][spec["frame0"]], spec["P"], init_trans, np.deg2rad(init_rot_deg),
                         rng).astype(np.float32)
