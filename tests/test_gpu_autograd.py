"""The scan log-likelihood as a torch.autograd.Function (hand-written CUDA
backward): P = 100,000 poses x N = 4,096 points against 50 keyframe lattices
at 0.2 m, FP32 forward and backward, checked against the FP64 oracle's
gradient through the SE(3) right Jacobian on 1,024 sampled particles and
against central differences with step 1e-4."""
import json

import numpy as np
import pytest

import oracle
import synth
from gpu_common import make_filter, torch_cuda

pytestmark = pytest.mark.gpu

P, N, K = 100_000, 4096, 50


@pytest.fixture(scope="module")
def setup():
    torch = torch_cuda()
    w = synth.forest_workload(seed=3, n_particles=P, n_points=N, n_keyframes=K, n_frames=1)
    f = make_filter(w, P, max_points=N)
    nbr = np.zeros((P, 3), np.int32)
    f.select(nbr)
    rng = np.random.default_rng(5)
    xi = np.concatenate([rng.normal(0, 0.01, (P, 3)), rng.normal(0, 0.03, (P, 3))], 1).astype(np.float32)
    xi[:64] = 0.0                      # the identity perturbation: Jr = I
    scan_d = torch.from_numpy(w["scans"][0]).cuda()
    return torch, w, f, nbr, xi, scan_d


def test_forward_backward_match_oracle(setup):
    torch, w, f, nbr, xi, scan_d = setup
    from paper_2504_18056_b300.autograd import scan_loglik
    xi_d = torch.from_numpy(xi).cuda().requires_grad_(True)
    wts = torch.rand(P, device="cuda") + 0.5
    ll = scan_loglik(xi_d, f, scan_d)
    (ll * wts).sum().backward()
    ll_h = ll.detach().cpu().numpy()
    grad = (xi_d.grad / wts[:, None]).cpu().numpy()
    rng = np.random.default_rng(6)
    idx = np.unique(np.concatenate([np.arange(8), rng.choice(P, 1024 - 8, replace=False)]))
    need = sorted(set(int(k) for k in nbr[idx].ravel()))
    tabs = {k: oracle.build_table(w["keyframes"][k]["points"], w["keyframes"][k]["grid"], 0.2, 1.0) for k in need}
    grids = [kf["grid"] for kf in w["keyframes"]]
    rel_ll, err_g, tol_g = [], [], []
    for i in idx:
        ks = [int(k) for k in nbr[i]]
        o = oracle.loglik_grad_xi(w["particles"][i].astype(np.float64), xi[i].astype(np.float64),
                                  [w["kf_particle_poses"][k][i] for k in ks], [tabs[k] for k in ks],
                                  [grids[k] for k in ks], w["scans"][0])
        rel_ll.append(abs(ll_h[i] - o["ll"]) / abs(o["ll"]))
        err_g.append(np.linalg.norm(grad[i] - o["g_xi"]))
        tol_g.append(1e-3 * max(np.linalg.norm(o["g_xi"]), 1e-2 * o["gabs"] * o["jr_norm"]) + o["slack"] * o["jr_norm"])
    rel_ll, err_g, tol_g = map(np.array, (rel_ll, err_g, tol_g))
    print("\nAUTOGRAD_PARITY " + json.dumps({"ll_rel_max": float(rel_ll.max()), "grad_err_over_tol_max": float((err_g / tol_g).max()),
                                            "grad_err_over_tol_median": float(np.median(err_g / tol_g))}))
    assert rel_ll.max() <= 1e-4
    assert np.all(err_g <= tol_g)


def test_backward_matches_central_differences(setup):
    """Central differences of the CUDA forward (step 1e-4) on 256 particles and
    all 6 directions, against the CUDA backward; the FP64 oracle's central
    differences at the same step (the same cell-face crossings) bound what the
    trilinear field's kinks contribute."""
    torch, w, f, nbr, xi, scan_d = setup
    from paper_2504_18056_b300.autograd import scan_loglik
    h = 1e-4
    xi_d = torch.from_numpy(xi).cuda().requires_grad_(True)
    ll = scan_loglik(xi_d, f, scan_d)
    ll.sum().backward()
    grad = xi_d.grad.cpu().numpy()
    idx = np.arange(0, P, P // 256)[:256]
    fd = np.zeros((len(idx), 6))
    base = torch.from_numpy(xi).cuda()
    with torch.no_grad():
        for d in range(6):
            e = torch.zeros(P, 6, device="cuda")
            e[:, d] = h
            lp = scan_loglik(base + e, f, scan_d).double().cpu().numpy()
            lm = scan_loglik(base - e, f, scan_d).double().cpu().numpy()
            fd[:, d] = ((lp - lm) / (2 * h))[idx]
    need = sorted(set(int(k) for k in nbr[idx[:32]].ravel()))
    tabs = {k: oracle.build_table(w["keyframes"][k]["points"], w["keyframes"][k]["grid"], 0.2, 1.0) for k in need}
    grids = [kf["grid"] for kf in w["keyframes"]]
    kink, noise = [], []
    for r, i in enumerate(idx[:32]):
        ks = [int(k) for k in nbr[i]]
        args = ([w["kf_particle_poses"][k][i] for k in ks], [tabs[k] for k in ks], [grids[k] for k in ks], w["scans"][0])
        T0 = w["particles"][i].astype(np.float64)
        x0 = xi[i].astype(np.float64)
        o = oracle.loglik_grad_xi(T0, x0, *args)
        for d in range(6):
            e = np.zeros(6)
            e[d] = h
            lp = oracle.loglik_grad_xi(T0, x0 + e, *args)["ll"]
            lm = oracle.loglik_grad_xi(T0, x0 - e, *args)["ll"]
            fd64 = (lp - lm) / (2 * h)
            kink.append(abs(fd64 - o["g_xi"][d]))           # field kinks within +-h
            noise.append(abs(fd[r, d] - fd64))               # float32 forward noise
    scale = np.maximum(np.abs(grad[idx]), 1e-2 * np.abs(grad[idx]).max(axis=1, keepdims=True))
    rel = np.abs(fd - grad[idx]) / scale
    stats = {"fd_rel_median": float(np.median(rel)), "fd_rel_p90": float(np.percentile(rel, 90)),
             "oracle_fd_kink_median": float(np.median(kink)), "gpu_fd_noise_median": float(np.median(noise)),
             "grad_abs_median": float(np.median(np.abs(grad[idx])))}
    print("\nAUTOGRAD_FD " + json.dumps(stats))
    assert np.median(rel) <= 2e-2
    assert np.percentile(rel, 90) <= 0.15


def test_forward_backward_timing(setup):
    """Device time of the autograd forward (value pass at T0 exp(xi)) and
    backward (gradient pass plus the right-Jacobian chain) at the full size,
    CUDA events after warm-up; reported, with a loose sanity bound only."""
    torch, w, f, nbr, xi, scan_d = setup
    from paper_2504_18056_b300.autograd import scan_loglik
    xi_d = torch.from_numpy(xi).cuda().requires_grad_(True)
    for _ in range(3):
        scan_loglik(xi_d, f, scan_d).sum().backward()
    reps = 10
    fwd, bwd = [], []
    for _ in range(reps):
        xi_d.grad = None
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        ll = scan_loglik(xi_d, f, scan_d)
        e1.record()
        ll.sum().backward()
        e2.record()
        torch.cuda.synchronize()
        fwd.append(e0.elapsed_time(e1))
        bwd.append(e1.elapsed_time(e2))
    lookups = P * N * 3
    t = {"forward_ms": float(np.median(fwd)), "backward_ms": float(np.median(bwd)),
         "forward_lookups_per_s": lookups / (np.median(fwd) * 1e-3),
         "backward_lookups_per_s": lookups / (np.median(bwd) * 1e-3)}
    print("\nAUTOGRAD_TIMING " + json.dumps(t))
    assert 0 < t["forward_ms"] < 1e3 and 0 < t["backward_ms"] < 1e3


def test_backward_refuses_a_changed_filter(box_room):
    """The backward re-reads the base poses and neighbours from the filter: a
    call that changed them after the forward (a new selection, a step) makes it
    raise instead of returning the gradient of another function."""
    torch = torch_cuda()
    from paper_2504_18056_b300.autograd import scan_loglik
    P = 256
    f = make_filter(box_room, P, max_points=1024)
    f.select()
    scan_d = torch.from_numpy(box_room["scans"][0]).cuda()
    xi = torch.zeros((P, 6), dtype=torch.float32, device="cuda", requires_grad=True)
    scan_loglik(xi, f, scan_d).sum().backward()          # unchanged filter: fine
    assert xi.grad is not None and torch.isfinite(xi.grad).all()
    for change in (lambda: f.select(), lambda: f.step(box_room["scans"][0], box_room["odometry"][0], box_room["cov"])):
        xi.grad = None
        ll = scan_loglik(xi, f, scan_d)
        change()
        with pytest.raises(RuntimeError, match="changed since the forward"):
            ll.sum().backward()
    f.close()


def test_locality_order_leaves_results_unchanged(box_room):
    """The differentiable log-likelihood runs its passes with the particles in a
    locality order (Morton buckets of their translations); each particle is still
    computed from its own data in one lane, so at xi = 0 the forward equals the
    plain value pass bit for bit, and the backward's gradient the gradient pass's
    (the chain rule through Jr(0) = I), for a set spread wider than the lanes'
    cells."""
    torch = torch_cuda()
    from paper_2504_18056_b300.autograd import scan_loglik
    P = 3000
    w = synth.box_room_workload(seed=4, n_particles=P, n_frames=1, init_trans=1.0, init_rot_deg=10.0)
    f = make_filter(w, P, max_points=1024)
    f.select()
    scan = np.ascontiguousarray(w["scans"][0])
    ll_ref = np.zeros(P, np.float32)
    g_ref = np.zeros((P, 6), np.float32)
    f.eval(scan, ll_ref)                                   # value pass, identity order
    f.eval(scan, None, g_ref)                              # gradient pass, identity order
    xi = torch.zeros((P, 6), dtype=torch.float32, device="cuda", requires_grad=True)
    ll = scan_loglik(xi, f, torch.from_numpy(scan).cuda())
    ll.sum().backward()
    np.testing.assert_array_equal(ll.detach().cpu().numpy(), ll_ref)
    np.testing.assert_array_equal(xi.grad.cpu().numpy(), g_ref)
    f.close()
