"""gmcs_resample_noalloc: systematic resampling for callers that cannot call
cudaMalloc (a memory manager owns the device budget, or a real-time loop cannot
take an allocation's device synchronisation). Its ancestors must equal those of
gmcs_resample, the context-based entry point, on two calls in a row (the
second smaller, so scratch left by the first must not leak into it)."""
import numpy as np
import pytest

import oracle


@pytest.mark.gpu
def test_noalloc_resample_matches_context_resample():
    import torch
    import paper_2504_18056_b300 as g
    assert torch.cuda.is_available()
    torch.cuda.init()
    f = g.Filter(g.NOALLOC_MAX_P, 1, 16)
    rng = np.random.default_rng(2024)
    for P, u in [(200_003, 0.6180339887), (70_001, 0.25)]:
        w = rng.random(P) ** 6
        w /= w.sum()
        w_d = torch.from_numpy(w).cuda()
        anc_ref = torch.zeros(P, dtype=torch.int32, device="cuda")
        f.resample(w_d, u, anc_ref)
        anc = torch.full((P,), -7, dtype=torch.int32, device="cuda")
        g.resample_noalloc(w_d, u, anc)
        torch.cuda.synchronize()
        got = anc.cpu().numpy()
        np.testing.assert_array_equal(got, anc_ref.cpu().numpy())
        np.testing.assert_array_equal(got, oracle.resample(w, u))
    f.close()


@pytest.mark.gpu
def test_noalloc_resample_rejects_oversize_and_host_buffers():
    import torch
    import paper_2504_18056_b300 as g
    torch.cuda.init()
    big = torch.full((g.NOALLOC_MAX_P + 1,), 1.0 / (g.NOALLOC_MAX_P + 1), dtype=torch.float64, device="cuda")
    anc = torch.zeros(g.NOALLOC_MAX_P + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GmcsError) as e:
        g.resample_noalloc(big, 0.5, anc)
    assert e.value.code == g.E_CAPACITY
    w_host = np.full(10, 0.1)
    with pytest.raises(g.GmcsError) as e:
        g.resample_noalloc(w_host, 0.5, torch.zeros(10, dtype=torch.int32, device="cuda"))
    assert e.value.code == g.E_INVALID
