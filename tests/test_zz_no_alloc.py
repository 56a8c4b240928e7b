"""tc_direct_static: direct summation for callers that cannot let the
library allocate device memory (a framework whose caching allocator owns the
device's memory budget, or a loop that cannot afford cudaMalloc's implicit
synchronisation).  Its results must match the allocating tc_direct within
the tolerance the direct-sum tests use, on two calls in a row (the second
call reuses the fixed scratch the first one left behind)."""
import numpy as np
import pytest

from paper_1211_2293_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_static_direct_matches_allocating_direct(tc):
    import torch

    n, ns, eps, G = 30000, 3000, 0.01, 1.5
    p, _, m = inputs.plummer(n, 11)
    P = torch.from_numpy(p).cuda()
    M = torch.from_numpy(m).cuda()
    ctx = tc.Context()
    ctx.build(P, M, 8)
    for call, seed in enumerate((3, 4)):
        idx = inputs.sample_indices(n, ns - 7 * call, seed=seed)
        ref_acc, ref_pot = ctx.direct(idx, eps, G)
        I = torch.from_numpy(idx).cuda()
        acc = torch.full((idx.shape[0], 3), float("nan"), dtype=torch.float64, device="cuda")
        pot = torch.full((idx.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        tc.tc_direct_static(P, M, I, eps, G, acc, pot)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        ph = pot.cpu().numpy()
        assert np.all(np.linalg.norm(a - ref_acc, axis=1) <= 1e-5 * np.linalg.norm(ref_acc, axis=1)), call
        assert np.all(np.abs(ph - ref_pot) <= 1e-6 * np.abs(ref_pot)), call


def test_static_direct_rejects_oversize_and_host_memory(tc):
    import torch

    n = 1000
    p, _, m = inputs.plummer(n, 12)
    P = torch.from_numpy(p).cuda()
    M = torch.from_numpy(m).cuda()
    idx = torch.zeros(8193, dtype=torch.int64, device="cuda")
    acc = torch.empty((8193, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.tc_direct_static(P, M, idx, 0.01, 1.0, acc)
    assert e.value.code == tc.TC_EINVAL and "8192" in str(e.value)
    idx_h = torch.zeros(4, dtype=torch.int64)
    with pytest.raises(tc.TcError) as e:
        tc.tc_direct_static(P, M, idx_h, 0.01, 1.0, acc)
    assert e.value.code == tc.TC_EINVAL
