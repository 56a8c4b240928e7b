"""tc_direct_static: direct summation for callers that cannot let the
library allocate device memory (a framework whose caching allocator owns the
device's memory budget, or a loop that cannot afford cudaMalloc's implicit
synchronisation).  Its results must match the allocating tc_direct within
the tolerance the direct-sum tests use, and the FP64 oracle's direct sum
within the float32 rounding bound of its terms, on calls in a row (each call
reuses the fixed scratch the previous one left behind).  An index outside
[0, n) gives a NaN row and leaves every other row correct."""
import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs

pytestmark = pytest.mark.gpu


def _abs_sum(p, m, idx, eps):
    """sum_j |a_ij| per target (FP64): the scale of the float32 rounding of
    the terms, which cancellation does not shrink"""
    p64, m64 = p.astype(np.float64), m.astype(np.float64)
    out = np.zeros(len(idx))
    for k0 in range(0, len(idx), 64):
        ii = idx[k0:k0 + 64]
        d = p64[None, :, :] - p64[ii][:, None, :]
        r2 = np.sum(d * d, axis=2) + eps * eps
        out[k0:k0 + 64] = np.sum(m64[None, :] * np.sqrt(r2 - eps * eps) / r2 ** 1.5, axis=1)
    return out


def test_static_direct_matches_allocating_direct_and_oracle(tc):
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
        or_acc, or_pot = oracle.direct(p, m, eps, G, idx=idx)
        amag = G * _abs_sum(p, m, idx, eps)
        I = torch.from_numpy(idx).cuda()
        acc = torch.full((idx.shape[0], 3), float("nan"), dtype=torch.float64, device="cuda")
        pot = torch.full((idx.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        tc.tc_direct_static(P, M, I, eps, G, acc, pot)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        ph = pot.cpu().numpy()
        # against the allocating entry point (same arithmetic, other slicing)
        assert np.all(np.linalg.norm(a - ref_acc, axis=1) <= 1e-5 * np.linalg.norm(ref_acc, axis=1)), call
        assert np.all(np.abs(ph - ref_pot) <= 1e-6 * np.abs(ref_pot)), call
        # against the FP64 oracle: float32 terms (a few ulps each, summed in
        # float32 over 256-source tiles) bound the error by 1e-5 |a| plus
        # 32 ulps of sum_j |a_ij|; the potential's terms all have one sign
        err = np.linalg.norm(a - or_acc, axis=1)
        assert np.all(err <= 1e-5 * np.linalg.norm(or_acc, axis=1) + 32 * 2.0 ** -24 * amag), call
        assert np.all(np.abs(ph - or_pot) <= 4e-6 * np.abs(or_pot)), call


def test_static_direct_nan_rows_for_invalid_indices_and_no_potential(tc):
    import torch

    n, eps, G = 5000, 0.01, 1.0
    p, _, m = inputs.plummer(n, 13)
    P = torch.from_numpy(p).cuda()
    M = torch.from_numpy(m).cuda()
    idx = inputs.sample_indices(n, 600, seed=5).copy()
    bad = np.array([0, 17, 599])
    idx[bad[0]], idx[bad[1]], idx[bad[2]] = -1, n, n + 12345
    good = np.setdiff1d(np.arange(idx.shape[0]), bad)
    or_acc, _ = oracle.direct(p, m, eps, G, idx=idx[good], want_pot=False)
    amag = G * _abs_sum(p, m, idx[good], eps)
    I = torch.from_numpy(idx).cuda()
    for call in range(2):
        acc = torch.zeros((idx.shape[0], 3), dtype=torch.float64, device="cuda")
        tc.tc_direct_static(P, M, I, eps, G, acc, None)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        assert np.all(np.isnan(a[bad])), call
        assert np.all(np.isfinite(a[good])), call
        err = np.linalg.norm(a[good] - or_acc, axis=1)
        assert np.all(err <= 1e-5 * np.linalg.norm(or_acc, axis=1) + 32 * 2.0 ** -24 * amag), call


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
    # host pageable memory, handed to the C ABI directly (the binding would
    # refuse a CPU tensor before the call)
    lib = tc.load()
    idx_h = np.zeros(4, np.int64)
    acc4 = torch.empty((4, 3), dtype=torch.float64, device="cuda")
    rc = lib.tc_direct_static(tc._ptr(P), tc._ptr(M), n, tc._ptr(idx_h), 4, 0.01, 1.0, tc._ptr(acc4), None, None)
    assert rc == tc.TC_EINVAL
