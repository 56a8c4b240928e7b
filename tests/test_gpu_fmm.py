"""GPU fast multipole method (tc_ctx_fmm) vs the oracle's FMM (a reading of
Sec. 5: monopoles at centres of mass, third-order local expansions, pair
acceptance r_A + r_B < theta |c_A - c_B| with r_X the cell's radius about its
centre of mass, dual traversal, M2L / L2L / L2P, P2P), through the C ABI.

Pairs, exactly: per target cell, the M2L and P2P pair counts and pair-set
hashes equal the oracle's for every cell whose walk, or an ancestor's, met
no pair within 1e-6 (relative) of the acceptance bound.  The GPU decides in
FP32 on cell-relative values, whose rounding moves the test by a few 1e-7
relative at most (see tc_fmm.cu), so outside those flagged cells the
decisions must agree; inside, either decision is right.

Forces, element-wise, for bodies of unflagged leaves: the oracle sums the
same terms in FP64; the GPU's FP32 terms and sums each round by at most a
few u = 2^-24 of the magnitudes involved, and every magnitude along the way
(an M2L term or its shift through at most ~20 levels of L2L, a P2P term, a
leaf's tile slices added at the end) is at most a small multiple of the pair
fields it stands for, so
|a_gpu - a_oracle| <= 64 u G A_i, A_i = sum_j m_j r_ij / (r_ij^2 + eps^2)^1.5.
Flagged bodies: the two results are both FMM values and differ by the
truncation error of the flipped pairs, a small fraction of |a|.
"""
import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs
from tests.helpers import abs_field, rel_err_rms

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _run(tc, p, m, leaf, theta, eps, G):
    ctx = tc.Context(verify=1)
    ctx.build(_dev(p), _dev(m), leaf)
    ctx.fmm(theta, eps, G)
    return ctx, ctx.get_acc().astype(np.float64)


def _compare(tc, p, m, leaf, theta, eps, G, tag):
    theta = float(np.float32(theta))
    ctx, a = _run(tc, p, m, leaf, theta, eps, G)
    t = oracle.Tree(p, m, leaf)
    a_or, st = t.fmm(theta, eps, G, per_node=True)
    n, M, _ = ctx.sizes()
    assert M == t.M
    g = ctx.fmm_pairs()
    tot = ctx.fmm_stats()
    assert tot["m2l"] == int(g["nm2l"].sum()) and tot["p2p"] == int(g["np2p"].sum())
    ok = st["flag"] == 0
    for k in ("nm2l", "np2p", "hm2l", "hp2p"):
        assert np.array_equal(g[k][ok], st[k][ok]), (tag, k, int(np.sum(g[k][ok] != st[k][ok])))
    if st["ties"] == 0:
        assert tot["m2l"] == st["m2l"] and tot["p2p"] == st["p2p"]
        assert tot["m2l_hash"] == st["m2l_hash"] and tot["p2p_hash"] == st["p2p_hash"]
    # bodies of unflagged leaves
    body_ok = np.zeros(n, bool)
    leaves = np.where((t.nchild == 0) & ok)[0]
    for v in leaves:
        body_ok[t.perm[t.first[v]:t.first[v] + t.count[v]]] = True
    A = G * abs_field(p, m, np.arange(n), eps)
    err = np.linalg.norm(a - a_or, axis=1)
    ratio = err / (64 * U32 * A)
    assert np.all(ratio[body_ok] <= 1.0), (tag, float(ratio[body_ok].max()))
    if (~body_ok).any():
        rel = err[~body_ok] / np.linalg.norm(a_or[~body_ok], axis=1)
        assert rel.max() <= 2e-2, (tag, float(rel.max()))
    assert body_ok.mean() >= 0.5, tag
    return ctx, a, a_or, st, float(ratio[body_ok].max())


@pytest.mark.parametrize("theta", [0.35, 0.6, 1.0])
def test_fmm_plummer_matches_oracle(tc, theta):
    p, _, m = inputs.plummer(20000, 21)
    _compare(tc, p, m, 16, theta, 0.01, 1.3, f"plummer {theta}")


def test_fmm_uniform_matches_oracle(tc):
    p, _, m = inputs.uniform_cube(30000, 22)
    _compare(tc, p, m, 8, 0.5, 0.02, 1.0, "uniform")


def test_fmm_leaves_above_a_warp(tc):
    # leaves of up to 100 bodies: a leaf's bodies are taken 32 at a time
    p, _, m = inputs.plummer(20000, 23)
    _compare(tc, p, m, 100, 0.6, 0.01, 1.0, "leaf 100")


def test_fmm_theta_zero_is_the_direct_sum(tc):
    p, _, m = inputs.plummer(4000, 24)
    ctx, a, a_or, st, _ = _compare(tc, p, m, 8, 0.0, 0.01, 1.0, "theta 0")
    assert ctx.fmm_stats()["m2l"] == 0 and st["m2l"] == 0
    ad, _ = oracle.direct(p, m, 0.01, 1.0, want_pot=False)
    assert np.all(np.linalg.norm(a - ad, axis=1) <= 64 * U32 * abs_field(p, m, np.arange(4000), 0.01))


def test_fmm_single_leaf_and_two_bodies(tc):
    # a root that is a leaf: every pair is its self P2P
    p, _, m = inputs.plummer(20, 25)
    ctx, a, a_or, st, _ = _compare(tc, p, m, 32, 0.5, 0.01, 1.0, "one leaf")
    assert ctx.fmm_stats()["p2p"] == 1 and ctx.fmm_stats()["m2l"] == 0
    # two far bodies: two M2L pairs and two (bodiless) self P2Ps, exact
    p2 = np.array([[-0.9, -0.8, -0.85], [0.9, 0.8, 0.95]], np.float32)
    m2 = np.array([0.3, 1.7], np.float32)
    ctx, a, a_or, st, _ = _compare(tc, p2, m2, 1, 1.5, 1e-3, 1.0, "two bodies")
    assert ctx.fmm_stats()["m2l"] == 2 and ctx.fmm_stats()["p2p"] == 2


def test_fmm_is_deterministic_and_repeatable(tc):
    p, _, m = inputs.plummer(50000, 26)
    ctx = tc.Context(verify=1)
    ctx.build(_dev(p), _dev(m), 16)
    ctx.fmm(0.5, 0.01, 1.0)
    a1 = ctx.get_acc().copy()
    s1 = ctx.fmm_stats()
    ctx.fmm(0.5, 0.01, 1.0)
    assert np.array_equal(ctx.get_acc(), a1) and ctx.fmm_stats() == s1


def test_fmm_regrows_its_lists(tc, monkeypatch):
    # initial pool and slab far too small: every pass that overflows is
    # discarded and rerun with the counted sizes; the result is the same
    p, _, m = inputs.plummer(50000, 27)
    ctx = tc.Context(verify=1)
    ctx.build(_dev(p), _dev(m), 16)
    ctx.fmm(0.4, 0.01, 1.0)
    ref = ctx.get_acc().copy()
    ref_st = ctx.fmm_stats()
    monkeypatch.setenv("TC_FMM_POOL", "64")
    monkeypatch.setenv("TC_FMM_SLAB", "8")
    ctx2 = tc.Context(verify=1)
    ctx2.build(_dev(p), _dev(m), 16)
    ctx2.fmm(0.4, 0.01, 1.0)
    assert np.array_equal(ctx2.get_acc(), ref) and ctx2.fmm_stats() == ref_st


def test_fmm_batch_of_systems(tc):
    # independent systems in one forest: each equals its own FMM
    sizes = [3000, 12000, 700]
    parts = [inputs.plummer(k, 30 + i) for i, k in enumerate(sizes)]
    p = np.concatenate([q[0] for q in parts])
    m = np.concatenate([q[2] for q in parts])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ctx = tc.Context(verify=1)
    ctx.build_batch(_dev(p), _dev(m), off, 16)
    ctx.fmm(0.5, 0.01, 1.0)
    a = ctx.get_acc().astype(np.float64)
    m2l = p2p = 0
    for s, (ps, _, ms) in enumerate(parts):
        t = oracle.Tree(ps, ms, 16)
        a_or, st = t.fmm(float(np.float32(0.5)), 0.01, 1.0)
        m2l += st["m2l"]
        p2p += st["p2p"]
        sl = slice(off[s], off[s + 1])
        A = abs_field(ps, ms, np.arange(sizes[s]), 0.01)
        err = np.linalg.norm(a[sl] - a_or, axis=1)
        if st["ties"] == 0:
            assert np.all(err <= 64 * U32 * A), s
        else:
            assert rel_err_rms(a[sl], a_or) <= 1e-3, s
    tot = ctx.fmm_stats()
    assert abs(tot["m2l"] - m2l) <= 64 and abs(tot["p2p"] - p2p) <= 64


def test_fmm_step_refuses_fmm_forces_and_stats_need_fmm(tc):
    p, _, m = inputs.plummer(3000, 28)
    ctx = tc.Context()
    ctx.build(_dev(p), _dev(m), 16)
    ctx.forces(0.5, 0.01, 1.0)
    with pytest.raises(tc.TcError) as e:
        ctx.fmm_stats()
    assert e.value.code == tc.TC_ESTATE
    ctx.fmm(0.5, 0.01, 1.0)
    # counts without verify, records and hashes only with it; the counts
    # do not depend on it
    st = ctx.fmm_stats()
    assert st["m2l_hash"] is None and st["m2l"] > 0
    with pytest.raises(tc.TcError) as e:
        ctx.fmm_pairs()
    assert e.value.code == tc.TC_ESTATE
    ctx.set_config(verify=1)
    ctx.fmm(0.5, 0.01, 1.0)
    st1 = ctx.fmm_stats()
    assert (st1["m2l"], st1["p2p"]) == (st["m2l"], st["p2p"]) and st1["m2l_hash"] is not None
    with pytest.raises(tc.TcError) as e:
        ctx.step(1e-3)
    assert e.value.code == tc.TC_ESTATE
    with pytest.raises(tc.TcError) as e:
        ctx.fmm(-0.1, 0.01, 1.0)
    assert e.value.code == tc.TC_EINVAL


def test_fmm_full_size_every_pair_once(tc):
    # 2^20 uniform bodies, softening 1e4 >> the cube (side 2): every pair
    # field is linear in the positions to (3.5 / 1e4)^2 ~ 1e-7, where
    # monopoles and local expansions are exact, so the FMM equals the direct
    # sum (sampled) within the float32 bound unless a pair of bodies is
    # dropped or counted twice.
    n, eps = 1 << 20, 1e4
    p, _, m = inputs.uniform_cube(n, 29)
    ctx = tc.Context()
    ctx.build(_dev(p), _dev(m), 16)
    ctx.fmm(0.5, eps, 1.0)
    a = ctx.get_acc().astype(np.float64)
    idx = inputs.sample_indices(n, 256, seed=29)
    ad, _ = oracle.direct(p, m, eps, 1.0, idx=idx, want_pot=False)
    A = abs_field(p, m, idx, eps, rows=4)
    err = np.linalg.norm(a[idx] - ad, axis=1)
    assert np.all(err <= 64 * U32 * A + 1e-6 * A)


def test_fmm_full_size_accuracy(tc):
    # 2^20 Plummer bodies at theta 0.25: the method's own error against the
    # direct sum (sampled), near the treecode's 1e-3 target
    n = 1 << 20
    p, _, m = inputs.plummer(n, 31)
    ctx = tc.Context()
    ctx.build(_dev(p), _dev(m), 16)
    ctx.fmm(0.25, 0.01, 1.0)
    a = ctx.get_acc().astype(np.float64)
    idx = inputs.sample_indices(n, 512, seed=31)
    ad, _ = oracle.direct(p, m, 0.01, 1.0, idx=idx, want_pot=False)
    assert rel_err_rms(a[idx], ad) <= 2e-3
