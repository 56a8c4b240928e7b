"""Quadrupole walk on the GPU against the oracle's quadrupole walk.

Same lists as the monopole walk (bit-exact for unflagged groups); forces and
potentials with every accepted cell's quadrupole term, at the monopole
walk's bar: 2e-5 relative for bodies whose sum is not dominated by
cancellation, and every body within 2e-5 |a| + 64 u sum |terms| (the
quadrupole term takes about three times the float operations of a
monopole term).  The quadrupole walk must also be markedly more accurate
against the direct sum than the monopole walk at the same theta.
"""
import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _bodies(kind, n, seed):
    if kind == "plummer":
        p, _, m = inputs.plummer(n, seed)
    elif kind == "uniform":
        p, _, m = inputs.uniform_cube(n, seed)
    else:
        rng = np.random.default_rng(seed)
        p = rng.standard_normal((n, 3)).astype(np.float32)
        m = rng.uniform(0.5, 1.5, n).astype(np.float32)
    return p, m


@pytest.mark.parametrize("kind,n,leaf,gmax,theta,eps,pot,tile", [
    ("plummer", 4096, 8, 64, 0.5, 0.01, 1, 128),
    ("plummer", 4096, 8, 32, 0.8, 0.01, 0, 64),
    ("plummer", 4096, 8, 128, 0.9, 0.01, 1, 256),
    ("uniform", 20000, 16, 64, 0.7, 1e-3, 0, 128),
    ("random", 777, 1, 32, 0.6, 0.05, 1, 128),
    ("random", 3, 1, 32, 0.5, 0.1, 1, 64),
])
def test_quadrupole_walk_matches_oracle(tc, kind, n, leaf, gmax, theta, eps, pot, tile):
    p, m = _bodies(kind, n, 11)
    ctx = tc.Context(gmax=gmax, precise=1, quad=1, quadrupole=1, want_pot=pot, verify=1, tile=tile)
    ctx.build(p, m, leaf)
    G = 0.9
    ctx.forces(theta, eps, G)
    acc, gpot = ctx.get_acc(with_pot=True) if pot else (ctx.get_acc(), None)
    L = ctx.lists()
    t = oracle.Tree(p, m, leaf, gmax)
    w = t.walk(theta, eps, G, want_pot=bool(pot), quadrupole=True)
    ok = w["flag"] == 0
    assert ok.mean() > 0.9
    assert np.array_equal(L["ncell"][ok], w["ncell"][ok])
    assert np.array_equal(L["nbody"][ok], w["nbody"][ok])
    assert np.array_equal(L["hash"][ok], w["hash"][ok])
    assert L["cells"] == int(np.sum(t.gcount * L["ncell"]))
    assert L["bodies"] == int(np.sum(t.gcount * L["nbody"]))
    assert L["interactions"] == L["cells"] + L["bodies"]
    body = np.zeros(n, bool)
    for g in np.where(ok)[0]:
        body[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
    a_or = w["acc"][body]
    err = np.linalg.norm(acc[body].astype(np.float64) - a_or, axis=1)
    amp = np.linalg.norm(a_or, axis=1)
    amag = w["amag"][body]
    assert np.all(err <= 2e-5 * amp + 64 * U32 * amag), (err / amp).max()
    well = amag <= 50 * amp
    assert (err[well] / amp[well]).max() <= 2e-5
    if pot:
        p_or = w["pot"][body]
        assert np.all(np.abs(gpot[body] - p_or) <= 2e-5 * np.abs(p_or))


def test_quadrupole_walk_is_more_accurate(tc):
    n = 32768
    p, m = _bodies("plummer", n, 12)
    idx = inputs.sample_indices(n, 1024, 13)
    ad, _ = oracle.direct(p, m, 1e-3, idx=idx, want_pot=False)
    errs = {}
    for q in (0, 1):
        ctx = tc.Context(precise=1, quad=1, quadrupole=q, want_pot=0)
        ctx.build(p, m, 16)
        ctx.forces(0.7, 1e-3)
        a = ctx.get_acc()[idx].astype(np.float64)
        errs[q] = np.sqrt(np.mean(np.sum((a - ad) ** 2, 1) / np.sum(ad ** 2, 1)))
    assert errs[1] < 0.5 * errs[0], errs


def test_quadrupole_config_is_validated(tc):
    with pytest.raises(tc.TcError):
        tc.Context(precise=0, quad=1, quadrupole=1)
    with pytest.raises(tc.TcError):
        tc.Context(precise=1, quad=0, quadrupole=1)
    with pytest.raises(tc.TcError):
        tc.Context(precise=1, quad=1, quadrupole=1, learned=1)
    # a graph-captured step with the quadrupole walk equals the eager one
    p, m = _bodies("plummer", 5000, 14)
    v = np.zeros_like(p)
    out = []
    for graph in (1, 0):
        ctx = tc.Context(precise=1, quad=1, quadrupole=1, graph=graph)
        ctx.build(p, m, 8)
        ctx.set_velocity(v)
        ctx.forces(0.6, 0.01)
        for _ in range(3):
            ctx.step(1e-3)
        out.append(ctx.get_state()[0])
    assert np.array_equal(out[0], out[1])
