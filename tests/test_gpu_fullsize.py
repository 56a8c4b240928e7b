"""Parity at the benchmark configurations' full sizes, in the launch
configuration the benchmark times, on sampled outputs the oracle computes
one group at a time.

* two Plummer spheres of 2^23 bodies each (N = 2^24, theta 0.75, leaf 16,
  eps 5e-4, precise mode): Morton order, keys, root cube, the whole node
  table (level, prefix, first, count, children) and the groups bit-exact,
  moments within FP64 rounding; list lengths of the sampled bodies' groups
  bit-exact (unflagged), forces within 2e-5 relative (well-conditioned)
  against the oracle's FP64 walk;
* 512 Plummer systems with N log-uniform in [1024, 65536] (theta 0.6, leaf
  8, eps 0.01, gmax 64): five sampled systems checked whole against the
  oracle run on that system alone.
"""
import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs
from tests.test_gpu_parity import _check_forces, _compare_tree, _dev

pytestmark = pytest.mark.gpu


def test_precision_workload_full_size_sampled(tc):
    n = 1 << 24
    p, _, m = inputs.two_plummer(n, seed=0)
    ctx = tc.Context(precise=1, want_pot=0, verify=1)
    ctx.build(_dev(p), _dev(m), 16)
    ctx.forces(0.75, 5e-4)
    acc = ctx.get_acc()
    L = ctx.lists()
    gmax = ctx.config()["gmax"]
    t = oracle.Tree(p, m, 16, gmax)
    _compare_tree(ctx, t, gmax)
    sample = inputs.sample_indices(n, 48, seed=5)
    inv = np.empty(n, np.int64)
    inv[t.perm] = np.arange(n)
    groups = np.unique(np.searchsorted(t.gfirst, inv[sample], side="right") - 1)
    checked = 0
    for g in groups:
        w = t.walk(0.75, 5e-4, groups=(int(g), int(g) + 1), want_pot=False)
        if w["flag"][g]:
            continue
        assert L["ncell"][g] == w["ncell"][g] and L["nbody"][g] == w["nbody"][g]
        assert L["hash"][g] == w["hash"][g]
        mask = np.zeros(n, bool)
        mask[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
        _check_forces(acc, None, w, t, mask)
        checked += 1
    assert checked >= 0.9 * len(groups)


def test_batch_workload_full_size_sampled(tc):
    sizes = inputs.batch_sizes(512, seed=0)
    parts = [inputs.plummer(int(k), seed=s) for s, k in enumerate(sizes)]
    pos = np.concatenate([q for q, _, _ in parts])
    mass = np.concatenate([q for _, _, q in parts])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ctx = tc.Context(gmax=64, verify=1, want_pot=0)
    ctx.build_batch(_dev(pos), _dev(mass), off, 8)
    ctx.forces(0.6, 0.01)
    acc = ctx.get_acc()
    L = ctx.lists()
    tr = ctx.tree()
    nsys, cubes = ctx.systems()
    assert nsys == 512 and ctx.sizes()[0] == int(off[-1])
    for s in (0, 77, 255, 400, 511):
        a, b = int(off[s]), int(off[s + 1])
        t = oracle.Tree(pos[a:b], mass[a:b], 8, 64)
        w = t.walk(0.6, 0.01, want_pot=False)
        assert np.array_equal(cubes[s], t.cube5)
        assert np.array_equal(tr["perm"][a:b].astype(np.int64) - a, t.perm.astype(np.int64))
        gs = np.where((tr["gfirst"] >= a) & (tr["gfirst"] < b))[0]
        assert np.array_equal(tr["gcount"][gs], t.gcount)
        ok = w["flag"] == 0
        assert np.array_equal(L["ncell"][gs][ok], w["ncell"][ok])
        assert np.array_equal(L["nbody"][gs][ok], w["nbody"][ok])
        body_ok = np.zeros(b - a, bool)
        for g in np.where(ok)[0]:
            body_ok[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
        _check_forces(acc[a:b], None, w, t, body_ok)


def test_learned_workload_full_size_sampled(tc):
    """2^22-body Plummer sphere (the learned workload's evaluation system),
    theta 0.9, band 0.5, a seeded network: the correction of every body of
    sampled groups against the band sum of the network's BF16 rounding
    model, within its radius (as at small size)."""
    from tests.test_gpu_mlp import _p64, _random_params

    n = 1 << 22
    p, _, m = inputs.plummer(n, seed=101)
    ctx = tc.Context(precise=1, quad=1, want_pot=0, verify=1, split=0)
    ctx.build(_dev(p), _dev(m), 16)
    X, T, _, _, _ = ctx.mlp_pairs(0.9, 1e-3, 0.5, 0.01, 3, 200000)
    mean, sd = X.mean(0), X.std(0)
    scale = np.where(sd > 0, 1 / np.maximum(sd, 1e-30), 0).astype(np.float32)
    yscale = np.sqrt(np.mean(T.astype(np.float64) ** 2, 0)).astype(np.float32)
    params = _random_params(17)
    maps = np.concatenate([mean, scale, yscale]).astype(np.float32)
    ctx.forces(0.9, 1e-3)
    a0 = ctx.get_acc().astype(np.float64)
    ctx.mlp_set(np.concatenate([params, maps]), 0.5)
    ctx.set_config(learned=1)
    ctx.forces(0.9, 1e-3)
    a1 = ctx.get_acc().astype(np.float64)
    t = oracle.Tree(p, m, 16, 64)
    sample = inputs.sample_indices(n, 64, seed=6)
    inv = np.empty(n, np.int64)
    inv[t.perm] = np.arange(n)
    groups = np.unique(np.searchsorted(t.gfirst, inv[sample], side="right") - 1)
    d_all, c_all, b_all = [], [], []
    for g in groups:
        corr, crad, flag, _ = t.learned_bf16(0.9, 1e-3, 0.5, _p64(params), maps, groups=(int(g), int(g) + 1))
        if flag[g]:
            continue
        idx = t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]
        d_all.append((a1 - a0)[idx])
        c_all.append(corr[idx])
        b_all.append(crad[idx] + 2.0 ** -24 * (np.abs(a1[idx]) + np.abs(a0[idx])))
    d = np.concatenate(d_all)
    c = np.concatenate(c_all)
    bound = np.concatenate(b_all)
    assert len(d_all) >= 0.9 * len(groups)
    assert np.all(np.abs(d - c) <= bound), (np.abs(d - c) / bound).max()
    print(f"2^22 band sum: {len(d_all)} groups, max |err| {np.abs(d - c).max():.3e}, "
          f"median bound {np.median(bound):.3e}, corr rms {np.sqrt(np.mean(c ** 2)):.3e}")
