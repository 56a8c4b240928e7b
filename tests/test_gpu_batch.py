"""Batches of independent systems (one forest, one walk launch, one step
graph) against the oracle run on each system alone; the captured step graph
against the same launches issued one by one; the device-side node-capacity
check; the launch-configuration autotuner."""
import os

import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs
from tests.test_gpu_parity import U32, _check_forces, _dev

pytestmark = pytest.mark.gpu


def _batch(sizes, seed0=0):
    parts = [inputs.plummer(k, seed=seed0 + s) for s, k in enumerate(sizes)]
    pos = np.concatenate([p for p, _, _ in parts])
    vel = np.concatenate([v for _, v, _ in parts])
    mass = np.concatenate([m for _, _, m in parts])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return pos, vel, mass, off


@pytest.mark.parametrize("gmax,theta", [(64, 0.6), (32, 0.5)])
def test_batch_matches_per_system_oracle(tc, gmax, theta):
    sizes = [1500, 37, 4096, 9, 2600, 1]
    pos, _, mass, off = _batch(sizes, 3)
    ctx = tc.Context(gmax=gmax, verify=1, want_pot=1, quad=1)
    ctx.build_batch(_dev(pos), _dev(mass), off, 8)
    ctx.forces(theta, 0.01)
    acc, pot = ctx.get_acc(with_pot=True)
    L = ctx.lists()
    tr = ctx.tree()
    nsys, cubes = ctx.systems()
    assert nsys == len(sizes)
    for s in range(nsys):
        a, b = off[s], off[s + 1]
        p, m = pos[a:b], mass[a:b]
        t = oracle.Tree(p, m, 8, gmax)
        w = t.walk(theta, 0.01)
        assert np.array_equal(cubes[s], t.cube5)
        assert np.array_equal(tr["perm"][a:b].astype(np.int64) - a, t.perm.astype(np.int64))
        assert np.array_equal(tr["keys"][a:b], t.keys)
        # this system's nodes, in the forest's breadth-first order
        mine = np.where((tr["first"] >= a) & (tr["first"] < b))[0]
        assert mine.size == t.M and tr["level"][mine[0]] == 0 and mine[0] == s
        local = {int(v): k for k, v in enumerate(mine)}
        assert np.array_equal(tr["level"][mine], t.level)
        assert np.array_equal(tr["first"][mine] - a, t.first)
        assert np.array_equal(tr["count"][mine], t.count)
        assert np.array_equal(tr["nchild"][mine], t.nchild)
        cf = np.array([local[int(v)] if v >= 0 else -1 for v in tr["child_first"][mine]])
        assert np.array_equal(cf, t.child_first)
        assert np.allclose(tr["mass"][mine], t.node_mass, rtol=1e-12, atol=0)
        gs = np.where((tr["gfirst"] >= a) & (tr["gfirst"] < b))[0]
        assert np.array_equal(tr["gfirst"][gs] - a, t.gfirst)
        assert np.array_equal(tr["gcount"][gs], t.gcount)
        ok = w["flag"] == 0
        assert np.array_equal(L["ncell"][gs][ok], w["ncell"][ok])
        assert np.array_equal(L["nbody"][gs][ok], w["nbody"][ok])
        body_ok = np.zeros(b - a, bool)
        for g in np.where(ok)[0]:
            body_ok[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
        if b - a > 1:
            _check_forces(acc[a:b], pot[a:b], w, t, body_ok)
        else:
            assert np.all(acc[a:b] == 0)
        # the direct-sum reference sums within the system only
        idx = np.arange(a, b, max(1, (b - a) // 50))
        ad, _ = ctx.direct(idx, 0.01)
        ao, _ = oracle.direct(p, m, 0.01, idx=idx - a)
        assert np.all(np.linalg.norm(ad - ao, axis=1) <= 1e-5 * np.linalg.norm(ao, axis=1) + 1e-30)


def test_graph_step_equals_eager_step(tc):
    sizes = [3000, 500, 7000]
    pos, vel, mass, off = _batch(sizes, 7)
    out = []
    for graph in (1, 0):
        ctx = tc.Context(graph=graph)
        ctx.build_batch(_dev(pos), _dev(mass), off, 8)
        ctx.set_velocity(_dev(vel))
        ctx.forces(0.6, 0.01)
        for _ in range(4):
            ctx.step(1e-3)
        out.append(ctx.get_state() + (ctx.get_acc(),))
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)


def test_batch_step_matches_single_systems(tc):
    """Stepping a batch equals stepping each system in a context of its own."""
    sizes = [2000, 800, 3000]
    pos, vel, mass, off = _batch(sizes, 11)
    ctx = tc.Context()
    ctx.build_batch(_dev(pos), _dev(mass), off, 8)
    ctx.set_velocity(_dev(vel))
    ctx.forces(0.6, 0.01)
    for _ in range(3):
        ctx.step(1e-3)
    xb, vb = ctx.get_state()
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        c1 = tc.Context()
        c1.build(_dev(pos[a:b]), _dev(mass[a:b]), 8)
        c1.set_velocity(_dev(vel[a:b]))
        c1.forces(0.6, 0.01)
        for _ in range(3):
            c1.step(1e-3)
        x1, v1 = c1.get_state()
        assert np.array_equal(x1, xb[a:b]) and np.array_equal(v1, vb[a:b])


def test_node_capacity_overflow_in_a_step_is_reported(tc):
    """Bodies sitting on two points give a tiny tree; a step that scatters
    them needs far more nodes than the table sized for it.  The device-side
    check stops the step (no kernel writes past the table) and the next
    synchronising call reports TC_EDEVICE; a new build recovers."""
    n = 20000
    pos = np.zeros((n, 3), np.float32)
    pos[n // 2:] = 1.0
    rng = np.random.default_rng(0)
    vel = rng.standard_normal((n, 3)).astype(np.float32)
    mass = np.full(n, 1.0 / n, np.float32)
    ctx = tc.Context()
    ctx.build(_dev(pos), _dev(mass), 8)
    ctx.set_velocity(_dev(vel))
    ctx.forces(0.5, 0.01)
    ctx.step(1.0)
    with pytest.raises(tc.TcError) as e:
        ctx.get_acc()
    assert e.value.code == tc.TC_EDEVICE and "capacity" in str(e.value)
    x, v = ctx.get_state()
    ctx.build(_dev(x), _dev(mass), 8)
    ctx.set_velocity(_dev(v))
    ctx.forces(0.5, 0.01)
    ctx.step(1e-3)
    ctx.get_acc()


def test_autotune_picks_a_valid_config_and_caches(tc, tmp_path, monkeypatch):
    p, _, m = inputs.plummer(20000, 2)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TC_AUTOTUNE_CACHE", str(cache))
    ctx = tc.Context()
    ctx.build(_dev(p), _dev(m), 8)
    best, ms = ctx.autotune(0.6, 0.01, reps=2)
    assert best["gmax"] in (32, 64, 128) and best["tile"] in (64, 128, 256) and best["warps"] in (2, 4)
    assert ms > 0 and cache.exists() and len(cache.read_text().splitlines()) == 1
    cfg = ctx.config()
    assert (cfg["gmax"], cfg["tile"], cfg["warps"]) == (best["gmax"], best["tile"], best["warps"])
    ctx2 = tc.Context()
    ctx2.build(_dev(p), _dev(m), 8)
    best2, ms2 = ctx2.autotune(0.6, 0.01, reps=2)
    assert (best2["gmax"], best2["tile"], best2["warps"]) == (best["gmax"], best["tile"], best["warps"])
    assert ms2 == pytest.approx(ms, rel=1e-5)
    assert len(cache.read_text().splitlines()) == 1
    ctx.forces(0.6, 0.01)
    ctx.get_acc()


def test_bounded_device_wait_gives_up_and_reports(tc):
    """Failure path without a GPU fault: a radix tile whose predecessor never
    publishes polls for a bounded time, sets its error bit (8) and returns;
    the device stays usable."""
    bits, ms = tc.selftest_bounded_wait()
    assert bits & 8
    assert 0 < ms < 20000
    # the device still works: a small build and force evaluation
    pos, _, mass, off = _batch([2000], 1)
    ctx = tc.Context()
    ctx.build(_dev(pos), _dev(mass), 8)
    ctx.forces(0.5, 0.01)
    assert np.all(np.isfinite(ctx.get_acc()))


def test_fp32_and_force_loop_probes(tc):
    """The FP32 probe reaches the derived CUDA-core peak (2 flops x 128 lanes x
    SMs x clock, within the clock's reach), and the force loop alone stays
    under the ceiling its instruction mix sets: 12 FMA-pipe operations per
    interaction counted as 20 flops, 20/24 of the FP32 peak."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = 2 * 128 * sms * 2.07e9 / 1e12
    scalar, paired = tc.probe_fp32(False), tc.probe_fp32(True)
    assert 0.5 * peak < scalar < 1.05 * peak
    assert 0.5 * peak < paired < 1.05 * peak
    loop = tc.probe_force()
    assert 0.1 * peak < loop <= 20.0 / 24.0 * 1.02 * max(scalar, paired)
