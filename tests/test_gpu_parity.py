"""GPU path vs the FP64 CPU oracle, through the C ABI (libtc.so).

Bit-exact: Morton permutation and keys, the node table (levels, prefixes,
body ranges, children), the groups, and the per-group interaction-list
lengths and hashes, except for groups the oracle flags as holding an
opening test within 1e-6 (relative) of the threshold.

Floating point: forces within 2e-5 relative of the oracle's FP64 forces on
the same tree and lists, for every body whose force is not dominated by
cancellation; every body within the float32 rounding bound of its list sum,
err <= 2e-5 |a| + 32 u sum_j |a_ij| (u = 2^-24).  Cell masses and centres of
mass within FP64 rounding.
"""
import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs
from tests.helpers import rel_err_rms

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _bodies(kind, n, seed):
    if kind == "plummer":
        p, v, m = inputs.plummer(n, seed)
    elif kind == "uniform":
        p, v, m = inputs.uniform_cube(n, seed)
    elif kind == "random":
        rng = np.random.default_rng(seed)
        p = rng.standard_normal((n, 3)).astype(np.float32)
        v = np.zeros((n, 3), np.float32)
        m = rng.uniform(0.5, 1.5, n).astype(np.float32)
    elif kind == "masses":
        # masses over twelve decades: the float-pair moment sums against FP64
        rng = np.random.default_rng(seed)
        p = rng.standard_normal((n, 3)).astype(np.float32)
        v = np.zeros((n, 3), np.float32)
        m = (10.0 ** rng.uniform(-6, 6, n)).astype(np.float32)
    elif kind == "offset":
        # a tight cluster far from the origin: m x sums of large terms
        rng = np.random.default_rng(seed)
        p = (1000.0 + 0.01 * rng.standard_normal((n, 3))).astype(np.float32)
        v = np.zeros((n, 3), np.float32)
        m = (10.0 ** rng.uniform(-3, 3, n)).astype(np.float32)
    elif kind == "coincident":
        p = np.zeros((n, 3), np.float32)
        p[: n // 2] = [0.5, 0.5, 0.5]
        p[n // 2:] = [-0.25, 0.75, 0.125]
        v = np.zeros((n, 3), np.float32)
        m = np.full(n, 1.0 / n, np.float32)
    else:
        raise ValueError(kind)
    return p, v, m


def _ctx(tc, **cfg):
    base = dict(gmax=64, verify=1, want_pot=1, precise=1, quad=1)
    base.update(cfg)
    return tc.Context(**base)


def _compare_tree(ctx, t, gmax):
    tr = ctx.tree()
    n, M, G = ctx.sizes()
    assert n == t.n and M == t.M, (M, t.M)
    assert np.array_equal(tr["perm"], t.perm)
    assert np.array_equal(tr["keys"], t.keys)
    assert np.array_equal(ctx.cube(), t.cube5)
    for k in ("level", "first", "count", "nchild", "child_first"):
        assert np.array_equal(tr[k].astype(np.int64), getattr(t, k).astype(np.int64)), k
    assert np.array_equal(tr["prefix"], t.prefix)
    side = t.side()
    assert np.allclose(tr["mass"], t.node_mass, rtol=1e-12, atol=0)
    scale = np.abs(t.com).max(1) + side
    assert np.all(np.abs(tr["com"] - t.com).max(1) <= 1e-12 * scale)
    if tr["quad"] is not None:
        # second moments are FP32.  A leaf of c bodies: offsets within two
        # roundings (formed against the cube centre split in two floats),
        # products and c running-sum roundings, each at most u = 2^-24 of a
        # term of size <= M s^2 / 4, plus the parallel-axis shift:
        # (c + 10) u M s^2 / 4.  A cell above: its children's offsets d
        # from its centre of mass are formed in FP32 from the stored
        # centre-of-mass offsets (three roundings of numbers <= s, one of d:
        # 3.5 u s), so 6 u m_c s^2 per child term, plus 12 roundings of terms
        # <= 1.25 M s^2, plus the children's errors, a quarter of theirs in
        # units of the parent's M s^2: at most 28 u M s^2 in all.  Together
        # (leaf_max + 122) 2^-26 M s^2, taken as leaf_max + 128 and with a
        # factor 2 of margin.
        qs = t.node_mass * side ** 2
        assert np.all(np.abs(tr["quad"] - t.quad).max(1) <= (t.leaf_max + 128) * 2.0 ** -25 * qs)
    t.make_groups(gmax)
    assert G == t.G
    assert np.array_equal(tr["gfirst"], t.gfirst)
    assert np.array_equal(tr["gcount"], t.gcount)
    assert np.array_equal(tr["gref"], t.gref)


@pytest.mark.parametrize("kind,n,leaf,gmax", [
    ("plummer", 4096, 8, 64), ("random", 1, 1, 32), ("random", 2, 1, 32), ("random", 9, 8, 32),
    ("random", 17, 4, 64), ("random", 100, 3, 128), ("uniform", 5000, 16, 64), ("coincident", 40, 4, 32),
    ("random", 3000, 1, 32), ("plummer", 20000, 64, 128), ("plummer", 30000, 256, 128),
    ("uniform", 30000, 300, 64), ("masses", 20000, 16, 64), ("offset", 20000, 16, 64)])
def test_tree_bit_exact(tc, kind, n, leaf, gmax):
    p, _, m = _bodies(kind, n, 7)
    ctx = _ctx(tc, gmax=gmax)
    ctx.build(_dev(p), _dev(m), leaf)
    t = oracle.Tree(p, m, leaf)
    _compare_tree(ctx, t, gmax)


def _check_forces(acc, pot, w, t, mask_bodies, tol=2e-5, kappa_max=50.0, excluded_max=0.01):
    """Forces against the oracle's: every body within tol |a| + 32 ulps of
    sum_j |a_ij| (the float32 rounding of the terms, which cancellation does
    not shrink); the bodies whose sum is not dominated by cancellation
    (kappa = sum_j |a_ij| / |a| <= kappa_max) within tol |a| outright.  The
    bodies left to the first bar are counted, printed, and held to at most
    excluded_max of the compared bodies."""
    a_or = w["acc"][mask_bodies]
    a_gpu = acc[mask_bodies].astype(np.float64)
    err = np.linalg.norm(a_gpu - a_or, axis=1)
    amp = np.linalg.norm(a_or, axis=1)
    amag = w["amag"][mask_bodies]
    kappa = amag / np.maximum(amp, 1e-300)
    assert np.all(err <= tol * amp + 32 * U32 * amag), (err / amp).max()
    well = kappa <= kappa_max
    n_ex = int((~well).sum())
    print(f"forces: {well.size} bodies compared, {n_ex} with kappa > {kappa_max:g} "
          f"({n_ex / max(1, well.size):.2e}), max rel err {((err / np.maximum(amp, 1e-300))[well]).max():.2e}")
    assert n_ex <= excluded_max * max(1, well.size), (n_ex, well.size)
    rel = err[well] / amp[well]
    assert rel.max() <= tol, rel.max()
    if pot is not None:
        p_or = w["pot"][mask_bodies]
        perr = np.abs(pot[mask_bodies] - p_or)
        assert np.all(perr <= tol * np.abs(p_or)), (perr / np.abs(p_or)).max()
    return float(rel.max()), n_ex


def _walk_case(tc, kind, n, leaf, gmax, theta, eps, G=1.0, precise=1, stack=1024, seed=3):
    p, _, m = _bodies(kind, n, seed)
    ctx = _ctx(tc, gmax=gmax, precise=precise, stack=stack)
    ctx.build(_dev(p), _dev(m), leaf)
    ctx.forces(theta, eps, G)
    acc, pot = ctx.get_acc(with_pot=True)
    L = ctx.lists()
    t = oracle.Tree(p, m, leaf, gmax)
    w = t.walk(theta, eps, G)
    return ctx, t, w, acc, pot, L


@pytest.mark.parametrize("kind,n,leaf,gmax,theta,eps", [
    ("plummer", 4096, 8, 64, 0.5, 0.01),
    ("plummer", 4096, 8, 32, 0.75, 0.01),
    ("plummer", 4096, 8, 128, 0.9, 0.01),
    ("uniform", 20000, 16, 64, 0.7, 1e-3),
    ("random", 777, 1, 32, 0.6, 0.05),
    ("coincident", 100, 4, 32, 0.5, 0.01),
    ("random", 2, 1, 32, 0.5, 0.1),
    ("random", 1, 1, 32, 0.5, 0.1),
])
def test_lists_and_forces_match_oracle(tc, kind, n, leaf, gmax, theta, eps):
    ctx, t, w, acc, pot, L = _walk_case(tc, kind, n, leaf, gmax, theta, eps, G=0.75)
    ok = w["flag"] == 0
    assert ok.mean() > 0.9
    assert np.array_equal(L["ncell"][ok], w["ncell"][ok])
    assert np.array_equal(L["nbody"][ok], w["nbody"][ok])
    assert np.array_equal(L["hash"][ok], w["hash"][ok])
    assert L["interactions"] == int(np.sum(t.gcount * (L["ncell"] + L["nbody"])))
    body_ok = np.zeros(n, bool)
    for g in np.where(ok)[0]:
        body_ok[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
    if n == 1:
        assert np.all(acc == 0)
        return
    _check_forces(acc, pot, w, t, body_ok)


def test_theta_zero_is_direct_summation(tc):
    n = 3000
    ctx, t, w, acc, pot, L = _walk_case(tc, "plummer", n, 8, 64, 0.0, 0.01, stack=4096)
    assert np.all(L["ncell"] == 0) and np.all(L["nbody"] == n)
    ad, pd = oracle.direct(*_bodies("plummer", n, 3)[::2], 0.01)
    _check_forces(acc, pot, dict(acc=ad, pot=pd, amag=w["amag"]), t, np.ones(n, bool))


def test_plain_mode_matches_oracle(tc):
    ctx, t, w, acc, pot, L = _walk_case(tc, "plummer", 4096, 8, 64, 0.5, 0.01, precise=0)
    ok = w["flag"] == 0
    assert np.array_equal(L["ncell"][ok], w["ncell"][ok])
    body_ok = np.zeros(t.n, bool)
    for g in np.where(ok)[0]:
        body_ok[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
    _check_forces(acc, pot, w, t, body_ok, tol=1e-4)


def test_full_size_uniform_1m_sampled(tc):
    """The bench workload (uniform cube, N = 2^20, leaf 16, eps 1e-3,
    theta 0.5 and 0.7, default launch configuration): whole tree bit-exact,
    lists and forces of sampled groups against the oracle, RMS error against
    direct summation on 4096 sampled bodies at or below 1e-3 at theta 0.5."""
    n = 1 << 20
    p, _, m = _bodies("uniform", n, 0)
    ctx = tc.Context(verify=1, want_pot=0)
    gmax = ctx.config()["gmax"]
    ctx.build(_dev(p), _dev(m), 16)
    t = oracle.Tree(p, m, 16)
    _compare_tree(ctx, t, gmax)
    for theta in (0.5, 0.7):
        ctx.forces(theta, 1e-3)
        acc = ctx.get_acc()
        L = ctx.lists()
        groups = []
        for g0 in np.linspace(0, t.G - 200, 6).astype(int):
            groups.append((g0, g0 + 200))
        body_ok = np.zeros(n, bool)
        w_all = dict(acc=np.full((n, 3), np.nan), amag=np.full(n, np.nan))
        for g0, g1 in groups:
            w = t.walk(theta, 1e-3, groups=(g0, g1), want_pot=False)
            sl = slice(g0, g1)
            ok = w["flag"][sl] == 0
            assert np.array_equal(L["ncell"][sl][ok], w["ncell"][sl][ok])
            assert np.array_equal(L["nbody"][sl][ok], w["nbody"][sl][ok])
            assert np.array_equal(L["hash"][sl][ok], w["hash"][sl][ok])
            for g in np.arange(g0, g1)[ok]:
                idx = t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]
                body_ok[idx] = True
                w_all["acc"][idx] = w["acc"][idx]
                w_all["amag"][idx] = w["amag"][idx]
        _check_forces(acc, None, w_all, t, body_ok)
        if theta == 0.5:
            idx = inputs.sample_indices(n, 4096, seed=1)
            ad, _ = ctx.direct(idx, 1e-3)
            assert rel_err_rms(acc[idx].astype(np.float64), ad) <= 1e-3


def test_direct_kernel_matches_oracle(tc):
    p, _, m = _bodies("plummer", 20000, 5)
    ctx = _ctx(tc)
    ctx.build(_dev(p), _dev(m), 8)
    idx = inputs.sample_indices(20000, 300, seed=2)
    a, ph = ctx.direct(idx, 0.01, 2.0)
    ao, po = oracle.direct(p, m, 0.01, 2.0, idx=idx)
    assert np.all(np.linalg.norm(a - ao, axis=1) <= 1e-5 * np.linalg.norm(ao, axis=1))
    assert np.all(np.abs(ph - po) <= 1e-6 * np.abs(po))


def test_step_matches_oracle(tc):
    """One kick-drift-kick step: the drift from the GPU's own state to
    within float32 rounding, the rebuilt tree bit-exact, the closing kick
    within the force tolerance."""
    n, dt, eps = 4096, 1e-3, 0.01
    p, v, m = _bodies("plummer", n, 0)
    ctx = _ctx(tc)
    ctx.build(_dev(p), _dev(m), 8)
    ctx.set_velocity(_dev(v))
    ctx.forces(0.5, eps)
    a0 = ctx.get_acc().astype(np.float64)
    x0, v0 = ctx.get_state()
    ctx.step(dt)
    x1, v1 = ctx.get_state()
    h = dt / 2
    vh = v0.astype(np.float64) + a0 * h
    x1o = x0.astype(np.float64) + vh * dt
    # float32 rounding of vh = fl(v + fl(a h)) and x1 = fl(x + fl(vh dt)),
    # each op within u = 2^-24 relative
    err_vh = U32 * (np.abs(a0 * h) + np.abs(vh))
    tol_x = 2 * (U32 * (np.abs(x1o) + np.abs(vh * dt)) + dt * err_vh)
    assert np.all(np.abs(x1 - x1o) <= tol_x)
    t = oracle.Tree(x1, m, 8)
    _compare_tree(ctx, t, 64)
    w = t.walk(0.5, eps)
    v1o = vh + w["acc"] * h
    tol_v = 2 * (err_vh + U32 * (np.abs(w["acc"] * h) + np.abs(v1o))) + 2e-5 * np.abs(w["acc"]) * h
    assert np.all(np.abs(v1 - v1o) <= tol_v)


def test_diag_matches_oracle(tc):
    p, v, m = _bodies("plummer", 4096, 0)
    ctx = _ctx(tc)
    ctx.build(_dev(p), _dev(m), 8)
    ctx.set_velocity(_dev(v))
    ctx.forces(0.5, 0.01)
    d = ctx.diag()
    _, pot = ctx.get_acc(with_pot=True)
    do = oracle.diag(p, v, m, pot)
    assert np.allclose(d, do, rtol=1e-10, atol=1e-12)
    t = oracle.Tree(p, m, 8, 64)
    w = t.walk(0.5, 0.01)
    assert abs(d[1] - oracle.diag(p, v, m, w["pot"])[1]) <= 1e-5 * abs(d[1])


def test_energy_and_momentum_over_steps(tc):
    """20 KDK steps of a Plummer sphere: momentum stays ~0 and the energy
    change is small (treecode force error + O(dt^2))."""
    p, v, m = _bodies("plummer", 8192, 4)
    ctx = _ctx(tc)
    ctx.build(_dev(p), _dev(m), 8)
    ctx.set_velocity(_dev(v))
    ctx.forces(0.5, 0.01)
    d0 = ctx.diag()
    for _ in range(20):
        ctx.step(1e-3)
    d1 = ctx.diag()
    E0, E1 = d0[0] + d0[1], d1[0] + d1[1]
    assert abs(E1 - E0) <= 2e-4 * abs(E0)
    assert np.abs(d1[2:5] - d0[2:5]).max() <= 1e-5


def test_checkpoint_resume_bit_identical(tc):
    p, v, m = _bodies("plummer", 4096, 6)
    ctx = _ctx(tc)
    ctx.build(_dev(p), _dev(m), 8)
    ctx.set_velocity(_dev(v))
    ctx.forces(0.6, 0.01)
    for _ in range(2):
        ctx.step(1e-3)
    xs, vs = ctx.get_state()
    for _ in range(3):
        ctx.step(1e-3)
    xa, va = ctx.get_state()
    ctx.set_state(xs, vs)
    ctx.forces(0.6, 0.01)
    for _ in range(3):
        ctx.step(1e-3)
    xb, vb = ctx.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_host_buffers_give_the_same_result(tc):
    p, _, m = _bodies("plummer", 4096, 9)
    c1 = _ctx(tc)
    c1.build(_dev(p), _dev(m), 8)
    c1.forces(0.5, 0.01)
    c2 = _ctx(tc)
    c2.build(p, m, 8)
    c2.forces(0.5, 0.01)
    assert np.array_equal(c1.get_acc(), c2.get_acc())


def test_default_context_calls(tc):
    p, _, m = _bodies("plummer", 2048, 1)
    tc.tc_build(_dev(p), _dev(m), 2048, 8)
    tc.tc_forces(0.5, 0.01, 1.0)
    tc.tc_step(1e-3)
    lib = tc.load()
    assert lib.tc_default()


# ---------------------------------------------------------------- errors
def test_invalid_arguments(tc):
    p, _, m = _bodies("random", 100, 1)
    ctx = _ctx(tc)
    with pytest.raises(tc.TcError) as e:
        ctx.forces(0.5, 0.01)
    assert e.value.code == tc.TC_ESTATE
    with pytest.raises(tc.TcError) as e:
        ctx.build(_dev(p[:0]), _dev(m[:0]), 8)
    assert e.value.code == tc.TC_EINVAL
    with pytest.raises(tc.TcError) as e:
        ctx.build(_dev(p), _dev(m), 0)
    assert e.value.code == tc.TC_EINVAL
    ctx.build(_dev(p), _dev(m), 8)
    with pytest.raises(tc.TcError) as e:
        ctx.step(1e-3)
    assert e.value.code == tc.TC_ESTATE
    for th, ep in ((-0.1, 0.01), (0.5, 0.0), (float("nan"), 0.01), (0.5, float("inf"))):
        with pytest.raises(tc.TcError) as e:
            ctx.forces(th, ep)
        assert e.value.code == tc.TC_EINVAL
    with pytest.raises(tc.TcError):
        ctx.set_config(gmax=48)
    ctx.forces(0.5, 0.01)  # still usable


@pytest.mark.parametrize("bad", ["nan_pos", "inf_pos", "zero_mass", "neg_mass"])
def test_bad_inputs_rejected(tc, bad):
    p, _, m = _bodies("random", 100, 2)
    if bad == "nan_pos":
        p[17, 1] = np.nan
    elif bad == "inf_pos":
        p[3, 0] = np.inf
    elif bad == "zero_mass":
        m[5] = 0.0
    else:
        m[9] = -1.0
    ctx = _ctx(tc)
    with pytest.raises(tc.TcError) as e:
        ctx.build(_dev(p), _dev(m), 8)
    assert e.value.code == tc.TC_EINVAL
    p2, _, m2 = _bodies("random", 100, 3)
    ctx.build(_dev(p2), _dev(m2), 8)  # the context recovers
    ctx.forces(0.5, 0.01)
    ctx.get_acc()


def test_walk_stack_overflow_is_reported(tc):
    """A stack too small for theta = 0 sets the kernel's error word (the
    kernel checks before every push) and the next sync reports it."""
    p, _, m = _bodies("plummer", 4096, 1)
    ctx = _ctx(tc, stack=64)
    ctx.build(_dev(p), _dev(m), 4)
    ctx.forces(0.0, 0.01)
    with pytest.raises(tc.TcError) as e:
        ctx.get_acc()
    assert e.value.code == tc.TC_EDEVICE
    ctx.set_config(stack=4096)
    ctx.forces(0.0, 0.01)
    ctx.get_acc()


def test_allocation_cap_is_reported(tc, monkeypatch):
    p, _, m = _bodies("random", 10000, 4)
    monkeypatch.setenv("TC_ALLOC_CAP_BYTES", "100000")
    ctx = _ctx(tc)
    with pytest.raises(tc.TcError) as e:
        ctx.build(_dev(p), _dev(m), 8)
    assert e.value.code == tc.TC_ENOMEM
    monkeypatch.delenv("TC_ALLOC_CAP_BYTES")
    ctx2 = _ctx(tc)
    ctx2.build(_dev(p), _dev(m), 8)


@pytest.mark.parametrize("gmax,theta", [(1, 0.5), (1, 0.8), (8, 0.6), (17, 0.7)])
def test_small_groups_and_per_body_lists(tc, gmax, theta):
    """gmax = 1 is the paper's per-body list: every body walks the tree with
    its own opening test (the group box is the body itself)."""
    n = 2000
    p, _, m = _bodies("plummer", n, 21)
    ctx = _ctx(tc, gmax=gmax)
    ctx.build(_dev(p), _dev(m), 8)
    ctx.forces(theta, 0.01)
    acc, pot = ctx.get_acc(with_pot=True)
    L = ctx.lists()
    t = oracle.Tree(p, m, 8, gmax)
    _compare_tree(ctx, t, gmax)
    if gmax == 1:
        assert t.G == n
    w = t.walk(theta, 0.01)
    ok = w["flag"] == 0
    assert ok.mean() > 0.9
    assert np.array_equal(L["ncell"][ok], w["ncell"][ok])
    assert np.array_equal(L["nbody"][ok], w["nbody"][ok])
    assert np.array_equal(L["hash"][ok], w["hash"][ok])
    body_ok = np.zeros(n, bool)
    for g in np.where(ok)[0]:
        body_ok[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
    _check_forces(acc, pot, w, t, body_ok)


@pytest.mark.parametrize("gmax,theta", [(64, 0.6), (1, 0.7), (32, 0.0)])
def test_group_list_export_matches_oracle(tc, gmax, theta):
    n = 3000
    p, _, m = _bodies("plummer", n, 22)
    ctx = _ctx(tc, gmax=gmax)
    ctx.build(_dev(p), _dev(m), 8)
    ctx.forces(0.5, 0.01)
    acc0 = ctx.get_acc().copy()
    L0 = ctx.lists(per_group=False)
    t = oracle.Tree(p, m, 8, gmax)
    w = t.walk(theta, 0.01, want_pot=False)
    G = ctx.sizes()[2]
    checked = 0
    for g in np.unique(np.linspace(0, G - 1, 12).astype(int)):
        if w["flag"][g]:
            continue
        cells, leaves = ctx.group_list(int(g), theta)
        oc, ol = t.group_list(int(g), theta)
        assert np.array_equal(np.sort(cells), np.sort(oc))
        assert np.array_equal(np.sort(leaves), np.sort(ol))
        checked += 1
    assert checked >= 8
    # forces and totals of the last force phase are untouched
    assert np.array_equal(ctx.get_acc(), acc0)
    assert ctx.lists(per_group=False)["interactions"] == L0["interactions"]
    # a short buffer gets the first entries, the lengths stay full
    import ctypes
    nc, nl = ctypes.c_int64(), ctypes.c_int64()
    buf_c = np.zeros(3, np.int32)
    buf_l = np.zeros(3, np.int32)
    rc = ctx._lib.tc_get_group_list(ctx._h, 0, ctypes.c_float(theta), buf_c.ctypes.data_as(ctypes.c_void_p),
                                    buf_l.ctypes.data_as(ctypes.c_void_p), 3, ctypes.byref(nc), ctypes.byref(nl))
    assert rc == 0
    full_c, full_l = ctx.group_list(0, theta)
    assert nc.value == len(full_c) and nl.value == len(full_l)
    assert np.array_equal(buf_c[:min(3, len(full_c))], full_c[:3])
    with pytest.raises(tc.TcError):
        ctx.group_list(G, theta)


@pytest.mark.parametrize("gmax", [64, 128])
def test_size_class_modes_agree(tc, gmax):
    """The walk's size classes change which kernel sums a group (one, two or
    four bodies per lane), never a body's list or the order of its sums:
    classes = 0 (one launch) and 1 (one launch per class) give the same
    lists and the same bits, both the oracle's forces to float32 rounding."""
    p, _, m = _bodies("plummer", 20000, 23)
    t = oracle.Tree(p, m, 16, gmax)
    # the workload mixes the classes: groups of <= 16, <= 32, <= 48, <= 64
    # (and more)
    c = t.gcount
    assert (c <= 16).any() and ((c > 16) & (c <= 32)).any()
    assert ((c > 32) & (c <= 48)).any() and ((c > 48) & (c <= 64)).any()
    if gmax == 128:
        assert ((c > 64) & (c <= 96)).any() and (c > 112).any()
    w = t.walk(0.6, 0.01)
    ok = w["flag"] == 0
    body_ok = np.zeros(len(p), bool)
    for g in np.where(ok)[0]:
        body_ok[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
    lists, accs = {}, {}
    for classes in (0, 1):
        ctx = _ctx(tc, gmax=gmax, classes=classes)
        ctx.build(_dev(p), _dev(m), 16)
        ctx.forces(0.6, 0.01)
        acc, pot = ctx.get_acc(with_pot=True)
        L = ctx.lists()
        lists[classes] = L
        accs[classes] = (acc.copy(), pot.copy())
        assert np.array_equal(L["ncell"][ok], w["ncell"][ok])
        assert np.array_equal(L["nbody"][ok], w["nbody"][ok])
        _check_forces(acc, pot, w, t, body_ok)
    for k in ("ncell", "nbody", "hash"):
        assert np.array_equal(lists[0][k], lists[1][k]), k
    assert lists[0]["interactions"] == lists[1]["interactions"]
    assert np.array_equal(accs[0][0], accs[1][0]) and np.array_equal(accs[0][1], accs[1][1])


@pytest.mark.parametrize("kind,n,leaf", [("uniform", 1 << 18, 16), ("plummer", 1 << 18, 16), ("plummer", 50000, 4)])
def test_step_sort_of_top_digits_gives_the_full_order(tc, kind, n, leaf):
    """Inside a step the radix passes sort only the key digits down to the
    last synchronised depth + 2 levels and complete every run of equal top
    digits by itself: Morton order, keys and tree equal the oracle's full
    sort on the stepped positions."""
    p, v, m = _bodies(kind, n, 41)
    ctx = _ctx(tc, gmax=64)
    ctx.build(_dev(p), _dev(m), leaf)
    ctx.forces(0.6, 0.01)
    ctx.sizes()  # synchronise: the depth hint
    rng = np.random.default_rng(42)
    ctx.set_velocity(_dev((0.1 * rng.standard_normal((n, 3))).astype(np.float32)))
    ctx.step(1e-3)
    pos, _ = ctx.get_state()
    t = oracle.Tree(pos, m, leaf, 64)
    _compare_tree(ctx, t, 64)


@pytest.mark.parametrize("cluster", [600, 5000])
def test_synchronised_build_with_a_stale_depth_hint(tc, cluster):
    """A synchronised build of a system of the same size as the last one
    sorts the digits down to that one's depth + 2 and completes the runs;
    a new system with a tight cluster gives long runs: completed in place up
    to 1024 bodies (600), else the build is redone sorting every digit
    (5000).  Either way the tree equals the oracle's full sort."""
    n = 20000
    p, _, m = _bodies("uniform", n, 51)
    ctx = _ctx(tc, gmax=64)
    ctx.build(_dev(p), _dev(m), 16)
    ctx.sizes()
    q = p.copy()
    q[:cluster] = (0.3 + 1e-5 * np.random.default_rng(52).random((cluster, 3))).astype(np.float32)
    ctx.build(_dev(q), _dev(m), 16)
    t = oracle.Tree(q, m, 16)
    _compare_tree(ctx, t, 64)


def test_step_builds_a_deeper_tree_than_the_last_synchronised_one(tc):
    """A captured step knows the tree depth only from an earlier build; its
    moment reduction gives each level down to that depth + 2 a launch and
    any deeper level one block; its sort orders the key digits down to that
    depth + 2 and completes longer runs of equal digits one block each.  The
    drift of one step moves 40 bodies into a cube of side 1e-6, so the
    step's tree is 15+ levels deeper than the last synchronised one: its
    order, moments and structure still equal the oracle's on the new
    positions."""
    p, _, m = _bodies("uniform", 4096, 31)
    ctx = _ctx(tc, gmax=64)
    ctx.build(_dev(p), _dev(m), 8)
    ctx.forces(0.5, 0.01)
    ctx.sizes()  # synchronise: the depth hint is this shallow tree's
    dt = 1e-6
    target = 0.9 + 1e-6 * np.random.default_rng(5).random((40, 3))
    v = np.zeros_like(p)
    v[:40] = ((target - p[:40]) / dt).astype(np.float32)
    ctx.set_velocity(_dev(v))
    ctx.step(dt)  # kick, drift into the cluster, rebuild inside the captured step, walk, kick
    pos, _ = ctx.get_state()
    t = oracle.Tree(pos, m, 8, 64)
    assert t.level.max() >= 15
    _compare_tree(ctx, t, 64)


@pytest.mark.parametrize("kind,n,leaf,gmax,theta,eps,precise,pot,tile,warps", [
    ("plummer", 20000, 8, 64, 0.6, 0.01, 1, 1, 128, 4),
    ("uniform", 50000, 16, 64, 0.5, 1e-3, 1, 0, 128, 4),
    ("plummer", 20000, 8, 128, 0.9, 0.01, 0, 1, 256, 2),
    ("plummer", 7000, 8, 32, 0.7, 0.01, 1, 0, 64, 1),
    ("random", 3000, 1, 17, 0.6, 0.05, 1, 1, 128, 3),
])
def test_split_walk_matches_one_warp_walk_and_oracle(tc, kind, n, leaf, gmax, theta, eps, precise, pot, tile, warps):
    """The producer/consumer walk (split = 1) builds the same lists as the
    one-warp walk (split = 0) -- lengths and set hashes of every group
    bit-exact -- and its forces meet the oracle bar; the two sums differ only
    in the order the tiles are added (within 2e-5 relative of each other)."""
    p, _, m = _bodies(kind, n, 11)
    out = {}
    for split in (0, 1):
        ctx = _ctx(tc, gmax=gmax, precise=precise, want_pot=pot, tile=tile, warps=warps, split=split)
        ctx.build(_dev(p), _dev(m), leaf)
        ctx.forces(theta, eps)
        if pot:
            acc, pt = ctx.get_acc(with_pot=True)
        else:
            acc, pt = ctx.get_acc(), None
        out[split] = (acc.copy(), None if pt is None else pt.copy(), ctx.lists())
    L0, L1 = out[0][2], out[1][2]
    for k in ("ncell", "nbody", "hash"):
        assert np.array_equal(L0[k], L1[k]), k
    assert L0["interactions"] == L1["interactions"]
    a0, a1 = out[0][0].astype(np.float64), out[1][0].astype(np.float64)
    assert np.all(np.linalg.norm(a1 - a0, axis=1) <= 2e-5 * np.linalg.norm(a0, axis=1) + 1e-30)
    t = oracle.Tree(p, m, leaf, gmax)
    w = t.walk(theta, eps)
    ok = np.zeros(n, bool)
    for g in np.where(w["flag"] == 0)[0]:
        ok[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
    _check_forces(out[1][0], out[1][1], w, t, ok, tol=2e-5 if precise else 1e-4)


@pytest.mark.parametrize("split", [0, 1])
def test_walk_stack_overflow_reported_both_walks(tc, split):
    """A stack too small for theta = 0 stops the affected groups of either
    walk with TC_EDEVICE; the context stays usable."""
    p, _, m = _bodies("plummer", 20000, 3)
    ctx = _ctx(tc, stack=64, split=split)
    ctx.build(_dev(p), _dev(m), 4)
    ctx.forces(0.0, 0.01)
    with pytest.raises(tc.TcError) as e:
        ctx.sync()
    assert e.value.code == tc.TC_EDEVICE
    ctx.set_config(stack=4096)
    ctx.forces(0.5, 0.01)
    ctx.sync()
