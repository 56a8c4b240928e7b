"""Pins of the oracle's learned-correction pieces (features, labels, MLP).

The label is pinned to the textbook multipole expansion: for a cell far
away it tends to the (normalised) quadrupole field computed here from the
quadrupole potential by finite differences; for a one-body cell it is zero.
The MLP's gradient is pinned to central finite differences of its loss, its
forward pass to a hand-wired network whose output is known in closed form.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs

H = 64


def _split(p):
    o = 0
    out = []
    for shape in ((13, H), (H,), (H, H), (H,), (H, 3), (3,)):
        k = int(np.prod(shape))
        out.append(p[o:o + k].reshape(shape))
        o += k
    return out


def _pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([a.ravel() for a in (W1, b1, W2, b2, W3, b3)])


def test_mlp_forward_hand_wired():
    """W1 = [I | 0], W2 = I, W3 picks columns 4, 0, 9: y = relu(x)[[4, 0, 9]] + b3."""
    W1 = np.zeros((13, H)); W1[:, :13] = np.eye(13)
    W2 = np.eye(H)
    W3 = np.zeros((H, 3)); W3[4, 0] = 1.0; W3[0, 1] = 2.0; W3[9, 2] = -1.0
    b3 = np.array([0.5, -0.25, 1.0])
    p = _pack(W1, np.zeros(H), W2, np.zeros(H), W3, b3)
    X = np.random.default_rng(1).standard_normal((20, 13))
    Y = oracle.mlp_forward(p, X)
    r = np.maximum(X, 0)
    expect = np.stack([r[:, 4], 2 * r[:, 0], -r[:, 9]], 1) + b3
    assert np.allclose(Y, expect, rtol=0, atol=1e-15)
    # biases reach the output through the ReLUs
    b1 = np.full(H, -1e9)
    p2 = _pack(W1, b1, W2, np.zeros(H), W3, b3)
    assert np.allclose(oracle.mlp_forward(p2, X), b3, atol=0)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = rng.standard_normal(oracle.MLP_NPARAM) * 0.3
    X = rng.standard_normal((9, 13))
    T = rng.standard_normal((9, 3))
    L, g = oracle.mlp_grad(p, X, T)
    Y = oracle.mlp_forward(p, X)
    assert L == pytest.approx(np.mean(np.sum((Y - T) ** 2, 1)), rel=1e-14)
    idx = rng.choice(oracle.MLP_NPARAM, 300, replace=False)
    idx = np.concatenate([idx, [oracle.MLP_NPARAM - 1, oracle.MLP_NPARAM - 4, 0, 13 * H]])
    fd = np.zeros(idx.size)
    for k, i in enumerate(idx):
        h = 1e-6
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd[k] = (oracle.mlp_grad(pp, X, T)[0] - oracle.mlp_grad(pm, X, T)[0]) / (2 * h)
    assert np.linalg.norm(fd - g[idx]) <= 1e-6 * np.linalg.norm(g[idx])
    # per-pair weights: the loss is the weighted mean, the gradient follows
    w = rng.uniform(0.1, 3.0, 9)
    Lw, gw = oracle.mlp_grad(p, X, T, w)
    assert Lw == pytest.approx(np.mean(w * np.sum((Y - T) ** 2, 1)), rel=1e-14)
    fdw = np.zeros(idx.size)
    for k, i in enumerate(idx[:60]):
        h = 1e-6
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fdw[k] = (oracle.mlp_grad(pp, X, T, w)[0] - oracle.mlp_grad(pm, X, T, w)[0]) / (2 * h)
    assert np.linalg.norm(fdw[:60] - gw[idx[:60]]) <= 1e-6 * np.linalg.norm(gw[idx[:60]])
    # a weight of 2 on every pair doubles loss and gradient
    L2, g2 = oracle.mlp_grad(p, X, T, np.full(9, 2.0))
    assert L2 == pytest.approx(2 * L, rel=1e-14) and np.allclose(g2, 2 * g, rtol=1e-13, atol=0)


def test_label_is_zero_for_one_body_cells():
    p, _, m = inputs.plummer(2000, 4)
    t = oracle.Tree(p, m, 1)
    ones = np.where(t.count == 1)[0][:50]
    x = np.array([3.0, -2.0, 1.5])
    for v in ones:
        assert np.abs(t.mlp_label(int(v), x, 1e-3)).max() <= 1e-12


def _quad_accel(Q, com, M, x, G=1.0):
    """Quadrupole field of a mass distribution with second moments Q about
    its centre of mass: Phi = -G (3 r^T Q r / r^2 - tr Q) / (2 r^3), r = x - com;
    a = -grad Phi by central differences."""
    Qm = np.array([[Q[0], Q[1], Q[2]], [Q[1], Q[3], Q[4]], [Q[2], Q[4], Q[5]]])

    def phi(y):
        r = y - com
        rr = np.sqrt(r @ r)
        return -G * (3 * (r @ Qm @ r) / rr ** 2 - np.trace(Qm)) / (2 * rr ** 3)

    h = 1e-5 * np.sqrt((x - com) @ (x - com))
    a = np.zeros(3)
    for k in range(3):
        e = np.zeros(3); e[k] = h
        a[k] = -(phi(x + e) - phi(x - e)) / (2 * h)
    return a


def test_label_tends_to_the_quadrupole_term():
    p, _, m = inputs.plummer(4000, 5)
    t = oracle.Tree(p, m, 8)
    cand = [v for v in range(t.M) if t.count[v] >= 40 and t.level[v] >= 2][:5]
    assert cand
    for v in cand:
        s = t.side(v)
        com = t.com[v]
        M = t.node_mass[v]
        errs = []
        for dist in (10.0, 20.0, 40.0):
            direction = np.array([0.48, -0.6, 0.64])
            x = com + dist * s * direction
            lab = t.mlp_label(v, x, 1e-9)
            r2 = np.sum((com - x) ** 2)
            q = _quad_accel(t.quad[v], com, M, x) * r2 ** 2 / (M * s ** 2)
            assert t.mlp_factor(v, x) == pytest.approx(M * s ** 2 / r2 ** 2, rel=1e-14)
            errs.append(np.linalg.norm(lab - q) / np.linalg.norm(q))
        # the remainder is the octupole and beyond: O(s / r) relative
        assert errs[0] < 0.35 and errs[1] < errs[0] and errs[2] < errs[1]


def test_features_definition_invariants():
    p, _, m = inputs.plummer(3000, 6)
    t = oracle.Tree(p, m, 8)
    x = np.array([0.3, 0.1, -0.2])
    for v in (5, 50, 500):
        f = t.mlp_features(v, x, 0.01, 1.0)
        s = t.side(v)
        assert np.linalg.norm(f[:3]) == pytest.approx(1.0 / f[3], rel=1e-14)
        assert f[4] == pytest.approx(0.01 / s, rel=1e-15)
        assert f[5] == pytest.approx(math.log2(t.count[v]), rel=1e-15)
        assert f[6] == pytest.approx(t.node_mass[v], rel=1e-15)
        Q = f[7:]
        Qm = np.array([[Q[0], Q[1], Q[2]], [Q[1], Q[3], Q[4]], [Q[2], Q[4], Q[5]]])
        assert np.linalg.eigvalsh(Qm).min() >= -1e-12
        # every body lies inside the cube: trace of Q/(M s^2) is at most 3/4
        assert np.trace(Qm) <= 0.75 + 1e-12


def _identity3(maps):
    """Hand-wired network whose output is its first three inputs:
    h = relu(+-x_k), y_k = h_2k - h_2k+1 = x_k."""
    W1 = np.zeros((13, H)); W2 = np.zeros((H, H)); W3 = np.zeros((H, 3))
    for k in range(3):
        W1[k, 2 * k], W1[k, 2 * k + 1] = 1.0, -1.0
        W3[2 * k, k], W3[2 * k + 1, k] = 1.0, -1.0
    for j in range(6):
        W2[j, j] = 1.0
    return _pack(W1, np.zeros(H), W2, np.zeros(H), W3, np.zeros(3)), np.asarray(maps, float)


def _group_box(t, g):
    xs = t.pos[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]].astype(np.float64)
    return xs.min(0), xs.max(0)


def _brute_accepted(t, g, theta):
    """Cells accepted by group g's walk, by definition: the cell passes the
    opening test and every ancestor fails it (holds a group body or is too
    close)."""
    lo, hi = _group_box(t, g)
    a0, a1 = t.gfirst[g], t.gfirst[g] + t.gcount[g]

    def passes(v):
        if t.first[v] < a1 and a0 < t.first[v] + t.count[v]:
            return False
        d = np.sqrt(np.sum(np.maximum(np.maximum(lo - t.com[v], t.com[v] - hi), 0.0) ** 2))
        return t.side(v) < theta * d

    out = []
    for v in range(t.M):
        if not passes(v):
            continue
        u, ok = t.parent[v], True
        while u >= 0:
            if passes(u):
                ok = False
                break
            u = t.parent[u]
        if ok:
            out.append(v)
    return out, lo, hi


def test_learned_oracle_matches_brute_force_cell_selection():
    """The band sum of the learned correction against a brute-force
    selection of the accepted cells, with a network that returns its
    normalised d/s features (so the evaluation point, the normalisation and
    the factor G M / r^2 are all visible)."""
    p, _, m = inputs.plummer(72, 9)
    t = oracle.Tree(p, m, 2, gmax=4)
    theta, band, eps, G = 0.8, 0.3, 0.01, 1.7
    mean = np.zeros(13); mean[:3] = [0.1, -0.2, 0.05]
    scale = np.ones(13); scale[:3] = [1.5, 0.5, 2.0]
    yscale = np.array([2.0, 3.0, 0.5])
    params, maps = _identity3(np.concatenate([mean, scale, yscale]))
    corr, flag, ev = t.learned(theta, eps, band, params, maps, G=G)
    assert (flag == 0).all()
    n_expect = 0
    for g in range(t.G):
        cells, lo, hi = _brute_accepted(t, g, theta)
        xg = 0.5 * (lo + hi)
        c = np.zeros(3)
        for v in cells:
            s = t.side(v)
            d = np.sqrt(np.sum(np.maximum(np.maximum(lo - t.com[v], t.com[v] - hi), 0.0) ** 2))
            if t.count[v] < 2 or s < band * d:
                continue
            dv = t.com[v] - xg
            y = (dv / s - mean[:3]) * scale[:3] * yscale
            c += G * t.node_mass[v] * s ** 2 / (dv @ dv) ** 2 * y
            n_expect += 1
        for j in range(t.gfirst[g], t.gfirst[g] + t.gcount[g]):
            assert np.allclose(corr[t.perm[j]], c, rtol=1e-12, atol=1e-12 * (np.abs(c).max() + 1e-300))
    assert ev == n_expect and ev > 0


def test_learned_oracle_exact_labels_give_the_direct_sum():
    """With one body per group (its box is the body itself), band 0 and the
    exact label, every accepted cell's monopole plus its correction is the
    cell's exact sum, so walk + correction is the direct sum."""
    p, _, m = inputs.plummer(400, 10)
    t = oracle.Tree(p, m, 1, gmax=1)
    assert t.G == t.n
    eps, G = 0.02, 1.3
    w = t.walk(0.7, eps, G, want_pot=False)
    corr, flag, ev = t.learned(0.7, eps, 0.0, None, None, G=G)
    acc_d, _ = oracle.direct(p, m, eps, G, want_pot=False)
    tot = w["acc"] + corr
    err = np.abs(tot - acc_d).max() / np.abs(acc_d).max()
    err_mono = np.abs(w["acc"] - acc_d).max() / np.abs(acc_d).max()
    assert err < 1e-12 and err_mono > 1e-6 and ev > 0


def test_learned_oracle_band_and_zero_model():
    p, _, m = inputs.plummer(500, 11)
    t = oracle.Tree(p, m, 4, gmax=16)
    zero = np.zeros(oracle.MLP_NPARAM)
    maps = np.concatenate([np.zeros(13), np.ones(13), np.ones(3)])
    corr, _, ev = t.learned(0.9, 0.01, 0.2, zero, maps)
    assert ev > 0 and not np.any(corr)
    # a band above theta selects nothing
    corr, _, ev = t.learned(0.9, 0.01, 1.0, zero, maps)
    assert ev == 0
    # the band only narrows the selection
    _, _, e1 = t.learned(0.9, 0.01, 0.0, zero, maps)
    _, _, e2 = t.learned(0.9, 0.01, 0.5, zero, maps)
    assert e1 > e2 > 0
