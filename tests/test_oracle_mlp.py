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
            q = _quad_accel(t.quad[v], com, M, x) * r2 / M
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
