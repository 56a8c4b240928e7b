"""Pins of the oracle's quadrupole walk (the classical comparator of the
learned correction).

The quadrupole term is pinned to central finite differences of the
second-order Taylor expansion of the softened potential, written out here
independently of the oracle's acceleration formula; to the multipole
remainder shrinking with distance; and to theta = 0 (no cell accepted, the
direct sum).
"""
import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs


def _phi_quad(Q, com, x, eps, G=1.0):
    """-(G/2) sum_ab Q_ab d^2/dy_a dy_b (|x - y|^2 + eps^2)^(-1/2) at y = com."""
    Qm = np.array([[Q[0], Q[1], Q[2]], [Q[1], Q[3], Q[4]], [Q[2], Q[4], Q[5]]])
    d = com - x
    rho2 = d @ d + eps ** 2
    hess = 3.0 * np.outer(d, d) / rho2 ** 2.5 - np.eye(3) / rho2 ** 1.5
    return -0.5 * G * np.sum(Qm * hess)


def _cluster_and_far_body(eps_spread=0.02, n=24, seed=4):
    rng = np.random.default_rng(seed)
    c = np.array([-0.5, -0.45, -0.55])
    pts = c + rng.uniform(-eps_spread, eps_spread, (n, 3))
    far = np.array([[0.9, 0.8, 0.7]])
    p = np.concatenate([pts, far]).astype(np.float32)
    m = rng.uniform(0.5, 1.5, n + 1).astype(np.float32)
    return p, m


def test_quadrupole_term_matches_finite_differences_of_its_potential():
    p, m = _cluster_and_far_body()
    t = oracle.Tree(p, m, 1, gmax=1)
    far = p.shape[0] - 1
    eps, G = 0.05, 1.7
    w0 = t.walk(10.0, eps, G)
    w2 = t.walk(10.0, eps, G, quadrupole=True)
    # the far body's walk accepts the root's child holding the cluster
    root_children = range(t.child_first[0], t.child_first[0] + t.nchild[0])
    v = [c for c in root_children if t.count[c] == far][0]
    x = p[far].astype(np.float64)
    h = 1e-5
    fd = np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd[k] = -(_phi_quad(t.quad[v], t.com[v], x + e, eps, G) - _phi_quad(t.quad[v], t.com[v], x - e, eps, G)) / (2 * h)
    da = w2["acc"][far] - w0["acc"][far]
    assert np.linalg.norm(da - fd) <= 1e-7 * np.linalg.norm(fd)
    dphi = w2["pot"][far] - w0["pot"][far]
    assert dphi == pytest.approx(_phi_quad(t.quad[v], t.com[v], x, eps, G), rel=1e-12)


def test_quadrupole_removes_the_leading_multipole_error():
    """For a far cell the monopole's error is O((s/r)^2) of the force and the
    quadrupole-corrected error O((s/r)^3): the ratio shrinks with distance."""
    rng = np.random.default_rng(5)
    pts = rng.uniform(-0.1, 0.1, (30, 3)) + np.array([-0.3, -0.3, -0.3])
    m = rng.uniform(0.5, 1.5, 31).astype(np.float32)
    ratios = []
    for dist in (1.0, 2.0, 4.0):
        far = np.array([[-0.3 + dist, -0.3 + 0.6 * dist, -0.3 + 0.3 * dist]])
        p = np.concatenate([pts, far]).astype(np.float32)
        t = oracle.Tree(p, m, 1, gmax=1)
        ad, _ = oracle.direct(p, m, 1e-6, idx=np.array([30]), want_pot=False)
        e0 = np.linalg.norm(t.walk(10.0, 1e-6)["acc"][30] - ad[0])
        e2 = np.linalg.norm(t.walk(10.0, 1e-6, quadrupole=True)["acc"][30] - ad[0])
        ratios.append(e2 / e0)
    assert ratios[0] < 0.5 and ratios[1] < ratios[0] and ratios[2] < ratios[1]


def test_quadrupole_walk_at_theta_zero_is_direct_summation():
    p, _, m = inputs.plummer(300, 6)
    t = oracle.Tree(p, m, 4, gmax=16)
    w = t.walk(0.0, 0.01, quadrupole=True)
    ad, pd = oracle.direct(p, m, 0.01)
    assert np.abs(w["acc"] - ad).max() <= 1e-13 * np.abs(ad).max()
    assert w["interactions"] == 300 * 300


def test_quadrupole_walk_is_more_accurate_than_monopole():
    p, _, m = inputs.plummer(3000, 7)
    t = oracle.Tree(p, m, 8, gmax=32)
    ad, _ = oracle.direct(p, m, 1e-3, want_pot=False)

    def rms(a):
        return np.sqrt(np.mean(np.sum((a - ad) ** 2, 1) / np.sum(ad ** 2, 1)))

    for theta in (0.5, 0.8):
        e0 = rms(t.walk(theta, 1e-3, want_pot=False)["acc"])
        e2 = rms(t.walk(theta, 1e-3, want_pot=False, quadrupole=True)["acc"])
        assert e2 < 0.5 * e0
