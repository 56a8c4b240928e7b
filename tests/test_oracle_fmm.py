"""Pins of the oracle's fast multipole method (a reading of the paper's
Sec. 5, stated in oracle/tc_oracle.c): monopoles at cell centres of mass,
third-order local expansions (the field, its Jacobian, its second and third
derivatives), pair acceptance r_A + r_B < theta |c_A - c_B| with r_X the
cell's radius about its centre of mass, dual traversal, M2L / L2L / L2P and
P2P.

* Radii: every body lies within r_X of c_X for every cell X holding it, a
  leaf's radius is its farthest body (brute force).

* theta = 0 accepts no pair: every interaction is P2P, the direct sum.
* Two bodies far apart: a monopole of one body is exact, and the local
  expansion evaluated at its own centre (the other body) is exact.
* Softening much larger than the system makes every field linear in the
  positions, where monopoles and the local expansions are exact: the FMM
  then equals the direct sum at any theta, which fails if the traversal
  drops or repeats a pair of bodies.
* A far source acting on a small cluster: the local expansion's error falls
  like (cluster size)^4 / distance^6, a fourth-order remainder of a field
  falling like distance^-2 (every derivative term right); a missing or
  wrong third-derivative term would leave distance^-5, a second-derivative
  one distance^-4, the Jacobian distance^-3.
"""
import numpy as np

import oracle
from paper_1211_2293_gb300 import inputs


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_theta_zero_is_the_direct_sum():
    p, _, m = inputs.plummer(2000, 3)
    t = oracle.Tree(p, m, 8, 64)
    a, st = t.fmm(0.0, 0.01)
    ad, _ = oracle.direct(p, m, 0.01, want_pot=False)
    assert st["m2l"] == 0 and st["p2p"] > 0
    assert _rel(a, ad).max() <= 1e-13


def test_two_bodies_exact():
    p = np.array([[-0.9, -0.8, -0.85], [0.9, 0.8, 0.95]], np.float32)
    m = np.array([0.3, 1.7], np.float32)
    t = oracle.Tree(p, m, 1, 1)
    ad, _ = oracle.direct(p, m, 1e-3, want_pot=False)
    # one-body leaves have radius 0, so any theta > 0 accepts them (cube
    # sides, about 2 here against a distance of 2.5, would not at 0.3): the
    # two leaves meet each other through M2L, each meets itself in a
    # (bodiless) P2P
    for theta in (0.3, 1.5):
        a, st = t.fmm(theta, 1e-3)
        assert st["m2l"] == 2 and st["p2p"] == 2
        assert _rel(a, ad).max() <= 1e-14


def test_radii_bound_every_body():
    p, _, m = inputs.plummer(3000, 9)
    t = oracle.Tree(p, m, 8, 64)
    r = t.fmm_radii()
    xs = p.astype(np.float64)
    for v in range(t.M):
        idx = t.perm[t.first[v]:t.first[v] + t.count[v]]
        far = np.sqrt(np.sum((xs[idx] - t.com[v]) ** 2, axis=1)).max()
        if t.nchild[v] == 0:
            assert abs(r[v] - far) <= 1e-12 * max(far, 1e-300), v
        else:
            assert far <= r[v] * (1 + 1e-12), v
            kids = range(t.child_first[v], t.child_first[v] + t.nchild[v])
            assert r[v] >= max(r[k] for k in kids), v


def test_every_pair_once_linear_field_limit():
    p, _, m = inputs.plummer(1500, 4)
    t = oracle.Tree(p, m, 4, 64)
    eps = 1e4  # >> system size (cutoff 10): fields linear to (size / eps)^2 = 1e-6
    ad, _ = oracle.direct(p, m, eps, want_pot=False)
    for theta in (0.3, 0.7, 1.2):
        a, st = t.fmm(theta, eps)
        assert st["m2l"] > 0
        assert _rel(a, ad).max() <= 1e-5, theta


def test_local_expansion_third_order():
    rng = np.random.default_rng(5)
    cluster = (rng.standard_normal((8, 3)) * 0.02).astype(np.float32)
    direction = np.array([1.0, 0.3, 0.2]) / np.linalg.norm([1.0, 0.3, 0.2])
    errs = []
    for D in (2.0, 4.0, 8.0):
        src = (direction * D).astype(np.float32)[None, :]
        p = np.concatenate([cluster, src]).astype(np.float32)
        m = np.concatenate([np.full(8, 1e-3), [1.0]]).astype(np.float32)
        t = oracle.Tree(p, m, 8, 1)
        a, st = t.fmm(1.5, 1e-4)
        assert st["m2l"] > 0
        # the source's field on the cluster: the cluster's own pairs are P2P
        # (exact), so the FMM error is the local expansion's
        ad, _ = oracle.direct(p, m, 1e-4, want_pot=False)
        errs.append(np.abs(a[:8] - ad[:8]).max())
    # the far field is G M / D^2; the first term a third-order expansion
    # drops is (cluster size)^4 G M / D^6, so each doubling of D divides the
    # error by 64 -- by 32 if the third derivatives were missing or wrong,
    # 16 without the second, 8 without the Jacobian
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 48.0 < r1 < 80.0 and 48.0 < r2 < 80.0, errs


def test_error_shrinks_with_theta():
    p, _, m = inputs.plummer(4000, 6)
    t = oracle.Tree(p, m, 8, 64)
    ad, _ = oracle.direct(p, m, 0.01, want_pot=False)
    rms = []
    for theta in (0.6, 0.3, 0.2):
        a, _ = t.fmm(theta, 0.01)
        rms.append(float(np.sqrt(np.mean(_rel(a, ad) ** 2))))
    assert rms[1] < rms[0] / 3 and rms[2] < rms[1] and rms[2] < 1e-3, rms


def test_per_target_records_sum_to_the_totals_and_flags_reach_the_subtree():
    p, _, m = inputs.plummer(6000, 8)
    t = oracle.Tree(p, m, 8, 64)
    a0, st0 = t.fmm(0.5, 0.01)
    a, st = t.fmm(0.5, 0.01, per_node=True)
    assert np.array_equal(a, a0)
    assert st["nm2l"].sum() == st0["m2l"] and st["np2p"].sum() == st0["p2p"]
    assert int(st["hm2l"].sum(dtype=np.uint64)) == st0["m2l_hash"]
    assert int(st["hp2p"].sum(dtype=np.uint64)) == st0["p2p_hash"]
    # a leaf's self pair is a P2P with itself as target
    leaves = np.where(t.nchild == 0)[0]
    assert np.all(st["np2p"][leaves] >= 1)
    # flags: a flagged parent flags all its children
    par = t.parent[1:]
    assert np.all(st["flag"][1:][st["flag"][par] == 1] == 1)
    assert (st0["ties"] == 0) == (st["flag"].sum() == 0)
