"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the force
law of Sec. 3.1 (golden values), closed forms (two-body, Kepler orbit,
Plummer virial energies), brute force on tiny inputs (recursive subdivision
by geometry, maximal accepted cells), invariants (partition of bodies,
masses, centre of mass inside its cube) and special cases (theta = 0 reduces
the treecode to direct summation).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs
from tests.helpers import cube_of, deinterleave, mix64, rel_err_rms

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_bodies(n, seed, scale=1.0, offset=0.0):
    rng = np.random.default_rng(seed)
    pos = (rng.standard_normal((n, 3)) * scale + offset).astype(np.float32)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    return pos, mass


# ---------------------------------------------------------------- root cube
@pytest.mark.parametrize("seed,scale,offset", [(0, 1.0, 0.0), (1, 1e-3, 5.0), (2, 100.0, -7.0)])
def test_root_cube_contains_all_bodies(seed, scale, offset):
    pos, _ = _random_bodies(500, seed, scale, offset)
    c0, L, h = oracle.root_cube(pos)
    m, e = math.frexp(L)
    assert m == 0.5, "side is a power of two"
    assert h == L / 2 ** 21
    p = pos.astype(np.float64)
    lo, hi = p.min(0), p.max(0)
    assert np.all(np.floor(c0 / h) * h == c0), "corner on the grid"
    assert np.all(c0 <= lo) and np.all(c0 > lo - h)
    assert np.all(hi < c0 + L), "largest body strictly inside"
    assert (hi - lo).max() * (1 + 2 ** -20) <= L < 2 * (hi - lo).max() * (1 + 2 ** -20)


def test_root_cube_degenerate():
    c0, L, h = oracle.root_cube(np.array([[0.25, -3.0, 7.0]], np.float32))
    assert L == 1.0 and np.all(c0 <= [0.25, -3.0, 7.0])
    with pytest.raises(ValueError):
        oracle.root_cube(np.array([[np.nan, 0, 0]], np.float32))


# ---------------------------------------------------------------- keys
def test_keys_match_geometric_descent():
    """Key digits = octant of the body at each level, found by comparing the
    body with the centre of its cube while descending (no bit tricks)."""
    pos, _ = _random_bodies(300, 3)
    c0, L, h = oracle.root_cube(pos)
    keys = oracle.morton_keys(pos, np.r_[c0, L, h])
    for i in range(pos.shape[0]):
        corner = c0.copy()
        side = L
        k = 0
        for lev in range(1, 22):
            side /= 2
            octant = 0
            for a, w in ((0, 4), (1, 2), (2, 1)):
                if float(pos[i, a]) >= corner[a] + side:
                    octant += w
                    corner[a] += side
            k = (k << 3) | octant
        assert int(keys[i]) == k


# ---------------------------------------------------------------- tree
def _brute_subdivide(pos, c0, L, leaf_max):
    """Recursive subdivision of the cube by geometry (Sec. 3.1)."""
    out = {}

    def rec(idx, corner, side, level):
        out[(level, tuple(np.round(corner / side).astype(np.int64)))] = len(idx)
        if len(idx) <= leaf_max or level == 21:
            return
        half = side / 2
        for o in range(8):
            bits = ((o >> 2) & 1, (o >> 1) & 1, o & 1)
            cc = corner + half * np.array(bits, dtype=np.float64)
            sel = [i for i in idx if all((pos[i, a] >= cc[a]) and (pos[i, a] < cc[a] + half) for a in range(3))]
            if sel:
                rec(sel, cc, half, level + 1)

    rec(list(range(pos.shape[0])), c0.copy(), L, 0)
    return out


@pytest.mark.parametrize("n,leaf_max,seed", [(1, 1, 0), (2, 1, 1), (9, 8, 2), (17, 4, 3), (200, 3, 4), (300, 8, 5)])
def test_tree_equals_geometric_subdivision(n, leaf_max, seed):
    pos, mass = _random_bodies(n, seed)
    t = oracle.Tree(pos, mass, leaf_max)
    p64 = pos.astype(np.float64)
    brute = _brute_subdivide(p64, t.c0, t.L, leaf_max)
    mine = {}
    for v in range(t.M):
        corner, side = cube_of(t, v)
        key = (int(t.level[v]), tuple(np.round((corner - t.c0 + 0) / side).astype(np.int64)))
        # brute keys are corner/side in absolute units: shift both by c0
        mine[key] = int(t.count[v])
    brute_rel = {}
    for (lev, ijk), c in brute.items():
        side = np.ldexp(t.L, -lev)
        rel = tuple(int(round(ijk[a] - t.c0[a] / side)) for a in range(3))
        brute_rel[(lev, rel)] = c
    assert mine == brute_rel


def _check_invariants(t, pos, mass):
    n = pos.shape[0]
    p = pos.astype(np.float64)[t.perm]
    m = mass.astype(np.float64)[t.perm]
    assert sorted(t.perm.tolist()) == list(range(n)), "perm is a permutation"
    assert np.all(np.diff(t.keys.astype(np.uint64).view(np.int64)) >= 0) or np.all(t.keys[1:] >= t.keys[:-1])
    ties = t.keys[1:] == t.keys[:-1]
    assert np.all(t.perm[1:][ties] > t.perm[:-1][ties]), "stable order of equal keys"
    # breadth-first order, children contiguous and in octant order
    order = np.lexsort((t.first, t.level))
    assert np.all(order == np.arange(t.M))
    leaves = np.where(t.nchild == 0)[0]
    cover = np.zeros(n, dtype=np.int64)
    for v in leaves:
        cover[t.first[v]:t.first[v] + t.count[v]] += 1
    assert np.all(cover == 1), "every body in exactly one leaf"
    for v in range(t.M):
        if t.nchild[v] == 0:
            assert t.count[v] <= t.leaf_max or t.level[v] == 21
        else:
            assert t.count[v] > t.leaf_max and t.level[v] < 21
            cs = np.arange(t.child_first[v], t.child_first[v] + t.nchild[v])
            assert np.all(t.parent[cs] == v)
            assert t.count[cs].sum() == t.count[v]
            assert t.first[cs[0]] == t.first[v]
            assert np.all(t.first[cs[1:]] == t.first[cs[:-1]] + t.count[cs[:-1]])
            assert np.all(t.level[cs] == t.level[v] + 1)
            digits = (t.prefix[cs] & np.uint64(7)).astype(int)
            assert np.all(np.diff(digits) > 0)
            assert np.all((t.prefix[cs] >> np.uint64(3)) == t.prefix[v])
        sl = slice(t.first[v], t.first[v] + t.count[v])
        msum = m[sl].sum()
        assert abs(t.node_mass[v] - msum) <= 1e-15 * msum * max(1, math.log2(t.count[v] + 1))
        corner, side = cube_of(t, v)
        # every body of the cell lies inside the cell's cube (to one FP64 ulp)
        tol = 2 * np.spacing(np.abs(corner) + side)
        assert np.all(p[sl] >= corner - tol) and np.all(p[sl] < corner + side + tol)
        assert np.all(t.com[v] >= corner - tol) and np.all(t.com[v] <= corner + side + tol)
        ref_com = (m[sl, None] * p[sl]).sum(0) / msum
        assert np.allclose(t.com[v], ref_com, rtol=0, atol=1e-13 * (np.abs(ref_com).max() + side))
        q = t.quad[v]
        Q = np.array([[q[0], q[1], q[2]], [q[1], q[3], q[4]], [q[2], q[4], q[5]]])
        assert np.linalg.eigvalsh(Q).min() >= -1e-12 * (abs(Q).max() + 1e-300)
    assert t.parent[0] == -1 and t.level[0] == 0 and t.count[0] == n


@pytest.mark.parametrize("maker,n,leaf,seed", [
    ("plummer", 4096, 8, 0), ("uniform", 3000, 16, 1), ("random", 777, 1, 2), ("random", 50, 64, 3)])
def test_tree_invariants(maker, n, leaf, seed):
    if maker == "plummer":
        pos, _, mass = inputs.plummer(n, seed)
    elif maker == "uniform":
        pos, _, mass = inputs.uniform_cube(n, seed)
    else:
        pos, mass = _random_bodies(n, seed)
    t = oracle.Tree(pos, mass, leaf)
    _check_invariants(t, pos, mass)


def test_coincident_bodies_make_a_level21_leaf():
    pos = np.zeros((40, 3), np.float32)
    pos[:20] = [0.5, 0.5, 0.5]
    pos[20:] = [-0.25, 0.75, 0.125]
    mass = np.ones(40, np.float32)
    t = oracle.Tree(pos, mass, 4)
    leaves = np.where(t.nchild == 0)[0]
    assert len(leaves) == 2
    assert np.all(t.level[leaves] == 21) and np.all(t.count[leaves] == 20)
    _check_invariants(t, pos, mass)


# ---------------------------------------------------------------- groups
@pytest.mark.parametrize("gmax,leaf", [(1, 8), (7, 8), (64, 8), (64, 16), (32, 64), (100000, 8)])
def test_groups_partition_and_packing(gmax, leaf):
    pos, _, mass = inputs.plummer(3000, 4)
    t = oracle.Tree(pos, mass, leaf, gmax)
    assert t.gfirst[0] == 0
    assert np.all(t.gfirst[1:] == t.gfirst[:-1] + t.gcount[:-1])
    assert t.gfirst[-1] + t.gcount[-1] == t.n
    assert np.all(t.gcount >= 1) and np.all(t.gcount <= gmax)
    for g in range(t.G):
        r = t.gref[g]
        assert t.first[r] <= t.gfirst[g] and t.gfirst[g] + t.gcount[g] <= t.first[r] + t.count[r]
    if gmax == 1:
        assert t.G == t.n
    if gmax >= t.n:
        assert t.G == 1
    # greedy packing: two neighbouring groups made of children of the same
    # parent could not have been merged
    for g in range(t.G - 1):
        a, b = t.gref[g], t.gref[g + 1]
        pa = a if t.count[a] > gmax else t.parent[a]
        pb = b if t.count[b] > gmax else t.parent[b]
        if pa == pb and t.count[pa] > gmax and t.nchild[pa] > 0:
            assert t.gcount[g] + t.gcount[g + 1] > gmax or t.count[a] > gmax


# ---------------------------------------------------------------- forces
def _golden_force_law():
    rows = []
    with open(os.path.join(GOLDEN, "two_body_force_law.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _golden_force_law())
def test_two_body_matches_paper_force_law(row):
    G, ma, mb, r, F = row
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    mass = np.array([ma, mb])
    acc, pot = oracle.direct(pos, mass, eps=r * 1e-9, G=G)
    assert acc[0, 0] * ma == pytest.approx(F, rel=1e-12)
    assert acc[1, 0] * mb == pytest.approx(-F, rel=1e-12)
    assert np.all(acc[:, 1:] == 0)
    assert pot[0] == pytest.approx(-G * mb / r, rel=1e-12)


def test_two_body_softened_tree_equals_closed_form():
    """Through the tree path (float32 inputs, leaf 1): the Plummer-softened
    two-body acceleration G m r / (r^2 + eps^2)^(3/2), equal and opposite."""
    pos = np.array([[0.5, 0.25, -1.0], [-0.75, 0.5, 0.25]], np.float32)
    mass = np.array([2.0, 0.5], np.float32)
    eps, G = 0.125, 1.5
    for theta in (0.0, 0.5, 10.0):
        acc, pot, t, w = oracle.tree_forces(pos, mass, theta, eps, G, leaf_max=1, gmax=1)
        r = pos.astype(np.float64)[1] - pos.astype(np.float64)[0]
        d2 = (r ** 2).sum() + eps ** 2
        a0 = G * 0.5 * r / d2 ** 1.5
        assert np.allclose(acc[0], a0, rtol=1e-14, atol=0)
        assert np.allclose(acc[1], -a0 * 2.0 / 0.5, rtol=1e-14, atol=0)
        assert pot[0] == pytest.approx(-G * 0.5 / math.sqrt(d2), rel=1e-14)


@pytest.mark.parametrize("maker,n,leaf,gmax", [("plummer", 1000, 8, 64), ("random", 513, 4, 16), ("uniform", 700, 16, 1)])
def test_theta_zero_is_direct_summation(maker, n, leaf, gmax):
    if maker == "plummer":
        pos, _, mass = inputs.plummer(n, 1)
    elif maker == "uniform":
        pos, _, mass = inputs.uniform_cube(n, 2)
    else:
        pos, mass = _random_bodies(n, 5)
    acc, pot, t, w = oracle.tree_forces(pos, mass, 0.0, 0.01, 1.0, leaf_max=leaf, gmax=gmax)
    assert np.all(w["ncell"] == 0) and np.all(w["nbody"] == n)
    ad, pd = oracle.direct(pos, mass, 0.01, 1.0)
    scale = np.abs(ad).max()
    assert np.abs(acc - ad).max() <= 1e-13 * scale
    assert np.abs(pot - pd).max() <= 1e-13 * np.abs(pd).max()


def test_direct_sum_conserves_momentum():
    pos, mass = _random_bodies(400, 7)
    acc, _ = oracle.direct(pos, mass, 0.05)
    fsum = (mass.astype(np.float64)[:, None] * acc).sum(0)
    fabs = (mass.astype(np.float64)[:, None] * np.abs(acc)).sum(0)
    assert np.all(np.abs(fsum) <= 1e-13 * fabs)


def test_tree_error_grows_with_theta_and_is_small():
    pos, _, mass = inputs.plummer(2048, 11)
    ad, _ = oracle.direct(pos, mass, 0.01)
    errs = []
    for th in (0.2, 0.4, 0.6, 0.8):
        acc, _, _, _ = oracle.tree_forces(pos, mass, th, 0.01, leaf_max=8, gmax=64)
        errs.append(rel_err_rms(acc, ad))
    assert all(a < b for a, b in zip(errs, errs[1:]))
    assert errs[0] < 1e-4 and errs[1] < 1e-3


# ---------------------------------------------------------------- walk lists
def _maximal_sets(t, g, theta):
    """Brute force: accepted cells whose ancestors were all opened, and
    leaves that were opened with all their ancestors."""
    dec = np.array([t.test(g, v, theta) for v in range(t.M)])
    opened = dec != 2
    ok = np.zeros(t.M, bool)
    for v in range(t.M):
        p = t.parent[v]
        good = True
        while p >= 0:
            if not opened[p]:
                good = False
                break
            p = t.parent[p]
        ok[v] = good
    cells = [v for v in range(1, t.M) if ok[v] and dec[v] == 2]
    leaves = [v for v in range(t.M) if ok[v] and opened[v] and t.nchild[v] == 0]
    return cells, leaves


@pytest.mark.parametrize("n,leaf,gmax,theta", [(300, 4, 16, 0.5), (512, 8, 64, 0.7), (200, 1, 1, 0.6), (150, 2, 8, 1.2)])
def test_walk_lists_equal_brute_force(n, leaf, gmax, theta):
    pos, _, mass = inputs.plummer(n, 21)
    t = oracle.Tree(pos, mass, leaf, gmax)
    w = t.walk(theta, 0.01)
    for g in range(t.G):
        cells, leaves = _maximal_sets(t, g, theta)
        assert w["ncell"][g] == len(cells)
        assert w["nbody"][g] == sum(int(t.count[v]) for v in leaves)
        h = sum(mix64(2 * c + 1) for c in cells) + sum(mix64(2 * v + 2) for v in leaves)
        assert int(w["hash"][g]) == h % (1 << 64)
        # the accepted cells and opened leaves partition all bodies
        cover = np.zeros(n, int)
        for v in cells + leaves:
            cover[t.first[v]:t.first[v] + t.count[v]] += 1
        assert np.all(cover == 1)
        # no accepted cell holds a body of the group
        for c in cells:
            assert t.first[c] + t.count[c] <= t.gfirst[g] or t.first[c] >= t.gfirst[g] + t.gcount[g]


def test_opening_test_is_strict_and_flags_ties():
    """s < theta*d strictly: at s == theta*d the cell is opened and the
    group is flagged as a tie."""
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]], np.float32)
    mass = np.ones(2, np.float32)
    t = oracle.Tree(pos, mass, 1, 1)
    assert t.L == 2.0
    other = [v for v in range(t.M) if t.level[v] == 1 and t.first[v] == 1][0]
    assert t.side(other) == 1.0
    w = t.walk(1.0, 0.01)
    assert w["ncell"][0] == 0 and w["flag"][0] == 1
    w = t.walk(1.0 + 1e-7, 0.01)
    assert w["ncell"][0] == 1 and w["flag"][0] == 1
    w = t.walk(1.1, 0.01)
    assert w["ncell"][0] == 1 and w["flag"][0] == 0


# ---------------------------------------------------------------- dynamics
def test_leapfrog_circular_kepler_orbit():
    """Two equal masses 1/2 on a circular orbit of separation 1 (G = 1):
    speeds 1/2, period 2 pi.  After one period the KDK leapfrog returns to
    the start to O(dt^2) and conserves angular momentum to rounding."""
    pos = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    vel = np.array([[0.0, 0.5, 0.0], [0.0, -0.5, 0.0]])
    mass = np.array([0.5, 0.5])
    nsteps = 2000
    dt = 2 * math.pi / nsteps
    p1, v1 = oracle.leapfrog_direct(pos, vel, mass, 1e-9, 1.0, dt, nsteps)
    assert np.abs(p1 - pos).max() < 5e-5
    d0 = oracle.diag(pos, vel, mass)
    d1 = oracle.diag(p1, v1, mass)
    assert np.abs(d1[5:] - d0[5:]).max() < 1e-14
    # the phase error of leapfrog on a circular orbit scales as dt^2
    p2, _ = oracle.leapfrog_direct(pos, vel, mass, 1e-9, 1.0, 2 * dt, nsteps // 2)
    e1, e2 = np.abs(p1 - pos).max(), np.abs(p2 - pos).max()
    assert 3.5 < e2 / e1 < 4.5


def test_leapfrog_time_reversible():
    pos, vel, mass = inputs.plummer(32, 5)
    p1, v1 = oracle.leapfrog_direct(pos, vel, mass, 0.05, 1.0, 1e-3, 50)
    p2, v2 = oracle.leapfrog_direct(p1, -v1, mass, 0.05, 1.0, 1e-3, 50)
    assert np.abs(p2 - pos.astype(np.float64)).max() < 1e-12
    assert np.abs(-v2 - vel.astype(np.float64)).max() < 1e-12


def test_diag_two_body_energy():
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    vel = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    mass = np.array([2.0, 1.0])
    _, pot = oracle.direct(pos, mass, 1e-12, 1.0)
    d = oracle.diag(pos, vel, mass, pot)
    assert d[0] == pytest.approx(0.5 * 2 * 1 + 0.5 * 1 * 4)
    assert d[1] == pytest.approx(-2.0 * 1.0 / 5.0, rel=1e-12)
    assert np.allclose(d[2:5], [2.0, 2.0, 0.0])
    assert np.allclose(d[5:], [0.0, 0.0, 3.0 * 2.0 - 4.0 * 0.0])


def test_energy_drift_small_with_tree_forces():
    """KDK with tree forces (theta 0.5) on a Plummer sphere: the relative
    energy change over 20 steps stays small (it is O(dt^2) plus the
    treecode's force error)."""
    pos, vel, mass = inputs.plummer(1024, 8)
    eps, dt = 0.01, 1e-3
    p = pos.astype(np.float64)
    v = vel.astype(np.float64)
    acc, pot, _, _ = oracle.tree_forces(p.astype(np.float32), mass, 0.5, eps)
    e0 = oracle.diag(p, v, mass, pot)
    for _ in range(20):
        v = oracle.kick(v, acc, dt / 2)
        p = oracle.drift(p, v, dt)
        acc, pot, _, _ = oracle.tree_forces(p.astype(np.float32), mass, 0.5, eps)
        v = oracle.kick(v, acc, dt / 2)
    e1 = oracle.diag(p, v, mass, pot)
    E0, E1 = e0[0] + e0[1], e1[0] + e1[1]
    assert abs(E1 - E0) / abs(E0) < 2e-4


# ---------------------------------------------------------------- inputs
def test_plummer_generator_matches_closed_forms():
    """Plummer (a = M = G = 1): enclosed mass r^3 / (1 + r^2)^(3/2)
    (Kolmogorov-Smirnov), potential energy -3 pi / 32 and kinetic energy
    3 pi / 64 (virial equilibrium), up to sampling noise and the r <= 10 cut."""
    pos, vel, mass = inputs.plummer(4096, 3)
    r = np.sqrt((pos.astype(np.float64) ** 2).sum(1))
    rs = np.sort(r)
    cdf = rs ** 3 / (1 + rs ** 2) ** 1.5 / (1000 / 101 ** 1.5)
    ecdf = np.arange(1, r.size + 1) / r.size
    assert np.abs(cdf - ecdf).max() < 1.63 / math.sqrt(r.size)  # KS at 1 %
    _, pot = oracle.direct(pos, mass, 1e-4)
    d = oracle.diag(pos, vel, mass, pot)
    assert d[1] == pytest.approx(-3 * math.pi / 32, rel=0.05)
    assert d[0] == pytest.approx(3 * math.pi / 64, rel=0.05)


def test_group_list_export_partitions_the_bodies():
    """A group's exported list (accepted cells + opened leaves) covers every
    body exactly once and is the set the walk's hash and lengths describe."""
    from tests.helpers import mix64

    p, _, m = inputs.plummer(600, 31)
    t = oracle.Tree(p, m, 4, gmax=16)
    w = t.walk(0.7, 0.01)
    for g in (0, 5, t.G // 2, t.G - 1):
        cells, leaves = t.group_list(g, 0.7)
        assert len(cells) == w["ncell"][g]
        assert int(t.count[leaves].sum()) == w["nbody"][g]
        cover = np.zeros(t.n, np.int64)
        for v in list(cells) + list(leaves):
            cover[t.first[v]:t.first[v] + t.count[v]] += 1
        assert np.all(cover == 1)
        h = sum(mix64(2 * int(v) + 1) for v in cells) + sum(mix64(2 * int(v) + 2) for v in leaves)
        assert (h % (1 << 64)) == int(w["hash"][g])
