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


# ---------------------------------------------------------------- BF16 rounding model
def _bf16_bits(x):
    """bfloat16 rounding of float32 values by their bit pattern (round half
    to even on the 16 dropped bits): an independent statement of the format"""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def test_bf16_rounding_values():
    """8-bit significand, ties to even: 1 + 2^-8 lies halfway between 1 and
    1 + 2^-7 and goes to 1; 1 + 3 2^-8 lies halfway between 1 + 2^-7 and
    1 + 2^-6 and goes to 1 + 2^-6; anything above a midpoint goes up."""
    cases = [(1 + 2.0 ** -8, 1.0), (1 + 3 * 2.0 ** -8, 1 + 2.0 ** -6), (1 + 2.0 ** -8 + 2.0 ** -20, 1 + 2.0 ** -7),
             (-(1 + 2.0 ** -8 + 2.0 ** -20), -(1 + 2.0 ** -7)), (255.0, 255.0), (257.0, 256.0), (259.0, 260.0),
             (0.0, 0.0), (3.0 * 2.0 ** -100, 3.0 * 2.0 ** -100)]
    for x, want in cases:
        assert oracle.bf16(x) == want, x
    # the same as rounding the float32 bit pattern, on random floats
    v = (np.random.default_rng(7).standard_normal(20000) * 10.0 ** np.random.default_rng(8).uniform(-6, 6, 20000))
    v32 = v.astype(np.float32)
    assert np.array_equal(oracle.bf16(v32.astype(np.float64)), _bf16_bits(v32).astype(np.float64))


def test_rounding_model_hand_wired():
    """One path through the network, with a hidden value on each side of a
    BF16 rounding boundary: z1 = 1 + 2^-8 (a tie, rounds to 1) and
    z1' = 1 + 2^-8 + 2^-12 (rounds up to 1 + 2^-7); layer 2 doubles, layer 3
    sums, so y = 2 (1) + 2 (1 + 2^-7) exactly, while the exact network gives
    2 (1 + 2^-8) + 2 (1 + 2^-8 + 2^-12)."""
    W1 = np.zeros((13, H)); W1[0, 0] = 1.0; W1[0, 1] = 1.0
    b1 = np.zeros(H); b1[0] = 2.0 ** -8; b1[1] = 2.0 ** -8 + 2.0 ** -12
    W2 = np.zeros((H, H)); W2[0, 0] = 2.0; W2[1, 1] = 2.0
    W3 = np.zeros((H, 3)); W3[0, 0] = 1.0; W3[1, 0] = 1.0; W3[1, 2] = -3.0
    p = _pack(W1, b1, W2, np.zeros(H), W3, np.array([0.0, 0.25, 0.0]))
    X = np.zeros((1, 13)); X[0, 0] = 1.0
    Y, R = oracle.mlp_forward_bf16(p, X)
    assert Y[0, 0] == 2.0 + 2.0 * (1 + 2.0 ** -7)
    assert Y[0, 1] == 0.25
    assert Y[0, 2] == -6.0 * (1 + 2.0 ** -7)
    exact = oracle.mlp_forward(p, X)
    assert exact[0, 0] == 4.0 + 4.0 * 2.0 ** -8 + 2.0 * 2.0 ** -12
    # an FP32 sum can move z1 = 1 + 2^-8 off the tie: the radius admits
    # both neighbours there; exactly representable values keep a radius of
    # a few FP32 ulps only
    assert R[0, 0] >= 2.0 * 2.0 ** -7 - 1e-12
    assert R[0, 1] <= 65 * 2.0 ** -23 * 0.25
    # inputs away from any boundary: the model equals the exact network
    p2 = _pack(W1, np.zeros(H), W2, np.zeros(H), W3, np.zeros(3))
    X2 = np.zeros((1, 13)); X2[0, 0] = 1.5
    Y2, R2 = oracle.mlp_forward_bf16(p2, X2)
    assert np.array_equal(Y2, oracle.mlp_forward(p2, X2))
    assert np.all(R2 <= 65 * 2.0 ** -23 * np.abs(Y2) * (1 + 1e-12))


def _emulate_fp32(p, X):
    """An FP32-accumulating implementation of the rounding model, written
    independently in numpy: BF16 operands (bit rounding of float32), products
    exact in float32, sums added one by one in float32."""
    W1, b1, W2, b2, W3, b3 = (a.astype(np.float32) for a in _split(p))
    W1, W2, W3 = _bf16_bits(W1), _bf16_bits(W2), _bf16_bits(W3)

    def dense(a, W, b):
        z = np.broadcast_to(b, (a.shape[0], W.shape[1])).astype(np.float32).copy()
        for i in range(W.shape[0]):
            z = (z + a[:, i:i + 1] * W[i][None, :]).astype(np.float32)
        return z

    x = _bf16_bits(X.astype(np.float32))
    h1 = _bf16_bits(np.maximum(dense(x, W1, b1), 0))
    h2 = _bf16_bits(np.maximum(dense(h1, W2, b2), 0))
    return dense(h2, W3, b3).astype(np.float64), (x, h1, h2)


def test_rounding_model_radius_holds_an_fp32_implementation():
    """The FP32 emulation lands inside the model's radius on every output of
    1000 random rows, and the radius is small: a BF16 flip of a hidden unit
    is rare, so the radius is a few FP32 ulps of the output for most rows."""
    rng = np.random.default_rng(21)
    W1 = rng.standard_normal((13, H)) * np.sqrt(2 / 13)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2 / H)
    W3 = rng.standard_normal((H, 3)) * np.sqrt(1 / H)
    p = _pack(W1, rng.standard_normal(H) * 0.1, W2, rng.standard_normal(H) * 0.1, W3, rng.standard_normal(3) * 0.1)
    p = p.astype(np.float32).astype(np.float64)
    X = (rng.standard_normal((1000, 13)) * 1.5).astype(np.float32).astype(np.float64)
    Y, R = oracle.mlp_forward_bf16(p, X)
    Ye, _ = _emulate_fp32(p, X)
    assert np.all(np.abs(Ye - Y) <= R)
    scale = np.sqrt(np.mean(Y ** 2))
    assert np.median(R) <= 1e-4 * scale
    # the rounding is visible: the model is not the exact network
    Yx = oracle.mlp_forward(p, X)
    d = np.abs(Yx - Y)
    assert d.max() > 10 * np.median(R) and np.sqrt(np.mean(d ** 2)) <= 2e-2 * scale


def test_rounding_model_gradient():
    """The rounding model's gradient stays within BF16 rounding of the exact
    gradient (pinned by finite differences above), every parameter block
    included; the loss matches its own forward; an FP32 emulation of the
    backward (dY, dH2, dH1 rounded to BF16 before their products, biases
    from the unrounded values) lands inside the radius."""
    rng = np.random.default_rng(22)
    p = (rng.standard_normal(oracle.MLP_NPARAM) * 0.3).astype(np.float32).astype(np.float64)
    n = 40
    X = rng.standard_normal((n, 13)).astype(np.float32).astype(np.float64)
    T = rng.standard_normal((n, 3)).astype(np.float32).astype(np.float64)
    w = rng.uniform(0.2, 3.0, n).astype(np.float32).astype(np.float64)
    L, Lr, g, gr = oracle.mlp_grad_bf16(p, X, T, w)
    Y, _ = oracle.mlp_forward_bf16(p, X)
    assert L == pytest.approx(np.mean(w * np.sum((Y - T) ** 2, 1)), rel=1e-13)
    Lx, gx = oracle.mlp_grad(p, X, T, w)
    o = 0
    for k in (13 * H, H, H * H, H, H * 3, 3):
        blk = slice(o, o + k)
        assert np.linalg.norm(g[blk] - gx[blk]) <= 2e-2 * np.linalg.norm(gx[blk]), k
        o += k
    # FP32 emulation of the backward
    W1, b1, W2, b2, W3, b3 = (a.astype(np.float32) for a in _split(p))
    W2b, W3b = _bf16_bits(W2), _bf16_bits(W3)
    ye, (xb, h1, h2) = _emulate_fp32(p, X)
    dy = (np.float32(2) * w[:, None].astype(np.float32) * (ye.astype(np.float32) - T.astype(np.float32))
          * np.float32(1.0 / n)).astype(np.float32)
    dyb = _bf16_bits(dy)
    dh2 = np.zeros((n, H), np.float32)
    for k in range(3):
        dh2 = (dh2 + dyb[:, k:k + 1] * W3b[:, k][None, :]).astype(np.float32)
    dh2 = np.where(h2 > 0, dh2, 0).astype(np.float32)
    dh2b = _bf16_bits(dh2)
    dh1 = np.zeros((n, H), np.float32)
    for j in range(H):
        dh1 = (dh1 + dh2b[:, j:j + 1] * W2b[:, j][None, :]).astype(np.float32)
    dh1 = np.where(h1 > 0, dh1, 0).astype(np.float32)
    dh1b = _bf16_bits(dh1)

    def rowsum(a):
        s = np.zeros(a.shape[1:], np.float32)
        for r in range(a.shape[0]):
            s = (s + a[r]).astype(np.float32)
        return s

    ge = np.concatenate([rowsum(xb[:, :, None] * dh1b[:, None, :]).ravel(), rowsum(dh1).ravel(),
                         rowsum(h1[:, :, None] * dh2b[:, None, :]).ravel(), rowsum(dh2).ravel(),
                         rowsum(h2[:, :, None] * dyb[:, None, :]).ravel(), rowsum(dy).ravel()]).astype(np.float64)
    assert np.all(np.abs(ge - g) <= gr)
    # the radius is a worst case over every BF16 flip an FP32 sum can cause
    # (each flip propagates through the later roundings), yet still small
    assert np.linalg.norm(gr) <= 2e-2 * np.linalg.norm(g)


def test_rounding_model_band_sum():
    """The band sum through the rounding model selects the same cells as the
    exact network's (same evaluations and flags), stays within BF16 rounding
    of it, and with a constant network (no hidden unit reaches the output)
    equals it up to the factor's rounding."""
    n = 3000
    p, _, m = inputs.plummer(n, 31)
    t = oracle.Tree(p, m, 8, 32)
    rng = np.random.default_rng(32)
    W1 = rng.standard_normal((13, H)) * np.sqrt(2 / 13)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2 / H)
    W3 = rng.standard_normal((H, 3)) * np.sqrt(1 / H)
    params = _pack(W1, rng.standard_normal(H) * 0.1, W2, rng.standard_normal(H) * 0.1, W3,
                   rng.standard_normal(3) * 0.1).astype(np.float32).astype(np.float64)
    maps = np.concatenate([np.zeros(13), np.full(13, 0.5), np.full(3, 0.01)])
    ce, fe, ee = t.learned(0.9, 1e-2, 0.5, params, maps)
    cb, rb, fb, eb = t.learned_bf16(0.9, 1e-2, 0.5, params, maps)
    assert ee == eb > 100 and np.array_equal(fe, fb)
    assert np.all(rb >= 0)
    scale = np.sqrt(np.mean(ce ** 2))
    assert np.sqrt(np.mean((cb - ce) ** 2)) <= 2e-2 * scale
    assert np.median(rb) <= 2e-3 * scale
    const = np.zeros(oracle.MLP_NPARAM)
    const[-3:] = [1.0, -2.0, 0.5]
    c1, _, _ = t.learned(0.9, 1e-2, 0.5, const, maps)
    c2, r2, _, _ = t.learned_bf16(0.9, 1e-2, 0.5, const, maps)
    assert np.allclose(c2, c1, rtol=1e-15, atol=0)
    assert np.all(r2 <= 1e-4 * np.abs(c1) + 1e-300)
