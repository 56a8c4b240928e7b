"""Learned far-field correction on the GPU against the FP64 oracle.

The network runs with BF16 operands and FP32 accumulation.  Its oracle is
the network's BF16 rounding model (oracle.mlp_forward_bf16 /
mlp_grad_bf16 / Tree.learned_bf16): the same operands rounded to BF16 at
the same points, sums exact, and beside every value the radius within which
an implementation making those roundings on FP32 sums must land (each FP32
addition off by at most one ulp of the largest partial sum; a BF16 rounding
whose input interval straddles a boundary admits both neighbours).  Every
output, gradient element and per-body correction is compared element by
element with its radius; the gradients also meet the 1e-2 norm-relative
bar per parameter block.

Inside the walk: a zero network leaves the forces bit-identical to the plain
precise walk; a constant network gives c * sum(G M s^2 / r^4) over the band
cells of each group (float geometry: 1e-4 relative); a random network is
compared with the rounding model's band sum of the same network, its
features computed in FP64 at the same point with the radius of their FP32
evaluation.  Training pairs (features and exact labels) are compared with
the oracle's definitions at the same (body, cell).
"""
import numpy as np
import pytest

import oracle
from paper_1211_2293_gb300 import inputs

pytestmark = pytest.mark.gpu

H = 64
NP = oracle.MLP_NPARAM


def bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _weights_bf16(params):
    p = np.asarray(params, np.float32).copy()
    o = 0
    for shape, is_w in (((13, H), True), ((H,), False), ((H, H), True), ((H,), False), ((H, 3), True),
                        ((3,), False)):
        k = int(np.prod(shape))
        if is_w:
            p[o:o + k] = bf16(p[o:o + k])
        o += k
    return p.astype(np.float64)


def _random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((13, H)) * np.sqrt(2 / 13) * scale
    b1 = rng.standard_normal(H) * 0.1
    W2 = rng.standard_normal((H, H)) * np.sqrt(2 / H) * scale
    b2 = rng.standard_normal(H) * 0.1
    W3 = rng.standard_normal((H, 3)) * np.sqrt(1 / H)
    b3 = rng.standard_normal(3) * 0.1
    return np.concatenate([a.ravel() for a in (W1, b1, W2, b2, W3, b3)]).astype(np.float32)


def _model(params, mean, scale, yscale):
    return np.concatenate([params, mean, scale, yscale]).astype(np.float32)


def _normalised_bf16(X, mean, scale):
    X32 = np.asarray(X, np.float32)
    return bf16((X32 - np.float32(mean)) * np.float32(scale)).astype(np.float64)


def _features(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 13)).astype(np.float32) * 2.0 + 0.5
    return X


def _normalised_f32(X, mean, scale):
    """(x - mean) * scale with each operation rounded to float32, as the
    library normalises features"""
    X32 = np.asarray(X, np.float32)
    return ((X32 - np.float32(mean)) * np.float32(scale)).astype(np.float32).astype(np.float64)


def _p64(params):
    return np.asarray(params, np.float32).astype(np.float64)


def test_forward_matches_oracle(tc):
    """Every output within the rounding model's radius (plus the final
    float32 scaling); the radius is a few FP32 ulps for most rows."""
    n = 1000  # 62 full 16-row tiles and a ragged tail of 8
    X = _features(n, 1)
    params = _random_params(2)
    mean = X.mean(0).astype(np.float32)
    scale = (1 / X.std(0)).astype(np.float32)
    yscale = np.array([0.5, 2.0, 1.0], np.float32)
    ctx = tc.Context()
    ctx.mlp_set(_model(params, mean, scale, yscale), band=0.5)
    Y = ctx.mlp_forward(X).astype(np.float64)
    Ym, R = oracle.mlp_forward_bf16(_p64(params), _normalised_f32(X, mean, scale))
    ys = yscale.astype(np.float64)
    Yo = Ym * ys
    bound = R * np.abs(ys) + 2.0 ** -24 * np.abs(Yo)
    err = np.abs(Y - Yo)
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()
    rms = np.sqrt(np.mean(Yo ** 2))
    assert np.median(bound) <= 1e-4 * rms
    print(f"forward: max |err| {err.max():.3e}, max bound {bound.max():.3e}, output rms {rms:.3e}")
    # one row, and the model read back unchanged
    assert np.allclose(ctx.mlp_forward(X[:1]), Y[:1], rtol=0, atol=0)
    m, band = ctx.mlp_get()
    assert band == 0.5 and np.array_equal(m, _model(params, mean, scale, yscale))


def test_loss_and_gradient_match_oracle(tc):
    """Loss and every gradient element within the rounding model's radius,
    with and without per-pair weights; each parameter block within 1e-2
    (norm-relative) of the model's gradient."""
    n = 200  # 12 tiles + 8 rows
    X = _features(n, 3)
    params = _random_params(4)
    mean = X.mean(0).astype(np.float32)
    scale = (1 / X.std(0)).astype(np.float32)
    yscale = np.array([0.5, 2.0, 1.0], np.float32)
    T = np.random.default_rng(5).standard_normal((n, 3)).astype(np.float32)
    W = np.random.default_rng(6).uniform(0.2, 3.0, n).astype(np.float32)
    Ts = (T / yscale).astype(np.float32).astype(np.float64)  # the library's float32 target scaling
    ctx = tc.Context()
    ctx.mlp_set(_model(params, mean, scale, yscale), band=0.5)
    Xn = _normalised_f32(X, mean, scale)
    for w in (None, W):
        loss, g = ctx.mlp_loss_grad(X, T, w)
        Lo, Lr, go, gr = oracle.mlp_grad_bf16(_p64(params), Xn, Ts, None if w is None else w.astype(np.float64))
        assert abs(loss - Lo) <= Lr + 2.0 ** -22 * abs(Lo)
        g = g.astype(np.float64)
        err = np.abs(g - go)
        # the GPU sums its float32 tile partial sums with atomics, in no set
        # order: covered by the radius's FP32 accumulation over the rows
        assert np.all(err <= gr), (err / np.maximum(gr, 1e-300)).max()
        o = 0
        for k in (13 * H, H, H * H, H, H * 3, 3):
            blk = slice(o, o + k)
            assert np.linalg.norm(g[blk] - go[blk]) <= 1e-2 * np.linalg.norm(go[blk]), k
            o += k
        print(f"gradient: norm-relative error {np.linalg.norm(g - go) / np.linalg.norm(go):.2e}, "
              f"radius {np.linalg.norm(gr) / np.linalg.norm(go):.2e}")


def _built(tc, n, seed, leaf=16, gmax=64, split=0):
    p, _, m = inputs.plummer(n, seed)
    # the plain walk the learned one is compared with runs on the same kernel
    # (split 0: one warp per group, the network inside the walk; 2: producer
    # and consumer warps, the network after the walk), so the walk's own sums
    # agree bit for bit
    ctx = tc.Context(gmax=gmax, precise=1, quad=1, want_pot=0, verify=1, split=split)
    ctx.build(p, m, leaf)
    return ctx, p, m


@pytest.mark.parametrize("split", [0, 2])
def test_zero_model_leaves_forces_bit_identical(tc, split):
    ctx, p, m = _built(tc, 20000, 6, split=split)
    ctx.forces(0.9, 1e-3)
    a0 = ctx.get_acc().copy()
    ctx.mlp_set(np.zeros(tc.MLP_NMODEL, np.float32), band=0.3)
    ctx.set_config(learned=1)
    ctx.mlp_evals()
    ctx.forces(0.9, 1e-3)
    a1 = ctx.get_acc()
    assert np.array_equal(a0, a1)
    assert ctx.mlp_evals() > 0


def _compare_band_sum(ctx, p, m, theta, eps, G, band, params, maps, rel=None, leaf=16, gmax=64):
    """GPU correction (learned walk minus plain walk) against the oracle's
    band sum, per body of every unflagged group: with rel, the exact network
    within rel of |corr|; without, the rounding model within its radius.
    Either way one float32 rounding of each walk's result is added."""
    ctx.set_config(learned=0)
    ctx.forces(theta, eps, G)
    a0 = ctx.get_acc().astype(np.float64)
    ctx.set_config(learned=1)
    ctx.mlp_evals()
    ctx.forces(theta, eps, G)
    a1 = ctx.get_acc().astype(np.float64)
    evals = ctx.mlp_evals()
    t = oracle.Tree(p, m, leaf, gmax=gmax)
    if rel is None:
        corr, crad, flag, ev = t.learned_bf16(theta, eps, band, _p64(params), maps, G=G)
    else:
        corr, flag, ev = t.learned(theta, eps, band, params, maps, G=G)
        crad = rel * np.abs(corr)
    # bodies of groups with no test near a bound
    ok = np.zeros(t.n, bool)
    for g in np.where(flag == 0)[0]:
        ok[t.perm[t.gfirst[g]:t.gfirst[g] + t.gcount[g]]] = True
    assert ok.mean() > 0.9
    d = (a1 - a0)[ok]
    c = corr[ok]
    bound = crad[ok] + 2.0 ** -24 * (np.abs(a1[ok]) + np.abs(a0[ok]))
    assert np.all(np.abs(d - c) <= bound), (np.abs(d - c) / bound).max()
    if (flag == 0).all():
        assert evals == ev
    else:
        assert abs(evals - ev) <= 0.02 * ev
    return d, c, bound


@pytest.mark.parametrize("split", [0, 2])
def test_constant_model_matches_oracle_band_sum(tc, split):
    ctx, p, m = _built(tc, 20000, 7, split=split)
    cvec = np.array([1.0, -0.5, 2.0], np.float32)
    params = np.zeros(NP, np.float32)
    params[-3:] = cvec
    maps = np.concatenate([np.zeros(13), np.ones(13), np.full(3, 0.01)]).astype(np.float32)
    ctx.mlp_set(np.concatenate([params, maps]), band=0.5)
    _compare_band_sum(ctx, p, m, 0.9, 1e-3, 1.3, 0.5, params, maps, rel=1e-4)


@pytest.mark.parametrize("split", [0, 2])
def test_random_model_matches_oracle_band_sum(tc, split):
    ctx, p, m = _built(tc, 16384, 8, split=split)
    # maps from real features of the same system
    X, T, _, _, _ = ctx.mlp_pairs(0.9, 1e-3, 0.4, 0.2, 11, 50000)
    assert len(X) > 1000
    mean = X.mean(0)
    sd = X.std(0)
    scale = np.where(sd > 0, 1 / np.maximum(sd, 1e-30), 0).astype(np.float32)
    yscale = np.sqrt(np.mean(T.astype(np.float64) ** 2, 0)).astype(np.float32)
    params = _random_params(12)
    maps = np.concatenate([mean, scale, yscale]).astype(np.float32)
    ctx.mlp_set(np.concatenate([params, maps]), band=0.4)
    d, c, bound = _compare_band_sum(ctx, p, m, 0.9, 1e-3, 1.0, 0.4, params, maps)
    rms = np.sqrt(np.mean(c ** 2))
    print(f"band sum: max |err| {np.abs(d - c).max():.3e}, median bound {np.median(bound):.3e}, corr rms {rms:.3e}")
    assert np.median(bound) <= 2e-2 * rms


def test_training_pairs_match_oracle(tc):
    n = 20000
    ctx, p, m = _built(tc, n, 9)
    theta, eps, band = 0.9, 2e-3, 0.5
    X, T, F, body, node = ctx.mlp_pairs(theta, eps, band, 0.05, 13, 100000)
    assert 1000 < len(X) < 100000
    t = oracle.Tree(p, m, 16, gmax=64)
    inv = np.empty(n, np.int64)
    inv[t.perm] = np.arange(n)
    msys = float(t.node_mass[0])
    rng = np.random.default_rng(0)
    for k in rng.choice(len(X), 300, replace=False):
        b, v = int(body[k]), int(node[k])
        x = p[b].astype(np.float64)
        f = t.mlp_features(v, x, eps, msys)
        lab = t.mlp_label(v, x, eps)
        assert np.allclose(X[k][:7], f[:7], rtol=2e-6, atol=2e-6 * np.abs(f[:4]).max())
        # moment ratios from FP32 second moments: (leaf_max + 128) 2^-25
        assert np.allclose(X[k][7:], f[7:], rtol=2e-6, atol=(16 + 128) * 2.0 ** -25)
        assert np.allclose(T[k], lab, rtol=1e-5, atol=1e-5 * np.abs(lab).max())
        assert F[k] == pytest.approx(t.mlp_factor(v, x), rel=1e-6)
        # the pair is a band cell accepted by the body's group
        g = int(np.searchsorted(t.gfirst, inv[b], side="right") - 1)
        assert t.test(g, v, theta) == 2
        assert t.count[v] >= 2
    # sampling: about prob x (number of band cells), reproducible by seed
    X2, T2, F2, b2, v2 = ctx.mlp_pairs(theta, eps, band, 0.05, 13, 100000)
    # one order: by the body's position in the tree (the oracle's tree has
    # the same permutation), then node
    assert np.all(np.diff(inv[body] * (1 << 32) + node) > 0)
    assert np.array_equal(body, b2) and np.array_equal(node, v2)
    assert np.array_equal(X, X2) and np.array_equal(T, T2) and np.array_equal(F, F2)
    Xa, _, _, _, _ = ctx.mlp_pairs(theta, eps, band, 1.0, 13, 2000000)
    assert abs(len(X) / len(Xa) - 0.05) < 0.01
    # the cap truncates
    Xc, _, _, _, _ = ctx.mlp_pairs(theta, eps, band, 1.0, 13, 100)
    assert len(Xc) == 100


def test_training_reduces_loss_and_error(tc):
    """Pairs from one Plummer sphere train the network on the GPU; on another
    sphere the learned walk at theta 0.9 has a smaller RMS error against the
    direct sum than the plain walk at the same theta."""
    theta, eps, band = 0.9, 1e-3, 0.5
    ctx_tr, _, _ = _built(tc, 131072, 21)
    X, T, F, _, _ = ctx_tr.mlp_pairs(theta, eps, band, 1.0, 5, 2_000_000)
    assert len(X) > 200000
    losses = ctx_tr.mlp_train(X, T, F, epochs=40, batch=1024, lr=2e-3, seed=3, band=band, factors=True)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.2 * losses[0]
    model, _ = ctx_tr.mlp_get()
    n = 65536
    ctx, p, m = _built(tc, n, 22)
    idx = inputs.sample_indices(n, 2048, 23)
    ad, _ = oracle.direct(p, m, eps, 1.0, idx=idx, want_pot=False)
    ctx.forces(theta, eps)
    a_plain = ctx.get_acc()[idx].astype(np.float64)
    ctx.mlp_set(model, band)
    ctx.set_config(learned=1)
    ctx.forces(theta, eps)
    a_learn = ctx.get_acc()[idx].astype(np.float64)

    def rms(a):
        return np.sqrt(np.mean(np.sum((a - ad) ** 2, 1) / np.sum(ad ** 2, 1)))

    e_plain, e_learn = rms(a_plain), rms(a_learn)
    print(f"theta {theta}: plain rms {e_plain:.3e}, learned rms {e_learn:.3e}, losses {losses[0]:.3g} -> "
          f"{losses[-1]:.3g}")
    assert e_learn < 0.85 * e_plain


def test_training_repeats_bit_for_bit(tc):
    """Pairs, feature maps and training are deterministic: two contexts on
    the same bodies with the same seeds end with the same model and losses,
    bit for bit (gradients are summed per warp and then in warp order, the
    pairs sorted by (body, node), the maps' sums taken in one order)."""
    theta, eps, band = 0.9, 1e-3, 0.5
    out = []
    for _ in range(2):
        ctx, _, _ = _built(tc, 32768, 31)
        X, T, F, _, _ = ctx.mlp_pairs(theta, eps, band, 0.5, 7, 1_000_000)
        losses = ctx.mlp_train(X, T, F, epochs=3, batch=1024, lr=2e-3, seed=3, band=band, factors=True)
        model, b = ctx.mlp_get()
        out.append((X, losses, model, b))
        ctx.close()
    assert len(out[0][0]) > 10000
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2]) and out[0][3] == out[1][3]


def test_learned_step_and_config_errors(tc):
    ctx, p, m = _built(tc, 8192, 30)
    with pytest.raises(tc.TcError):
        ctx.set_config(learned=1, precise=0)
    with pytest.raises(tc.TcError):
        ctx.set_config(learned=1, quad=0)
    ctx.set_config(learned=1)
    with pytest.raises(tc.TcError):
        ctx.forces(0.9, 1e-3)  # no model yet
    ctx.mlp_set(np.zeros(tc.MLP_NMODEL, np.float32), band=0.5)
    ctx.forces(0.9, 1e-3)
    a = ctx.get_acc().copy()
    ctx.set_config(learned=0)
    ctx.forces(0.9, 1e-3)
    assert np.array_equal(a, ctx.get_acc())
    # a graph-captured step with the learned walk runs and stays finite
    ctx.set_config(learned=1)
    ctx.set_velocity(np.zeros((8192, 3), np.float32))
    for _ in range(3):
        ctx.step(1e-4)
    pos, vel = ctx.get_state()
    assert np.all(np.isfinite(pos)) and np.all(np.isfinite(vel))
    bad = np.zeros(tc.MLP_NMODEL, np.float32)
    bad[5] = np.nan
    with pytest.raises(tc.TcError):
        ctx.mlp_set(bad, 0.5)
    with pytest.raises(tc.TcError):
        ctx.mlp_set(np.zeros(tc.MLP_NMODEL, np.float32), -1.0)


def test_deferred_band_record_overflow_is_reported(tc, monkeypatch):
    """A learned split walk that records more band cells than its buffer
    holds stops with TC_EDEVICE instead of writing past it (the buffer cut
    to 4096 entries through TC_BAND_CAP); with the buffer restored the same
    context runs the learned walk again."""
    ctx, p, m = _built(tc, 20000, 40, split=2)
    rng = np.random.default_rng(41)
    params = (rng.standard_normal(tc.MLP_NPARAM) * 0.1).astype(np.float32)
    model = np.concatenate([params, np.zeros(13), np.ones(13), np.full(3, 1e-3)]).astype(np.float32)
    ctx.mlp_set(model, band=0.3)
    ctx.set_config(learned=1)
    monkeypatch.setenv("TC_BAND_CAP", "4096")
    ctx.forces(0.9, 1e-3)
    with pytest.raises(tc.TcError) as e:
        ctx.sync()
    assert e.value.code == tc.TC_EDEVICE and "band" in str(e.value)
    monkeypatch.delenv("TC_BAND_CAP")
    ctx.forces(0.9, 1e-3)
    ctx.sync()
    assert ctx.mlp_evals() > 4096
