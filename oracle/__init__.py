"""FP64 CPU oracle of the treecode force phase (Sec. 3.1 of the paper).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
product library (``paper_1211_2293_gb300``) never imports, links or runs it.
It shares no code with the GPU path.

The arithmetic lives in plain C (``tc_oracle.c``, double precision, built with
``-ffp-contract=off``); this module compiles it with gcc on first use and
wraps it with ctypes and numpy.  Readings of the paper used here are listed in
the header of ``tc_oracle.c`` (R1..R7).

Parity pins: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force or textbook special cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tc_oracle.c")
_HDR = os.path.join(_HERE, "tc_oracle.h")
_SO = os.path.join(_HERE, "libtc_oracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no GPU needed)."""
    with _lock:
        stale = (not os.path.exists(_SO)) or any(
            os.path.getmtime(p) > os.path.getmtime(_SO) for p in (_SRC, _HDR)
        )
        if force or stale:
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    D = ctypes.c_double
    lib.or_root_cube.argtypes = [P, I64, P]
    lib.or_root_cube.restype = ctypes.c_int
    lib.or_keys.argtypes = [P, I64, P, P]
    lib.or_keys.restype = None
    lib.or_tree_build.argtypes = [P, P, I64, ctypes.c_int]
    lib.or_tree_build.restype = P
    lib.or_tree_free.argtypes = [P]
    lib.or_tree_free.restype = None
    lib.or_tree_nnodes.argtypes = [P]
    lib.or_tree_nnodes.restype = I64
    lib.or_tree_nbodies.argtypes = [P]
    lib.or_tree_nbodies.restype = I64
    lib.or_tree_get_cube.argtypes = [P, P]
    lib.or_tree_get_perm.argtypes = [P, P]
    lib.or_tree_get_keys.argtypes = [P, P]
    lib.or_tree_get_nodes.argtypes = [P] + [P] * 7
    lib.or_tree_get_moments.argtypes = [P, P, P, P]
    lib.or_tree_make_groups.argtypes = [P, ctypes.c_int]
    lib.or_tree_make_groups.restype = I64
    lib.or_tree_get_groups.argtypes = [P, P, P, P]
    lib.or_tree_walk.argtypes = [P, D, D, D, I64, I64, P, P, P, P, P, P, P]
    lib.or_tree_walk.restype = I64
    lib.or_tree_walk_order.argtypes = [P, D, D, D, ctypes.c_int, I64, I64, P, P, P, P, P, P, P]
    lib.or_tree_walk_order.restype = I64
    lib.or_tree_test.argtypes = [P, I64, I64, D]
    lib.or_tree_test.restype = ctypes.c_int
    lib.or_direct.argtypes = [P, P, I64, D, D, P, I64, P, P]
    lib.or_direct.restype = None
    lib.or_direct64.argtypes = [P, P, I64, D, D, P, I64, P, P]
    lib.or_direct64.restype = None
    lib.or_kick.argtypes = [P, P, I64, D]
    lib.or_drift.argtypes = [P, P, I64, D]
    lib.or_diag.argtypes = [P, P, P, P, I64, P]
    lib.or_mlp_features.argtypes = [P, I64, P, D, D, P]
    lib.or_mlp_features.restype = None
    lib.or_mlp_label.argtypes = [P, I64, P, D, D, P]
    lib.or_mlp_label.restype = None
    lib.or_mlp_forward.argtypes = [P, P, I64, P]
    lib.or_mlp_forward.restype = None
    lib.or_mlp_grad.argtypes = [P, P, P, P, I64, P]
    lib.or_mlp_factor.argtypes = [P, I64, P, D]
    lib.or_mlp_factor.restype = D
    lib.or_mlp_grad.restype = D
    lib.or_tree_group_list.argtypes = [P, D, I64, P, I64, P, I64, P, P]
    lib.or_tree_group_list.restype = None
    lib.or_tree_learned.argtypes = [P, D, D, D, D, P, P, I64, I64, P, P]
    lib.or_tree_learned.restype = I64
    lib.or_tree_learned_bf16.argtypes = [P, D, D, D, D, P, P, I64, I64, P, P, P]
    lib.or_tree_learned_bf16.restype = I64
    lib.or_fmm.argtypes = [P, D, D, D, P, P]
    lib.or_fmm.restype = None
    lib.or_fmm_nodes.argtypes = [P, D, D, D, P, P, P, P, P, P, P]
    lib.or_fmm_nodes.restype = None
    lib.or_fmm_radii.argtypes = [P, P]
    lib.or_fmm_radii.restype = None
    lib.or_bf16.argtypes = [D]
    lib.or_bf16.restype = D
    lib.or_mlp_forward_bf16.argtypes = [P, P, P, I64, P, P]
    lib.or_mlp_forward_bf16.restype = None
    lib.or_mlp_grad_bf16.argtypes = [P, P, P, P, P, I64, P, P, P]
    lib.or_mlp_grad_bf16.restype = D
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def root_cube(pos):
    """(c0[3], L, h) of the root cube (reading R1) for float32 positions."""
    lib = _load()
    pos = _f32(pos).reshape(-1, 3)
    out = np.zeros(5)
    if lib.or_root_cube(_ptr(pos), pos.shape[0], _ptr(out)) != 0:
        raise ValueError("root cube: empty input or non-finite coordinate")
    return out[:3].copy(), float(out[3]), float(out[4])


def morton_keys(pos, cube5):
    lib = _load()
    pos = _f32(pos).reshape(-1, 3)
    cube5 = _f64(cube5)
    keys = np.zeros(pos.shape[0], dtype=np.uint64)
    lib.or_keys(_ptr(pos), pos.shape[0], _ptr(cube5), _ptr(keys))
    return keys


class Tree:
    """The oracle's oct-tree of one body set (Sec. 3.1), with groups."""

    def __init__(self, pos, mass, leaf_max: int, gmax: int | None = None):
        self._lib = _load()
        self.pos = _f32(pos).reshape(-1, 3)
        self.mass = _f32(mass).reshape(-1)
        n = self.pos.shape[0]
        h = self._lib.or_tree_build(_ptr(self.pos), _ptr(self.mass), n, int(leaf_max))
        if not h:
            raise ValueError("oracle tree build rejected the input")
        self._h = h
        self.n = n
        self.leaf_max = int(leaf_max)
        self.M = int(self._lib.or_tree_nnodes(h))
        cube = np.zeros(5)
        self._lib.or_tree_get_cube(h, _ptr(cube))
        self.cube5 = cube
        self.c0, self.L, self.h = cube[:3].copy(), float(cube[3]), float(cube[4])
        self.perm = np.zeros(n, dtype=np.uint32)
        self._lib.or_tree_get_perm(h, _ptr(self.perm))
        self.keys = np.zeros(n, dtype=np.uint64)
        self._lib.or_tree_get_keys(h, _ptr(self.keys))
        M = self.M
        self.level = np.zeros(M, dtype=np.int32)
        self.prefix = np.zeros(M, dtype=np.uint64)
        self.first = np.zeros(M, dtype=np.int64)
        self.count = np.zeros(M, dtype=np.int64)
        self.child_first = np.zeros(M, dtype=np.int64)
        self.nchild = np.zeros(M, dtype=np.int32)
        self.parent = np.zeros(M, dtype=np.int64)
        self._lib.or_tree_get_nodes(
            h, _ptr(self.level), _ptr(self.prefix), _ptr(self.first), _ptr(self.count),
            _ptr(self.child_first), _ptr(self.nchild), _ptr(self.parent),
        )
        self.node_mass = np.zeros(M)
        self.com = np.zeros((M, 3))
        self.quad = np.zeros((M, 6))
        self._lib.or_tree_get_moments(h, _ptr(self.node_mass), _ptr(self.com), _ptr(self.quad))
        self.G = 0
        if gmax is not None:
            self.make_groups(gmax)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_tree_free(h)
            self._h = None

    def make_groups(self, gmax: int):
        G = int(self._lib.or_tree_make_groups(self._h, int(gmax)))
        if G < 0:
            raise ValueError("gmax must be >= 1")
        self.G = G
        self.gmax = int(gmax)
        self.gfirst = np.zeros(G, dtype=np.int64)
        self.gcount = np.zeros(G, dtype=np.int64)
        self.gref = np.zeros(G, dtype=np.int64)
        self._lib.or_tree_get_groups(self._h, _ptr(self.gfirst), _ptr(self.gcount), _ptr(self.gref))
        return G

    def side(self, v=None):
        lv = self.level if v is None else self.level[v]
        return np.ldexp(self.L, -np.asarray(lv))

    def walk(self, theta, eps, G=1.0, groups=None, want_pot=True, quadrupole=False):
        """Walk + force for a range of groups (default: all).

        Returns dict with acc (n x 3, original order; NaN for bodies outside
        the walked groups), pot, amag (sum of |term| per body), ncell, nbody,
        hash, flag (per group, -1 for groups not walked) and the number of
        interactions.  quadrupole: accepted cells add their quadrupole term."""
        if self.G == 0:
            raise RuntimeError("make_groups first")
        g0, g1 = (0, self.G) if groups is None else groups
        acc = np.full((self.n, 3), np.nan)
        pot = np.full(self.n, np.nan) if want_pot else None
        amag = np.full(self.n, np.nan)
        ncell = np.full(self.G, -1, dtype=np.int64)
        nbody = np.full(self.G, -1, dtype=np.int64)
        hsh = np.zeros(self.G, dtype=np.uint64)
        flag = np.full(self.G, -1, dtype=np.int32)
        inter = self._lib.or_tree_walk_order(
            self._h, float(theta), float(eps), float(G), int(bool(quadrupole)), int(g0), int(g1),
            _ptr(acc), _ptr(pot), _ptr(amag), _ptr(ncell), _ptr(nbody), _ptr(hsh), _ptr(flag),
        )
        return dict(acc=acc, pot=pot, amag=amag, ncell=ncell, nbody=nbody, hash=hsh, flag=flag,
                    interactions=int(inter))

    def group_list(self, group: int, theta: float):
        """(accepted cells, opened leaves) of one group's walk, in walk order."""
        nc, nl = ctypes.c_int64(), ctypes.c_int64()
        self._lib.or_tree_group_list(self._h, float(theta), int(group), None, 0, None, 0, ctypes.byref(nc),
                                     ctypes.byref(nl))
        cells = np.zeros(nc.value, np.int64)
        leaves = np.zeros(nl.value, np.int64)
        self._lib.or_tree_group_list(self._h, float(theta), int(group), _ptr(cells), nc.value, _ptr(leaves),
                                     nl.value, ctypes.byref(nc), ctypes.byref(nl))
        return cells, leaves

    def test(self, group: int, node: int, theta: float) -> int:
        return int(self._lib.or_tree_test(self._h, int(group), int(node), float(theta)))

    def mlp_features(self, node: int, x, eps: float, msys: float):
        """13 features of (point x, cell node) for the learned correction."""
        x = _f64(x)
        f = np.zeros(13)
        self._lib.or_mlp_features(self._h, int(node), _ptr(x), float(eps), float(msys), _ptr(f))
        return f

    def learned(self, theta, eps, band, params=None, maps=None, G=1.0, groups=None):
        """Learned correction of the group walk (cells in the band evaluated
        at the centre of the group's box).  params None: exact labels.
        Returns (corr n x 3 original order, NaN outside the walked groups;
        flag per group, -1 if not walked; number of evaluations)."""
        if self.G == 0:
            raise RuntimeError("make_groups first")
        g0, g1 = (0, self.G) if groups is None else groups
        corr = np.full((self.n, 3), np.nan)
        flag = np.full(self.G, -1, dtype=np.int32)
        p = None if params is None else _f64(params)
        m = None if maps is None else _f64(maps)
        if p is not None:
            assert p.size == MLP_NPARAM and m is not None and m.size == 29
        ev = self._lib.or_tree_learned(self._h, float(theta), float(eps), float(G), float(band),
                                       None if p is None else _ptr(p), None if m is None else _ptr(m),
                                       int(g0), int(g1), _ptr(corr), _ptr(flag))
        return corr, flag, int(ev)

    def learned_bf16(self, theta, eps, band, params, maps, G=1.0, groups=None):
        """The band sum of ``learned`` with the network's BF16 rounding model:
        (corr, radius of an FP32 implementation (n x 3), flag, evaluations);
        NaN outside the walked groups."""
        if self.G == 0:
            raise RuntimeError("make_groups first")
        g0, g1 = (0, self.G) if groups is None else groups
        corr = np.full((self.n, 3), np.nan)
        crad = np.full((self.n, 3), np.nan)
        flag = np.full(self.G, -1, dtype=np.int32)
        p = _f64(params)
        m = _f64(maps)
        assert p.size == MLP_NPARAM and m.size == 29
        ev = self._lib.or_tree_learned_bf16(self._h, float(theta), float(eps), float(G), float(band), _ptr(p),
                                            _ptr(m), int(g0), int(g1), _ptr(corr), _ptr(crad), _ptr(flag))
        return corr, crad, flag, int(ev)

    def fmm_radii(self):
        """r_X of every cell (the FMM's acceptance radii), FP64."""
        r = np.zeros(self.M)
        self._lib.or_fmm_radii(self._h, _ptr(r))
        return r

    def fmm(self, theta, eps, G=1.0, per_node=False):
        """Fast multipole accelerations (n x 3, original order) and the
        traversal's statistics: dict(m2l, p2p, ties, m2l_hash, p2p_hash);
        with per_node, also per target cell (M each): nm2l, np2p, hm2l, hp2p
        and flag (a tie in the cell's walk or an ancestor's)."""
        acc = np.zeros((self.n, 3))
        st = np.zeros(5, np.int64)
        if not per_node:
            self._lib.or_fmm(self._h, float(theta), float(eps), float(G), _ptr(acc), _ptr(st))
        else:
            M = self.M
            rec = dict(nm2l=np.zeros(M, np.int64), np2p=np.zeros(M, np.int64), hm2l=np.zeros(M, np.uint64),
                       hp2p=np.zeros(M, np.uint64), flag=np.zeros(M, np.int32))
            self._lib.or_fmm_nodes(self._h, float(theta), float(eps), float(G), _ptr(acc), _ptr(st),
                                   _ptr(rec["nm2l"]), _ptr(rec["np2p"]), _ptr(rec["hm2l"]), _ptr(rec["hp2p"]),
                                   _ptr(rec["flag"]))
        out = dict(m2l=int(st[0]), p2p=int(st[1]), ties=int(st[2]), m2l_hash=int(st[3]) & (2**64 - 1),
                   p2p_hash=int(st[4]) & (2**64 - 1))
        if per_node:
            out.update(rec)
        return acc, out

    def mlp_factor(self, node: int, x, G: float = 1.0):
        """G M s^2 / r^4 of cell node at point x (the acceleration unit of a label)."""
        return float(self._lib.or_mlp_factor(self._h, int(node), _ptr(_f64(x)), float(G)))

    def mlp_label(self, node: int, x, eps: float, G: float = 1.0):
        """(a_exact - a_mono) / (G M s^2 / r^4) of cell node at point x."""
        x = _f64(x)
        t = np.zeros(3)
        self._lib.or_mlp_label(self._h, int(node), _ptr(x), float(eps), float(G), _ptr(t))
        return t


def direct(pos, mass, eps, G=1.0, idx=None, want_pot=True):
    """Direct summation (exact result the treecode approximates), FP64.

    pos/mass float32 (the GPU's inputs) or float64.  idx: original indices
    of the bodies to evaluate (default all).  Returns (acc[ns,3], pot[ns])."""
    lib = _load()
    is64 = np.asarray(pos).dtype == np.float64
    pos = (_f64 if is64 else _f32)(pos).reshape(-1, 3)
    mass = (_f64 if is64 else _f32)(mass).reshape(-1)
    n = pos.shape[0]
    idx = np.arange(n, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    acc = np.zeros((idx.shape[0], 3))
    pot = np.zeros(idx.shape[0]) if want_pot else None
    fn = lib.or_direct64 if is64 else lib.or_direct
    fn(_ptr(pos), _ptr(mass), n, float(eps), float(G), _ptr(idx), idx.shape[0], _ptr(acc), _ptr(pot))
    return acc, pot


def kick(vel, acc, h):
    lib = _load()
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    acc = _f64(acc)
    lib.or_kick(_ptr(vel), _ptr(acc), vel.size // 3, float(h))
    return vel


def drift(pos, vel, dt):
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    vel = _f64(vel)
    lib.or_drift(_ptr(pos), _ptr(vel), pos.size // 3, float(dt))
    return pos


def diag(pos, vel, mass, pot=None):
    """[KE, PE, Px, Py, Pz, Lx, Ly, Lz] in FP64."""
    lib = _load()
    pos, vel, mass = _f64(pos), _f64(vel), _f64(mass)
    pot = None if pot is None else _f64(pot)
    out = np.zeros(8)
    lib.or_diag(_ptr(pos), _ptr(vel), _ptr(mass), _ptr(pot), mass.size, _ptr(out))
    return out


def tree_forces(pos, mass, theta, eps, G=1.0, leaf_max=8, gmax=64, want_pot=True):
    """Build + groups + walk for all bodies; returns (acc, pot, tree, walk)."""
    t = Tree(pos, mass, leaf_max, gmax)
    w = t.walk(theta, eps, G, want_pot=want_pot)
    return w["acc"], w["pot"], t, w


def leapfrog_direct(pos, vel, mass, eps, G, dt, nsteps):
    """KDK leapfrog with direct-sum forces, all FP64 (reading R7)."""
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    mass = _f64(mass)
    acc, _ = direct(pos, mass, eps, G, want_pot=False)
    for _ in range(nsteps):
        vel = kick(vel, acc, 0.5 * dt)
        pos = drift(pos, vel, dt)
        acc, _ = direct(pos, mass, eps, G, want_pot=False)
        vel = kick(vel, acc, 0.5 * dt)
    return pos, vel


MLP_NPARAM = 13 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3


def mlp_forward(params, X):
    """MLP 13 -> 64 -> 64 -> 3 (ReLU), FP64; params packed W1, b1, W2, b2, W3, b3."""
    lib = _load()
    params = _f64(params)
    X = _f64(X).reshape(-1, 13)
    Y = np.zeros((X.shape[0], 3))
    lib.or_mlp_forward(_ptr(params), _ptr(X), X.shape[0], _ptr(Y))
    return Y


def mlp_grad(params, X, T, w=None):
    """(loss, gradient) of the (weighted) mean squared error, FP64."""
    lib = _load()
    params = _f64(params)
    X = _f64(X).reshape(-1, 13)
    T = _f64(T).reshape(-1, 3)
    w = None if w is None else _f64(w).reshape(-1)
    g = np.zeros(MLP_NPARAM)
    loss = lib.or_mlp_grad(_ptr(params), _ptr(X), _ptr(T), _ptr(w), X.shape[0], _ptr(g))
    return float(loss), g


def bf16(x):
    """Nearest bfloat16 value (8-bit significand, ties to even), FP64."""
    lib = _load()
    a = np.asarray(x, np.float64)
    return np.vectorize(lib.or_bf16, otypes=[np.float64])(a) if a.ndim else lib.or_bf16(float(a))


def mlp_forward_bf16(params, X, Xr=None):
    """BF16 rounding model of the network (inputs, weights and hidden
    activations rounded to bfloat16, sums exact): (Y[n,3], R[n,3]) with R
    the radius within which an implementation making the same roundings on
    FP32 sums lands, for inputs within Xr (n x 13, None: exact) of X."""
    lib = _load()
    params = _f64(params)
    X = _f64(X).reshape(-1, 13)
    Xr = None if Xr is None else _f64(np.broadcast_to(Xr, X.shape))
    Y = np.zeros((X.shape[0], 3))
    R = np.zeros((X.shape[0], 3))
    lib.or_mlp_forward_bf16(_ptr(params), _ptr(X), _ptr(Xr), X.shape[0], _ptr(Y), _ptr(R))
    return Y, R


def mlp_grad_bf16(params, X, T, w=None, Xr=None):
    """(loss, loss radius, gradient, gradient radius) of the BF16 rounding
    model (the backward's product operands dY, dH2, dH1 rounded as well)."""
    lib = _load()
    params = _f64(params)
    X = _f64(X).reshape(-1, 13)
    T = _f64(T).reshape(-1, 3)
    w = None if w is None else _f64(w).reshape(-1)
    Xr = None if Xr is None else _f64(np.broadcast_to(Xr, X.shape))
    g = np.zeros(MLP_NPARAM)
    gr = np.zeros(MLP_NPARAM)
    lrad = ctypes.c_double()
    loss = lib.or_mlp_grad_bf16(_ptr(params), _ptr(X), _ptr(Xr), _ptr(T), _ptr(w), X.shape[0], _ptr(g), _ptr(gr),
                                ctypes.byref(lrad))
    return float(loss), lrad.value, g, gr
