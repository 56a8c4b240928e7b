"""Thin Python binding of libtc (include/tc.h): argument marshalling only.

Every step of the treecode runs in the CUDA library; this module converts
torch tensors / numpy arrays to pointers, passes the current torch CUDA
stream, and turns error codes into exceptions.  If the library is missing it
raises -- there is no fallback.

Same names as the C ABI: ``build``, ``forces``, ``step`` on a ``Context``
(``tc_ctx_build`` ...) and module-level ``tc_build``/``tc_forces``/``tc_step``
on the library's implicit default context.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtc.so")

TC_OK, TC_EINVAL, TC_ENOMEM, TC_ESTATE, TC_EDEVICE, TC_ECUDA = 0, -1, -2, -3, -4, -5
_NAMES = {TC_EINVAL: "TC_EINVAL", TC_ENOMEM: "TC_ENOMEM", TC_ESTATE: "TC_ESTATE",
          TC_EDEVICE: "TC_EDEVICE", TC_ECUDA: "TC_ECUDA"}

# every symbol declared in include/tc.h
EXPORTS = [
    "tc_create", "tc_destroy", "tc_set_config", "tc_get_config", "tc_set_stream", "tc_ctx_build",
    "tc_ctx_set_velocity", "tc_ctx_forces", "tc_ctx_step", "tc_get_acc", "tc_get_state", "tc_set_state",
    "tc_get_sizes", "tc_get_tree", "tc_get_nodes", "tc_get_groups", "tc_get_cube", "tc_get_lists",
    "tc_diag", "tc_direct", "tc_sync", "tc_last_error", "tc_build", "tc_forces", "tc_step", "tc_default",
    "tc_set_timing", "tc_get_timings", "tc_direct_static", "tc_ctx_build_batch", "tc_get_systems",
    "tc_autotune", "tc_mlp_set", "tc_mlp_get", "tc_mlp_forward", "tc_mlp_loss_grad", "tc_mlp_train",
    "tc_mlp_pairs", "tc_mlp_evals", "tc_get_group_list", "tc_selftest_bounded_wait",
    "tc_probe_fp32",
    "tc_probe_force",
    "tc_ctx_fmm", "tc_get_fmm_stats", "tc_get_fmm_pairs",
]

MLP_NPARAM = 13 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3
TC_MLP_WEIGHTS, TC_MLP_FACTORS = 0, 1
MLP_NMODEL = MLP_NPARAM + 13 + 13 + 3


class TcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class tc_config(ctypes.Structure):
    _fields_ = [("gmax", ctypes.c_int32), ("warps", ctypes.c_int32), ("precise", ctypes.c_int32),
                ("want_pot", ctypes.c_int32), ("verify", ctypes.c_int32), ("stack", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("quad", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("learned", ctypes.c_int32), ("quadrupole", ctypes.c_int32),
                ("classes", ctypes.c_int32), ("split", ctypes.c_int32)]


_lib = None


def load(path: str | None = None):
    """Load libtc.so (built by ``paper_1211_2293_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libtc.so not found at {p}: run `python -m paper_1211_2293_gb300.build`")
    lib = ctypes.CDLL(p)
    P, I32, I64, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    sig = {
        "tc_create": ([ctypes.POINTER(P), P], I32),
        "tc_destroy": ([P], None),
        "tc_set_config": ([P, ctypes.POINTER(tc_config)], I32),
        "tc_get_config": ([P, ctypes.POINTER(tc_config)], I32),
        "tc_set_stream": ([P, P], I32),
        "tc_ctx_build": ([P, P, P, I64, I32], I32),
        "tc_ctx_set_velocity": ([P, P], I32),
        "tc_ctx_forces": ([P, F, F, F], I32),
        "tc_ctx_step": ([P, F], I32),
        "tc_get_acc": ([P, P, P], I32),
        "tc_get_state": ([P, P, P], I32),
        "tc_set_state": ([P, P, P], I32),
        "tc_get_sizes": ([P, P, P, P], I32),
        "tc_get_tree": ([P, P, P], I32),
        "tc_get_nodes": ([P] + [P] * 9, I32),
        "tc_get_groups": ([P, P, P, P], I32),
        "tc_get_cube": ([P, P], I32),
        "tc_get_lists": ([P] + [P] * 6, I32),
        "tc_diag": ([P, P], I32),
        "tc_direct": ([P, P, I64, F, F, P, P], I32),
        "tc_sync": ([P], I32),
        "tc_last_error": ([P], ctypes.c_char_p),
        "tc_build": ([P, P, I64, I32], I32),
        "tc_forces": ([F, F, F], I32),
        "tc_step": ([F], I32),
        "tc_default": ([], P),
        "tc_set_timing": ([P, I32], I32),
        "tc_get_timings": ([P, P], I32),
        "tc_direct_static": ([P, P, I64, P, I64, F, F, P, P, P], I32),
        "tc_ctx_build_batch": ([P, P, P, P, I64, I32], I32),
        "tc_get_systems": ([P, P, P], I32),
        "tc_autotune": ([P, F, F, F, I32, ctypes.POINTER(tc_config), ctypes.POINTER(ctypes.c_double)], I32),
        "tc_mlp_set": ([P, P, F], I32),
        "tc_mlp_get": ([P, P, P], I32),
        "tc_mlp_forward": ([P, P, I64, P], I32),
        "tc_mlp_loss_grad": ([P, P, P, P, I64, P, P], I32),
        "tc_mlp_train": ([P, P, P, P, I32, I64, I32, I32, F, ctypes.c_uint64, F, P], I32),
        "tc_mlp_pairs": ([P, F, F, F, F, ctypes.c_uint64, I64, P, P, P, P, P, P], I32),
        "tc_mlp_evals": ([P, P], I32),
        "tc_get_group_list": ([P, I64, F, P, P, I64, P, P], I32),
        "tc_selftest_bounded_wait": ([P, P], I32),
        "tc_probe_fp32": ([I32, P], I32),
        "tc_probe_force": ([P], I32),
        "tc_ctx_fmm": ([P, F, F, F], I32),
        "tc_get_fmm_stats": ([P, P, P, P], I32),
        "tc_get_fmm_pairs": ([P, P, P, P, P], I32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int, ctx=None):
    if rc != TC_OK:
        msg = _lib.tc_last_error(ctx)
        raise TcError(rc, msg.decode() if msg else "")


def _ptr(x):
    """Pointer of a torch tensor (host or CUDA) or numpy array; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(x.data_ptr())


def _current_stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def probe_fp32(paired: bool = False) -> float:
    """Measured FP32 TFLOP/s of the current device (FMA chains; see tc.h)."""
    lib = load()
    t = ctypes.c_double()
    _check(lib.tc_probe_fp32(int(bool(paired)), ctypes.byref(t)))
    return t.value


def probe_force() -> float:
    """Measured TFLOP/s of the walk's force loop alone, 20 flops per
    interaction (see tc.h)."""
    lib = load()
    t = ctypes.c_double()
    _check(lib.tc_probe_force(ctypes.byref(t)))
    return t.value


def selftest_bounded_wait():
    """(error bits, elapsed ms) of a device wait made to run out (see tc.h)."""
    lib = load()
    bits = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(lib.tc_selftest_bounded_wait(ctypes.byref(bits), ctypes.byref(ms)))
    return bits.value, ms.value


class Context:
    """One treecode system on the current CUDA device (a ``tc_ctx``)."""

    def __init__(self, stream=None, **config):
        lib = load()
        h = ctypes.c_void_p()
        s = _current_stream() if stream is None else ctypes.c_void_p(int(stream))
        _check(lib.tc_create(ctypes.byref(h), s))
        self._h = h
        self._lib = lib
        if config:
            self.set_config(**config)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, rc):
        _check(rc, self._h)

    # ------------------------------------------------------------ config
    def config(self) -> dict:
        c = tc_config()
        self._c(self._lib.tc_get_config(self._h, ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in tc_config._fields_}

    def set_config(self, **kw):
        d = self.config()
        d.update(kw)
        c = tc_config(**{k: int(v) for k, v in d.items()})
        self._c(self._lib.tc_set_config(self._h, ctypes.byref(c)))

    def set_stream(self, stream):
        self._c(self._lib.tc_set_stream(self._h, ctypes.c_void_p(int(stream))))

    # ------------------------------------------------------------ the path
    def build(self, pos, mass, leaf_max: int):
        n = int(mass.shape[0])
        self._c(self._lib.tc_ctx_build(self._h, _ptr(pos), _ptr(mass), n, int(leaf_max)))
        self.n = n

    def build_batch(self, pos, mass, offsets, leaf_max: int):
        """Independent systems: bodies [offsets[s], offsets[s+1]) form system s."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        self._c(self._lib.tc_ctx_build_batch(self._h, _ptr(pos), _ptr(mass), _ptr(off), off.shape[0] - 1,
                                             int(leaf_max)))
        self.n = int(off[-1])

    def systems(self):
        """(nsys, cubes[nsys, 5]) with cube = (c0x, c0y, c0z, L, h)."""
        ns = ctypes.c_int64()
        self._c(self._lib.tc_get_systems(self._h, ctypes.byref(ns), None))
        cubes = np.zeros((ns.value, 5))
        self._c(self._lib.tc_get_systems(self._h, None, _ptr(cubes)))
        return ns.value, cubes

    def autotune(self, theta: float, eps: float, G: float = 1.0, reps: int = 3):
        best = tc_config()
        ms = ctypes.c_double()
        self._c(self._lib.tc_autotune(self._h, float(theta), float(eps), float(G), int(reps), ctypes.byref(best),
                                      ctypes.byref(ms)))
        return {f: getattr(best, f) for f, _ in tc_config._fields_}, ms.value

    # ---------------------------------------------------------- learned correction
    def mlp_set(self, model, band: float):
        model = np.ascontiguousarray(model, dtype=np.float32)
        assert model.size == MLP_NMODEL
        self._c(self._lib.tc_mlp_set(self._h, _ptr(model), float(band)))

    def mlp_get(self):
        model = np.zeros(MLP_NMODEL, np.float32)
        band = ctypes.c_float()
        self._c(self._lib.tc_mlp_get(self._h, _ptr(model), ctypes.byref(band)))
        return model, band.value

    def mlp_forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 13)
        Y = np.zeros((X.shape[0], 3), np.float32)
        self._c(self._lib.tc_mlp_forward(self._h, _ptr(X), X.shape[0], _ptr(Y)))
        return Y

    def mlp_loss_grad(self, X, T, W=None):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 13)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(-1, 3)
        W = None if W is None else np.ascontiguousarray(W, dtype=np.float32).reshape(-1)
        g = np.zeros(MLP_NPARAM, np.float32)
        loss = ctypes.c_float()
        self._c(self._lib.tc_mlp_loss_grad(self._h, _ptr(X), _ptr(T), _ptr(W), X.shape[0], _ptr(g),
                                           ctypes.byref(loss)))
        return loss.value, g

    def mlp_train(self, X, T, W=None, epochs=40, batch=1024, lr=2e-3, seed=0, band=0.5, factors=False):
        """Train a fresh model on pairs (X, T).  W: loss weights (None: 1), or
        with factors=True the pairs' label factors F (weights F^2 / mean F^2,
        formed by the library)."""
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 13)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(-1, 3)
        W = None if W is None else np.ascontiguousarray(W, dtype=np.float32).reshape(-1)
        losses = np.zeros(int(epochs), np.float32)
        mode = TC_MLP_FACTORS if factors else TC_MLP_WEIGHTS
        self._c(self._lib.tc_mlp_train(self._h, _ptr(X), _ptr(T), _ptr(W), mode, X.shape[0], int(epochs), int(batch),
                                       float(lr), int(seed), float(band), _ptr(losses)))
        return losses

    def mlp_pairs(self, theta, eps, band, prob, seed, max_pairs):
        """(X, T, F, body, node) of pairs generated by a walk at theta."""
        X = np.zeros((max_pairs, 13), np.float32)
        T = np.zeros((max_pairs, 3), np.float32)
        F = np.zeros(max_pairs, np.float32)
        b = np.zeros(max_pairs, np.int64)
        v = np.zeros(max_pairs, np.int64)
        npairs = ctypes.c_int64()
        self._c(self._lib.tc_mlp_pairs(self._h, float(theta), float(eps), float(band), float(prob), int(seed),
                                       int(max_pairs), _ptr(X), _ptr(T), _ptr(F), _ptr(b), _ptr(v),
                                       ctypes.byref(npairs)))
        k = npairs.value
        return X[:k], T[:k], F[:k], b[:k], v[:k]

    def mlp_evals(self):
        v = ctypes.c_int64()
        self._c(self._lib.tc_mlp_evals(self._h, ctypes.byref(v)))
        return v.value

    def set_velocity(self, vel):
        self._c(self._lib.tc_ctx_set_velocity(self._h, _ptr(vel)))

    def forces(self, theta: float, eps: float, G: float = 1.0):
        self._c(self._lib.tc_ctx_forces(self._h, float(theta), float(eps), float(G)))

    def fmm(self, theta: float, eps: float, G: float = 1.0):
        """Fast multipole accelerations on the current tree (read with get_acc)."""
        self._c(self._lib.tc_ctx_fmm(self._h, float(theta), float(eps), float(G)))

    def fmm_stats(self) -> dict:
        """M2L and P2P pair counts of the last fmm() and the pair-set hashes
        (None unless verify is set)."""
        m, p = ctypes.c_int64(), ctypes.c_int64()
        h = np.zeros(2, np.uint64) if self.config()["verify"] else None
        self._c(self._lib.tc_get_fmm_stats(self._h, ctypes.byref(m), ctypes.byref(p), _ptr(h)))
        return dict(m2l=m.value, p2p=p.value, m2l_hash=None if h is None else int(h[0]),
                    p2p_hash=None if h is None else int(h[1]))

    def fmm_pairs(self) -> dict:
        """Per target cell of the last fmm(): nm2l, np2p, hm2l, hp2p."""
        M = self.sizes()[1]
        rec = dict(nm2l=np.zeros(M, np.int64), np2p=np.zeros(M, np.int64), hm2l=np.zeros(M, np.uint64),
                   hp2p=np.zeros(M, np.uint64))
        self._c(self._lib.tc_get_fmm_pairs(self._h, _ptr(rec["nm2l"]), _ptr(rec["np2p"]), _ptr(rec["hm2l"]),
                                           _ptr(rec["hp2p"])))
        return rec

    def step(self, dt: float):
        self._c(self._lib.tc_ctx_step(self._h, float(dt)))

    def sync(self):
        self._c(self._lib.tc_sync(self._h))

    def set_timing(self, on: bool = True):
        self._c(self._lib.tc_set_timing(self._h, int(bool(on))))

    def timings(self) -> dict:
        """Phase times (ms, summed since the last call) and kernel launches."""
        out = np.zeros(6)
        self._c(self._lib.tc_get_timings(self._h, _ptr(out)))
        return dict(build_ms=out[0], walk_ms=out[1], update_ms=out[2], launches=int(out[3]),
                    launches_total=int(out[4]), graph_kernels=int(out[5]))

    # ------------------------------------------------------------ outputs
    def get_acc(self, acc=None, pot=None, with_pot=False):
        n = self.sizes()[0]
        if acc is None:
            acc = np.empty((n, 3), np.float32)
        if pot is None and with_pot:
            pot = np.empty(n, np.float32)
        self._c(self._lib.tc_get_acc(self._h, _ptr(acc), _ptr(pot)))
        return (acc, pot) if with_pot or pot is not None else acc

    def get_state(self):
        n = self.sizes()[0]
        pos = np.empty((n, 3), np.float32)
        vel = np.empty((n, 3), np.float32)
        self._c(self._lib.tc_get_state(self._h, _ptr(pos), _ptr(vel)))
        return pos, vel

    def set_state(self, pos, vel):
        self._c(self._lib.tc_set_state(self._h, _ptr(pos), _ptr(vel)))

    def sizes(self):
        n, m, g = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._c(self._lib.tc_get_sizes(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(g)))
        return n.value, m.value, g.value

    def cube(self):
        out = np.zeros(5)
        self._c(self._lib.tc_get_cube(self._h, _ptr(out)))
        return out

    def tree(self):
        n, M, G = self.sizes()
        perm = np.empty(n, np.uint32)
        keys = np.empty(n, np.uint64)
        self._c(self._lib.tc_get_tree(self._h, _ptr(perm), _ptr(keys)))
        a = {k: np.empty(M, np.int32) for k in ("level", "first", "count", "child_first", "nchild")}
        a["prefix"] = np.empty(M, np.uint64)
        a["mass"] = np.empty(M)
        a["com"] = np.empty((M, 3))
        a["quad"] = np.empty((M, 6)) if self.config()["quad"] else None
        self._c(self._lib.tc_get_nodes(self._h, _ptr(a["level"]), _ptr(a["prefix"]), _ptr(a["first"]),
                                       _ptr(a["count"]), _ptr(a["child_first"]), _ptr(a["nchild"]),
                                       _ptr(a["mass"]), _ptr(a["com"]), _ptr(a["quad"])))
        gf, gc, gr = np.empty(G, np.int32), np.empty(G, np.int32), np.empty(G, np.int32)
        self._c(self._lib.tc_get_groups(self._h, _ptr(gf), _ptr(gc), _ptr(gr)))
        a.update(perm=perm, keys=keys, gfirst=gf, gcount=gc, gref=gr)
        return a

    def lists(self, per_group=True):
        G = self.sizes()[2]
        nc = np.empty(G, np.int32) if per_group else None
        nb = np.empty(G, np.int32) if per_group else None
        hs = np.empty(G, np.uint64) if per_group else None
        it, ce, bo = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._c(self._lib.tc_get_lists(self._h, _ptr(nc), _ptr(nb), _ptr(hs), ctypes.byref(it),
                                       ctypes.byref(ce), ctypes.byref(bo)))
        return dict(ncell=nc, nbody=nb, hash=hs, interactions=it.value, cells=ce.value, bodies=bo.value)

    def group_list(self, group: int, theta: float):
        """(accepted cells, opened leaves) of one group's walk, in walk order."""
        nc, nl = ctypes.c_int64(), ctypes.c_int64()
        self._c(self._lib.tc_get_group_list(self._h, int(group), float(theta), None, None, 0, ctypes.byref(nc),
                                            ctypes.byref(nl)))
        cap = max(nc.value, nl.value)
        cells = np.zeros(cap, np.int32)
        leaves = np.zeros(cap, np.int32)
        self._c(self._lib.tc_get_group_list(self._h, int(group), float(theta), _ptr(cells), _ptr(leaves), cap,
                                            ctypes.byref(nc), ctypes.byref(nl)))
        return cells[:nc.value], leaves[:nl.value]

    def diag(self):
        out = np.zeros(8)
        self._c(self._lib.tc_diag(self._h, _ptr(out)))
        return out

    def direct(self, idx, eps: float, G: float = 1.0):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        acc = np.empty((idx.shape[0], 3))
        pot = np.empty(idx.shape[0])
        self._c(self._lib.tc_direct(self._h, _ptr(idx), idx.shape[0], float(eps), float(G), _ptr(acc), _ptr(pot)))
        return acc, pot


# the three calls on the library's implicit default context
def tc_build(pos, mass, n: int, leaf_max: int):
    lib = load()
    _check(lib.tc_build(_ptr(pos), _ptr(mass), int(n), int(leaf_max)))


def tc_forces(theta: float, eps: float, G: float = 1.0):
    lib = load()
    _check(lib.tc_forces(float(theta), float(eps), float(G)))


def tc_step(dt: float):
    lib = load()
    _check(lib.tc_step(float(dt)))


def _check_static_args(pos, mass, idx, acc, pot):
    """Shapes, element types and devices of tc_direct_static's arguments,
    checked before anything reaches the C ABI (which sees bare pointers and
    would read or write past a buffer that is too short or of another
    type).  Returns the common CUDA device."""
    import torch

    def need(name, x, dtype, shape):
        if not isinstance(x, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if x.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
        if tuple(x.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}, got {tuple(x.shape)}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")

    if not isinstance(mass, torch.Tensor) or mass.dim() != 1:
        raise ValueError("mass must be a 1-D torch.Tensor")
    if not isinstance(idx, torch.Tensor) or idx.dim() != 1:
        raise ValueError("idx must be a 1-D torch.Tensor")
    n, ns = int(mass.shape[0]), int(idx.shape[0])
    need("pos", pos, torch.float32, (n, 3))
    need("mass", mass, torch.float32, (n,))
    need("idx", idx, torch.int64, (ns,))
    need("acc", acc, torch.float64, (ns, 3))
    if pot is not None:
        need("pot", pot, torch.float64, (ns,))
    devs = {x.device for x in (pos, mass, idx, acc, pot) if x is not None}
    if len(devs) != 1 or next(iter(devs)).type != "cuda":
        raise ValueError(f"all arrays must be CUDA tensors on one device, got {sorted(str(d) for d in devs)}")
    return next(iter(devs))


def tc_direct_static(pos, mass, idx, eps: float, G: float, acc, pot=None, stream=None):
    """Direct summation into caller-owned device buffers; allocates nothing
    on the device (see include/tc.h).  pos (n, 3) float32, mass (n,)
    float32, idx (ns,) int64, acc (ns, 3) float64, pot (ns,) float64 or
    None: contiguous CUDA tensors on one device.  The call runs on that
    device, on `stream` (a CUDA stream of that device) or its current torch
    stream."""
    import torch

    dev = _check_static_args(pos, mass, idx, acc, pot)
    lib = load()
    with torch.cuda.device(dev):
        s = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream) if stream is None else \
            ctypes.c_void_p(int(stream))
        _check(lib.tc_direct_static(_ptr(pos), _ptr(mass), int(mass.shape[0]), _ptr(idx), int(idx.shape[0]),
                                    float(eps), float(G), _ptr(acc), _ptr(pot), s))
