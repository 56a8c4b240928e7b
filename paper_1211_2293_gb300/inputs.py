"""Seeded synthetic inputs (bodies) for the treecode.

This module holds the input recipes only -- none of the treecode's own
arithmetic -- so both the CUDA path and the CPU oracle are fed from it.

Random numbers come from a counter-based generator: the k-th draw of stream
``s`` under seed ``seed`` is the SplitMix64 finaliser of
``key(seed, s) + (k + 1) * 0x9E3779B97F4A7C15`` (Steele, Lea & Flood 2014),
mapped to a double in [0, 1) by its top 53 bits.  Every body owns a block of
counters, so a body's values do not depend on how many others are drawn.

Recipes
-------
* ``plummer``  Plummer sphere, scale radius a = 1, total mass 1, G = 1:
  radius by inverse CDF r = (X^(-2/3) - 1)^(-1/2), redrawn while r > cutoff
  (Aarseth, Henon & Wielen 1974); isotropic direction; speed v = q sqrt(2)
  (1 + r^2)^(-1/4) with q drawn by von Neumann rejection on
  g(q) = q^2 (1 - q^2)^(7/2) (bound 0.1).  Positions/velocities returned as
  float32, masses 1/N.
* ``uniform_cube``  uniform in [-1, 1]^3, at rest, masses 1/N.
* ``two_plummer``  two Plummer spheres of n/2 bodies (each of mass 1/2,
  velocities scaled by sqrt(1/2)), centred at (-d/2, 0, 0) and (+d/2, 0, 0)
  and approaching each other at relative speed ``v_rel``.
* ``batch_sizes``  N_k = floor(exp(U(ln lo, ln hi))) for k systems.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_BLOCK = 256  # counters reserved per body and stream


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        base = np.array([(int(seed) * 0x100000001B3 + int(stream) * 0x2545F4914F6CDD1D) & (2**64 - 1)],
                        dtype=np.uint64)
        return _mix(base + _GOLDEN)[0]


def uniforms(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) for the given counters of one (seed, stream)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(_key(seed, stream) + (c + np.uint64(1)) * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _per_body(seed, stream, idx, k):
    return uniforms(seed, stream, idx.astype(np.uint64) * np.uint64(_BLOCK) + np.uint64(k))


def _isotropic(seed, stream, idx):
    u = _per_body(seed, stream, idx, 0)
    w = _per_body(seed, stream, idx, 1)
    cz = 2.0 * u - 1.0
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    ph = 2.0 * np.pi * w
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)


def plummer(n: int, seed: int = 0, cutoff: float = 10.0, with_velocity: bool = True):
    """Plummer sphere (a = 1, M = 1, G = 1); returns (pos, vel, mass) float32."""
    n = int(n)
    idx = np.arange(n, dtype=np.int64)
    r = np.empty(n)
    todo = idx.copy()
    k = 0
    while todo.size:
        if k >= _BLOCK:
            raise RuntimeError("plummer: radius rejection ran out of counters")
        x = _per_body(seed, 0, todo, k)
        x = np.maximum(x, 1e-300)
        rr = 1.0 / np.sqrt(np.maximum(x ** (-2.0 / 3.0) - 1.0, 1e-300))
        ok = rr <= cutoff
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
        k += 1
    pos = _isotropic(seed, 1, idx) * r[:, None]
    vel = np.zeros((n, 3))
    if with_velocity:
        q = np.empty(n)
        todo = idx.copy()
        k = 0
        while todo.size:
            if 2 * k + 1 >= _BLOCK:
                raise RuntimeError("plummer: velocity rejection ran out of counters")
            qq = _per_body(seed, 2, todo, 2 * k)
            yy = 0.1 * _per_body(seed, 2, todo, 2 * k + 1)
            ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
            q[todo[ok]] = qq[ok]
            todo = todo[~ok]
            k += 1
        speed = q * np.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
        vel = _isotropic(seed, 3, idx) * speed[:, None]
    mass = np.full(n, 1.0 / n)
    return pos.astype(np.float32), vel.astype(np.float32), mass.astype(np.float32)


def uniform_cube(n: int, seed: int = 0, half: float = 1.0):
    """Uniform bodies in [-half, half]^3 at rest; returns (pos, vel, mass)."""
    n = int(n)
    idx = np.arange(n, dtype=np.int64)
    u = np.stack([_per_body(seed, 4, idx, a) for a in range(3)], axis=1)
    pos = (2.0 * u - 1.0) * half
    return pos.astype(np.float32), np.zeros((n, 3), np.float32), np.full(n, 1.0 / n, np.float32)


def two_plummer(n: int, seed: int = 0, separation: float = 6.0, v_rel: float = 0.5, cutoff: float = 10.0):
    """Two Plummer spheres of n//2 bodies each approaching head-on."""
    n = int(n)
    h = n // 2
    out_p, out_v = [], []
    for s, sign in ((0, -1.0), (1, 1.0)):
        m = h if s == 0 else n - h
        p, v, _ = plummer(m, seed=seed * 2 + s + 1000, cutoff=cutoff)
        p = p.astype(np.float64)
        v = v.astype(np.float64) * np.sqrt(0.5)
        p[:, 0] += sign * separation / 2.0
        v[:, 0] -= sign * v_rel / 2.0
        out_p.append(p)
        out_v.append(v)
    pos = np.concatenate(out_p).astype(np.float32)
    vel = np.concatenate(out_v).astype(np.float32)
    return pos, vel, np.full(n, 1.0 / n, np.float32)


def batch_sizes(k: int, seed: int = 0, lo: int = 1024, hi: int = 65536) -> np.ndarray:
    """k system sizes, log-uniform in [lo, hi]."""
    u = uniforms(seed, 7, np.arange(int(k), dtype=np.uint64))
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def sample_indices(n: int, k: int, seed: int = 0) -> np.ndarray:
    """k distinct body indices out of n (seeded, without replacement), sorted."""
    k = min(int(k), int(n))
    u = uniforms(seed, 9, np.arange(int(n), dtype=np.uint64))
    return np.sort(np.argsort(u, kind="stable")[:k]).astype(np.int64)
