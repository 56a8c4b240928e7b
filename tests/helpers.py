"""Small independent helpers for the tests (geometry from first principles)."""
import numpy as np


def deinterleave(prefix: int, level: int):
    """Integer cube corner (in units of the level's cube side) of a Morton
    prefix: digit k (from the top) holds x, y, z bits of level k+1."""
    ix = iy = iz = 0
    for k in range(level):
        d = (int(prefix) >> (3 * (level - 1 - k))) & 7
        ix = (ix << 1) | ((d >> 2) & 1)
        iy = (iy << 1) | ((d >> 1) & 1)
        iz = (iz << 1) | (d & 1)
    return ix, iy, iz


def cube_of(tree, v):
    """(corner[3], side) of node v in absolute coordinates, exact dyadics."""
    lv = int(tree.level[v])
    side = np.ldexp(tree.L, -lv)
    i = deinterleave(int(tree.prefix[v]), lv)
    corner = np.array([tree.c0[a] + i[a] * side for a in range(3)])
    return corner, side


def mix64(z: int) -> int:
    m = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def rel_err_rms(a, b):
    num = np.sum((a - b) ** 2, axis=1)
    den = np.sum(b ** 2, axis=1)
    return float(np.sqrt(np.mean(num / den)))


def abs_field(pos, mass, idx, eps, rows=64):
    """sum_j m_j |x_j - x_i| / (|x_j - x_i|^2 + eps^2)^(3/2) for i in idx
    (FP64): the sum of the magnitudes of the softened pair fields, the scale
    of the float32 rounding of a sum of those terms however they cancel."""
    p = np.asarray(pos, np.float64)
    m = np.asarray(mass, np.float64)
    idx = np.asarray(idx, np.int64)
    out = np.zeros(idx.shape[0])
    for k0 in range(0, idx.shape[0], rows):
        d = p[None, :, :] - p[idx[k0:k0 + rows]][:, None, :]
        r2 = np.einsum("ijk,ijk->ij", d, d)
        out[k0:k0 + rows] = (np.sqrt(r2) * (r2 + eps * eps) ** -1.5) @ m
    return out
