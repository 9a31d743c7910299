"""Shared test helpers: tolerances and comparisons (no method arithmetic)."""
import math

import numpy as np

MISS = 0xFFFFFFFF


def t_close(t_gpu, t_ref, rays, rel=1e-5):
    """|dt| <= rel * max(t, |origin|_inf, 1): FP32 positions carry an
    absolute error proportional to their magnitude, so a hit very close to a
    far-from-zero origin cannot have a small error relative to t alone."""
    scale = np.maximum(np.maximum(np.abs(t_ref), np.abs(rays[:, 0:3]).max(1)), 1.0)
    return np.abs(t_gpu - t_ref) <= rel * scale


def bary_fp64(rays, verts, idx, prim):
    """Unclipped barycentrics (b0, b1, b2) and t of each ray's plane hit with
    triangle `prim`, in float64 (validity check of an alternative hit)."""
    V = verts.astype(np.float64)
    tri = idx[prim.astype(np.int64)]
    v0, v1, v2 = V[tri[:, 0]], V[tri[:, 1]], V[tri[:, 2]]
    o = rays[:, 0:3].astype(np.float64)
    d = rays[:, 3:6].astype(np.float64)
    e1, e2 = v1 - v0, v2 - v0
    p = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, p)
    s = o - v0
    u = np.einsum("ij,ij->i", s, p) / det
    q = np.cross(s, e1)
    v = np.einsum("ij,ij->i", d, q) / det
    t = np.einsum("ij,ij->i", e2, q) / det
    return 1 - u - v, u, v, t


def image_parity(mean_a, var_a, mean_b, var_b):
    """Mean relative L1 and the number of pixel channels outside 4 sigma."""
    l1 = np.abs(mean_a - mean_b).sum() / max(np.abs(mean_b).sum(), 1e-30)
    sig = np.sqrt(var_a + var_b)
    out = np.abs(mean_a - mean_b) > 4 * sig + 1e-6 * np.maximum(np.abs(mean_b), 1e-3)
    return l1, int(out.sum()), out.size


def allowed_4sigma(n):
    """Max(1, 3 x the Gaussian expectation 6.3e-5 n) exceedances."""
    return max(1, int(math.ceil(3 * 6.334e-5 * n)))
