"""The exact result the FMM approximates ("O1"): direct smoothed Biot-Savart sums, FP64.

Test infrastructure (see ``oracle/__init__``).

* Element field (Eq. 1, smoothed by Eq. 2):  v_j(y) = K(|y - x_j|; a) w_j x (y - x_j) / |y - x_j|^3
  (no 1/(4 pi), as printed; a = 0 means K = 1, the singular field of Eq. 1).
* Core (Eq. vem1):  K(r; a) = erf(r / (a sqrt 2)) - sqrt(2/pi) (r/a) exp(-r^2 / (2 a^2)).
* Velocity at element i (Eq. s1.1): sum over j != i, j excluded by index.
* Gradient u_{lk} = d v_k / d y_l, and the stretching s_k = sum_l w_{i,l} u_{lk}
  (Eqs. s1.1, evf4).
"""
import math

import numpy as np
from scipy.special import erf

__all__ = ["core_K", "core_dK", "pair_terms", "direct", "direct_at"]

SQRT_2_OVER_PI = math.sqrt(2.0 / math.pi)


def core_K(r, a):
    """Eq. vem1 (K = 1 when a = 0)."""
    r = np.asarray(r, dtype=np.float64)
    if a == 0:
        return np.ones_like(r)
    return erf(r / (a * math.sqrt(2.0))) - SQRT_2_OVER_PI * (r / a) * np.exp(-r * r / (2.0 * a * a))


def core_dK(r, a):
    """dK/dr of Eq. vem1: sqrt(2/pi) r^2 / a^3 exp(-r^2/(2 a^2)) (0 when a = 0)."""
    r = np.asarray(r, dtype=np.float64)
    if a == 0:
        return np.zeros_like(r)
    return SQRT_2_OVER_PI * r * r / a ** 3 * np.exp(-r * r / (2.0 * a * a))


def pair_terms(d, w_src, a):
    """Contribution of sources with strengths w_src at offsets d = y - x_j.

    Returns (v, u) with v_k = f (w x d)_k and
    u_{lk} = f' d_l (w x d)_k / r + f (w x e_l)_k,  f = K / r^3, f' = df/dr.
    For a > 0 and r = 0 (a distinct element at the same point) f and f'/r take
    their limits from Eq. vem1: K = sqrt(2/pi) (r/a)^3 (1/3 - (r/a)^2/10 + ...),
    so f -> sqrt(2/pi) / (3 a^3) and f'/r -> -sqrt(2/pi) / (5 a^5)."""
    d = np.asarray(d, dtype=np.float64)
    r = np.sqrt((d * d).sum(axis=-1))
    K, dK = core_K(r, a), core_dK(r, a)
    with np.errstate(invalid="ignore", divide="ignore"):
        f = K / r ** 3
        fp_r = (dK / r ** 3 - 3.0 * K / r ** 4) / r
    if a > 0:
        f = np.where(r == 0, SQRT_2_OVER_PI / (3.0 * a ** 3), f)
        fp_r = np.where(r == 0, -SQRT_2_OVER_PI / (5.0 * a ** 5), fp_r)
    wxd = np.cross(w_src, d)
    v = f[..., None] * wxd
    u = fp_r[..., None, None] * d[..., :, None] * wxd[..., None, :]
    eye = np.eye(3)
    # (w x e_l)_k for l = 0..2 -> array [..., l, k]
    wxe = np.stack([np.cross(w_src, eye[l]) for l in range(3)], axis=-2)
    u = u + f[..., None, None] * wxe
    return v, u


def direct_at(x, w, a, targets, chunk=64):
    """v, u = grad v ([l, k] = d_l v_k) and s at the elements ``targets``
    (indices into x), summing over every element j != target."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    w = np.asarray(w, dtype=np.float64).reshape(-1, 3)
    targets = np.asarray(targets, dtype=np.int64)
    M = targets.shape[0]
    v = np.zeros((M, 3))
    u = np.zeros((M, 3, 3))
    for c0 in range(0, M, chunk):
        t = targets[c0:c0 + chunk]
        d = x[t][:, None, :] - x[None, :, :]                     # (chunk, N, 3)
        same = t[:, None] == np.arange(x.shape[0])[None, :]
        d = np.where(same[..., None], 1.0, d)                     # placeholder, zeroed below
        vv, uu = pair_terms(d, np.broadcast_to(w[None], d.shape), a)
        vv = np.where(same[..., None], 0.0, vv)
        uu = np.where(same[..., None, None], 0.0, uu)
        v[c0:c0 + chunk] = vv.sum(axis=1)
        u[c0:c0 + chunk] = uu.sum(axis=1)
    s = np.einsum("il,ilk->ik", w[targets], u)
    return v, u, s


def direct(x, w, a, chunk=64):
    """O1 at every element."""
    return direct_at(x, w, a, np.arange(np.asarray(x).reshape(-1, 3).shape[0]), chunk=chunk)
