"""Helpers shared by the oracle pins: finite-difference fields of Lamb-Helmholtz pairs.

These evaluate the potentials from their definition (Eq. rsbf6) and differentiate
numerically, so they are independent of the coefficient formulas under test."""
import numpy as np

from oracle import expansions, operators


def real_coeffs(p, rng, decay=0.7):
    """Random coefficients of a real harmonic function: c_n^{-m} = (-1)^m conj(c_n^m)."""
    c = operators.empty(p)
    for n in range(p):
        for m in range(0, n + 1):
            val = rng.normal() + (1j * rng.normal() if m > 0 else 0.0)
            val *= decay ** n
            c[n, m + p - 1] = val
            c[n, -m + p - 1] = (-1) ** m * np.conj(val)
    return c


def potential(c, r, basis):
    f = expansions.eval_R if basis == "R" else expansions.eval_S
    return f(c, r)


def fd_grad(fun, r, h):
    """Fourth-order central differences of a scalar function at points r (N, 3)."""
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    g = np.zeros(r.shape, dtype=np.complex128)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        g[:, k] = (-fun(r + 2 * e) + 8 * fun(r + e) - 8 * fun(r - e) + fun(r - 2 * e)) / (12 * h)
    return g


def lh_velocity(phi, chi, r, basis, h=1e-4):
    """v = grad phi + curl(r chi) = grad phi + (grad chi) x r (Eq. 4), by finite differences."""
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    gphi = fd_grad(lambda q: potential(phi, q, basis), r, h)
    gchi = fd_grad(lambda q: potential(chi, q, basis), r, h)
    return gphi + np.cross(gchi, r)


def lh_velocity_shifted(phi, chi, r, t, basis, h=1e-4):
    """v(r + t) of a pair expanded about the origin: grad phi + (grad chi) x (r + t)."""
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    q = r + np.asarray(t)
    gphi = fd_grad(lambda s: potential(phi, s, basis), q, h)
    gchi = fd_grad(lambda s: potential(chi, s, basis), q, h)
    return gphi + np.cross(gchi, q)


def biot_savart(xs, ws, y):
    """Eq. 1 at points y: sum_l w_l x (y - x_l) / |y - x_l|^3."""
    y = np.asarray(y, dtype=np.float64).reshape(-1, 3)
    d = y[:, None, :] - np.asarray(xs)[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    return (np.cross(np.broadcast_to(np.asarray(ws)[None], d.shape), d) / r[..., None] ** 3).sum(axis=1)
