"""Solid harmonics of the paper's Sec. 3.3 (Eqs. rsbf1-rsbf7), FP64, full m.

Test infrastructure (see ``oracle/__init__``).

The associated Legendre functions P_n^m of Eq. rsbf3 carry the Condon-Shortley
factor (-1)^m. They are taken from ``scipy.special.lpmv`` (a library primitive,
which uses the same phase); tests pin it against Rodrigues' formula evaluated in
exact rational arithmetic.
"""
import math

import numpy as np
from scipy.special import lpmv

__all__ = ["spherical", "legendre", "R_nm", "S_nm", "R_table", "S_table", "fact"]


def fact(k):
    """k! as a float (exact up to 22!, correctly rounded beyond)."""
    return float(math.factorial(int(k)))


def spherical(r):
    """Eq. rsbf1: (x, y, z) -> (|r|, mu = cos(theta), varphi).

    At r = 0 the angles are arbitrary; mu = 1, varphi = 0 is returned."""
    r = np.asarray(r, dtype=np.float64)
    x, y, z = r[..., 0], r[..., 1], r[..., 2]
    rho = np.sqrt(x * x + y * y + z * z)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(rho > 0, z / np.where(rho > 0, rho, 1.0), 1.0)
    mu = np.clip(mu, -1.0, 1.0)
    phi = np.arctan2(y, x)
    return rho, mu, phi


def legendre(n, m, mu):
    """P_n^m(mu) of Eq. rsbf3 for m >= 0 (Condon-Shortley phase included)."""
    if m < 0 or m > n:
        return np.zeros_like(np.asarray(mu, dtype=np.float64))
    return lpmv(m, n, mu)


def R_nm(n, m, r):
    """Regular (local) solid harmonic R_n^m(r), Eq. rsbf2; zero for |m| > n (Eq. rsbf7)."""
    rho, mu, phi = spherical(r)
    am = abs(m)
    if am > n:
        return np.zeros(rho.shape, dtype=np.complex128)
    return ((-1.0) ** n * (1j ** am) / fact(n + am)) * rho ** n * legendre(n, am, mu) * np.exp(1j * m * phi)


def S_nm(n, m, r):
    """Singular (multipole) solid harmonic S_n^m(r), Eq. rsbf2; zero for |m| > n."""
    rho, mu, phi = spherical(r)
    am = abs(m)
    if am > n:
        return np.zeros(rho.shape, dtype=np.complex128)
    return ((1j ** (-am)) * fact(n - am)) / rho ** (n + 1) * legendre(n, am, mu) * np.exp(1j * m * phi)


def _table(regular, nmax, r):
    """Eq. rsbf2 for all n <= nmax, |m| <= n: array [..., n, m + nmax]."""
    rho, mu, phi = spherical(r)
    out = np.zeros(rho.shape + (nmax + 1, 2 * nmax + 1), dtype=np.complex128)
    for m in range(0, nmax + 1):
        eim = np.exp(1j * m * phi)
        for n in range(m, nmax + 1):
            P = legendre(n, m, mu)
            if regular:
                val = ((-1.0) ** n * (1j ** m) / fact(n + m)) * rho ** n * P
            else:
                val = ((1j ** (-m)) * fact(n - m)) / rho ** (n + 1) * P
            out[..., n, m + nmax] = val * eim
            out[..., n, -m + nmax] = val * np.conj(eim)      # e^{-i m phi}; |m| enters elsewhere
    return out


def R_table(nmax, r):
    """All R_n^m(r) for n <= nmax: array [..., n, m + nmax]."""
    return _table(True, nmax, r)


def S_table(nmax, r):
    """All S_n^m(r) for n <= nmax: array [..., n, m + nmax]."""
    return _table(False, nmax, r)
