"""Translation, differential and conversion operators on coefficient arrays (FP64).

Test infrastructure (see ``oracle/__init__``).

Coefficient arrays are complex, shape (p, 2p-1), c_n^m at ``c[n, m + p - 1]``.
Terms beyond the truncation (n >= p or |m| > n) are zero.

* Translations: Eq. mr3 gives the reexpansion coefficients (F|G)_{n'n}^{m'm}(t);
  Eq. mr2 says that the coefficient map is their transpose:
  new_{n'}^{m'} = sum_{n,m} (F|G)_{n'n}^{m'm}(t) old_n^m.  The translation vector
  is t = (new centre) - (old centre) (Eq. bas1: phi_hat(r) = phi(r + t)).
* Differential operators in coefficient form: D_r (Eq. dr2), D_t (Eq. dt3),
  D_{r x t} (Eq. drt7), in the R and S bases.
* Conversions: Eq. drt10 (R expansions, after M2L and L2L) and Eq. drt11
  (S expansions, after M2M), transcribed term by term.
"""
import functools

import numpy as np

from .basis import R_table, S_table

__all__ = [
    "get", "empty", "translation_matrix", "translate", "C",
    "apply_Dr", "apply_Dt", "apply_Drxt", "convert_R", "convert_S",
    "flatten", "unflatten", "resize",
]


def empty(p):
    return np.zeros((p, 2 * p - 1), dtype=np.complex128)


def resize(c, p):
    """The same expansion with p terms (n < p): truncated, or padded with zeros."""
    q = c.shape[0]
    out = empty(p)
    k = min(p, q)
    out[:k, p - 1 - (k - 1): p - 1 + k] = c[:k, q - 1 - (k - 1): q - 1 + k]
    return out


def get(c, n, m):
    """c_n^m with the truncation/zero conventions of Eq. rsbf7."""
    p = c.shape[0]
    if n < 0 or n >= p or abs(m) > n:
        return 0.0 + 0.0j
    return c[n, m + p - 1]


@functools.lru_cache(maxsize=None)
def _flat_pos(p):
    """(row, column) of the (p, 2p-1) array for flat index n*n + n + m."""
    rows, cols = [], []
    for n in range(p):
        for m in range(-n, n + 1):
            rows.append(n)
            cols.append(m + p - 1)
    return np.array(rows), np.array(cols)


def flatten(c):
    """(p, 2p-1) array -> vector over (n, m), index n*n + n + m."""
    rows, cols = _flat_pos(c.shape[0])
    return c[rows, cols]


def unflatten(v, p):
    c = empty(p)
    rows, cols = _flat_pos(p)
    c[rows, cols] = v
    return c


@functools.lru_cache(maxsize=None)
def _index_sets(p):
    """All (n', m', n, m) with n, n' < p, |m| <= n, |m'| <= n'."""
    rows = []
    for n2 in range(p):
        for m2 in range(-n2, n2 + 1):
            for n in range(p):
                for m in range(-n, n + 1):
                    rows.append((n2 * n2 + n2 + m2, n * n + n + m, n2, m2, n, m))
    return np.array(rows, dtype=np.int64)


def translation_matrix(kind, t, p):
    """Dense p^2 x p^2 map new = T @ old for one translation by t (Eqs. mr2, mr3).

    kind: "RR" (local to local, (R|R) = R_{n-n'}^{m-m'}(t)),
          "SR" (multipole to local, (S|R) = S_{n+n'}^{m-m'}(t)),
          "SS" (multipole to multipole, (S|S) = R_{n'-n}^{m-m'}(t)).
    Entries whose basis function has negative degree or |order| > degree are 0."""
    idx = _index_sets(p)
    out_i, in_i, n2, m2, n, m = (idx[:, k] for k in range(6))
    T = np.zeros((p * p, p * p), dtype=np.complex128)
    mu = m - m2
    if kind == "RR":
        deg = n - n2
        tab = R_table(p - 1, np.asarray(t, dtype=np.float64))
        nmax = p - 1
    elif kind == "SS":
        deg = n2 - n
        tab = R_table(p - 1, np.asarray(t, dtype=np.float64))
        nmax = p - 1
    elif kind == "SR":
        deg = n + n2
        tab = S_table(2 * p - 2, np.asarray(t, dtype=np.float64))
        nmax = 2 * p - 2
    else:
        raise ValueError(kind)
    ok = (deg >= 0) & (np.abs(mu) <= deg)
    T[out_i[ok], in_i[ok]] = tab[deg[ok], mu[ok] + nmax]
    return T


def translate(kind, c, t):
    p = c.shape[0]
    return unflatten(translation_matrix(kind, t, p) @ flatten(c), p)


# ---------------------------------------------------------------------------
# Shifted access: C(c, dn, dm)[n, m] = c_{n+dn}^{m+dm} for every (n, m) at once
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=None)
def _grid(p):
    n = np.arange(p)[:, None] * np.ones((1, 2 * p - 1))
    m = np.arange(-(p - 1), p)[None, :] * np.ones((p, 1))
    n.setflags(write=False)
    m.setflags(write=False)
    return n, m


@functools.lru_cache(maxsize=None)
def _valid(p):
    n, m = _grid(p)
    v = np.abs(m) <= n
    v.setflags(write=False)
    return v


def C(c, dn, dm):
    """Array whose (..., n, m) entry is c_{n+dn}^{m+dm}, zero outside the truncation.

    ``c`` has shape (..., p, 2p-1); leading axes are carried along."""
    p = c.shape[-2]
    pad = np.zeros(c.shape[:-2] + (p + 2, 2 * p + 1), dtype=np.complex128)
    pad[..., 1:p + 1, 1:2 * p] = c * _valid(p)
    return pad[..., 1 + dn: 1 + dn + p, 1 + dm: 1 + dm + 2 * p - 1]


# ---------------------------------------------------------------------------
# Differential operators in coefficient form (Appendix A)
# ---------------------------------------------------------------------------

def apply_Dr(c, basis):
    """Eq. dr2: D_r is diagonal, n in the R basis and -(n+1) in the S basis."""
    n, m = _grid(c.shape[-2])
    lam = n if basis == "R" else -(n + 1)
    return lam * c * _valid(c.shape[-2])


def apply_Dt(c, t, basis):
    """Eq. dt3: coefficients of D_t f, f = sum c_n^m F_n^m (F = R or S).

    R basis: (D c)_n^m = 1/2 (t_y + i t_x) c_{n+1}^{m-1} - 1/2 (t_y - i t_x) c_{n+1}^{m+1} - t_z c_{n+1}^m
    S basis: the same with n-1 in place of n+1."""
    tx, ty, tz = (float(v) for v in t)
    s = 1 if basis == "R" else -1
    out = (0.5 * (ty + 1j * tx) * C(c, s, -1)
           - 0.5 * (ty - 1j * tx) * C(c, s, +1)
           - tz * C(c, s, 0))
    return out * _valid(c.shape[-2])


def apply_Drxt(c, t, basis):
    """Eq. drt7: coefficients of D_{r x t} f (diagonal in n).

    R basis: (D c)_n^m = (t_x + i t_y)(n-m)/2 c_n^{m+1} - (t_x - i t_y)(n+m)/2 c_n^{m-1} - i t_z m c_n^m
    S basis: (D c)_n^m = -(t_x + i t_y)(n+m+1)/2 c_n^{m+1} + (t_x - i t_y)(n-m+1)/2 c_n^{m-1} - i t_z m c_n^m
    (row (n, m) of the matrices of Eq. drt7: n' = n and m' = m + 1, m - 1 or m)."""
    tx, ty, tz = (float(v) for v in t)
    n, m = _grid(c.shape[-2])
    if basis == "R":
        out = ((tx + 1j * ty) * (n - m) / 2.0 * C(c, 0, +1)
               - (tx - 1j * ty) * (n + m) / 2.0 * C(c, 0, -1)
               - 1j * tz * m * C(c, 0, 0))
    else:
        out = (-(tx + 1j * ty) * (n + m + 1) / 2.0 * C(c, 0, +1)
               + (tx - 1j * ty) * (n - m + 1) / 2.0 * C(c, 0, -1)
               - 1j * tz * m * C(c, 0, 0))
    return out * _valid(c.shape[-2])


# ---------------------------------------------------------------------------
# Conversion operators (Appendix A.4)
# ---------------------------------------------------------------------------

def convert_R(phi_hat, chi_hat, t):
    """Eq. drt10: restore the Lamb-Helmholtz form of translated R expansions.

    phi~_n^m = phi^_n^m - 1/n [ (t_x + i t_y)(n-m)/2 chi^_n^{m+1}
                               - (t_x - i t_y)(n+m)/2 chi^_n^{m-1} - i t_z m chi^_n^m ],
               phi~_0^0 = phi^_0^0
    chi~_n^m = chi^_n^m + 1/(n+1) [ 1/2 (t_y + i t_x) chi^_{n+1}^{m-1}
                                   - 1/2 (t_y - i t_x) chi^_{n+1}^{m+1} - t_z chi^_{n+1}^m ]
    chi^ beyond the truncation (n + 1 = p) is zero."""
    tx, ty, tz = (float(v) for v in t)
    p = phi_hat.shape[-2]
    n, m = _grid(p)
    c = chi_hat
    inv_n = np.where(n > 0, 1.0 / np.maximum(n, 1), 0.0)      # the n = 0 row of phi is unchanged
    dphi = -inv_n * ((tx + 1j * ty) * (n - m) / 2.0 * C(c, 0, +1)
                     - (tx - 1j * ty) * (n + m) / 2.0 * C(c, 0, -1)
                     - 1j * tz * m * C(c, 0, 0))
    dchi = (1.0 / (n + 1)) * (0.5 * (ty + 1j * tx) * C(c, 1, -1)
                              - 0.5 * (ty - 1j * tx) * C(c, 1, +1)
                              - tz * C(c, 1, 0))
    v = _valid(p)
    return (phi_hat + dphi) * v, (chi_hat + dchi) * v


def convert_S(phi_hat, chi_hat, t):
    """Eq. drt11: restore the Lamb-Helmholtz form of translated S expansions.

    phi~_n^m = phi^_n^m + 1/(n+1) [ -(t_x + i t_y)(n+m+1)/2 chi^_n^{m+1}
                                   + (t_x - i t_y)(n-m+1)/2 chi^_n^{m-1} - i t_z m chi^_n^m ]
    chi~_n^m = chi^_n^m - 1/n [ 1/2 (t_y + i t_x) chi^_{n-1}^{m-1}
                               - 1/2 (t_y - i t_x) chi^_{n-1}^{m+1} - t_z chi^_{n-1}^m ],
               chi~_0^0 = chi^_0^0"""
    tx, ty, tz = (float(v) for v in t)
    p = phi_hat.shape[-2]
    n, m = _grid(p)
    c = chi_hat
    dphi = (1.0 / (n + 1)) * (-(tx + 1j * ty) * (n + m + 1) / 2.0 * C(c, 0, +1)
                              + (tx - 1j * ty) * (n - m + 1) / 2.0 * C(c, 0, -1)
                              - 1j * tz * m * C(c, 0, 0))
    inv_n = np.where(n > 0, 1.0 / np.maximum(n, 1), 0.0)      # the n = 0 row of chi is unchanged
    dchi = -inv_n * (0.5 * (ty + 1j * tx) * C(c, -1, -1)
                     - 0.5 * (ty - 1j * tx) * C(c, -1, +1)
                     - tz * C(c, -1, 0))
    v = _valid(p)
    return (phi_hat + dphi) * v, (chi_hat + dchi) * v
