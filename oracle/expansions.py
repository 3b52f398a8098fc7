"""Multipole generation (Sec. 4.3) and local-expansion evaluation (Sec. 4.5), FP64.

Test infrastructure (see ``oracle/__init__``).
"""
import numpy as np

from .basis import R_table, S_table
from .operators import C, _grid, _valid, apply_Dt, empty

__all__ = [
    "p2m_method2", "p2m_method1", "eval_R", "eval_S",
    "velocity_coefficients", "gradient_coefficients", "l2p",
]


def _neg_m(tab, nmax):
    """tab[..., n, m] -> tab[..., n, -m] (maps R_n^m to R_n^{-m})."""
    return tab[..., ::-1]


def _g_table(r_l, p):
    """g_{ln}^m = R_n^{-m}(-r_l) of Eq. eve1, for n < p (array [..., n, m + p - 1])."""
    return _neg_m(R_table(p - 1, -np.asarray(r_l, dtype=np.float64)), p - 1)


def p2m_method2(x, w, centre, p):
    """Sec. 4.3.2, Eq. eve4: S-expansion coefficients (phi, chi) of the elements
    at x (N, 3) with strengths w (N, 3) about ``centre``, summed over the elements.

    phi_n^m = 1/(n+1) [ (w_x - i w_y)(n-m+1)/2 g_n^{m-1} - (w_x + i w_y)(n+m+1)/2 g_n^{m+1}
                        - i w_z m g_n^m ]
    chi_n^m = -1/n [ 1/2 (w_y + i w_x) g_{n-1}^{m-1} - 1/2 (w_y - i w_x) g_{n-1}^{m+1}
                     - w_z g_{n-1}^m ],  chi_0^0 = 0
    with g_n^m = R_n^{-m}(-r_l), r_l = x_l - centre."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    w = np.asarray(w, dtype=np.float64).reshape(-1, 3)
    if x.shape[0] == 0:
        return empty(p), empty(p)
    g = _g_table(x - np.asarray(centre, dtype=np.float64), p)          # (N, p, 2p-1)
    n, m = _grid(p)
    wx, wy, wz = (w[:, k][:, None, None] for k in range(3))
    phi = (1.0 / (n + 1)) * ((wx - 1j * wy) * (n - m + 1) / 2.0 * C(g, 0, -1)
                             - (wx + 1j * wy) * (n + m + 1) / 2.0 * C(g, 0, +1)
                             - 1j * wz * m * C(g, 0, 0))
    inv_n = np.where(n > 0, 1.0 / np.maximum(n, 1), 0.0)                 # chi_0^0 = 0
    chi = -inv_n * (0.5 * (wy + 1j * wx) * C(g, -1, -1)
                    - 0.5 * (wy - 1j * wx) * C(g, -1, +1)
                    - wz * C(g, -1, 0))
    v = _valid(p)
    return (phi * v).sum(axis=0), (chi * v).sum(axis=0)


def _dipole_coefficients(r_l, moment, p):
    """S-expansion of the dipole q.(r - r_l)/|r - r_l|^3 about the origin.

    The dipole equals (q . grad_{r_l}) |r - r_l|^{-1}; with Eq. rsbf5 its
    coefficients are (q . grad_{r_l}) R_n^{-m}(-r_l) = -[(D_q R_n^{-m})](-r_l),
    and Eq. dt2 gives D_q R_n^mu = 1/2[(q_y + i q_x) R_{n-1}^{mu+1}
    - (q_y - i q_x) R_{n-1}^{mu-1}] - q_z R_{n-1}^mu."""
    Rm = R_table(p - 1, -np.asarray(r_l, dtype=np.float64))              # R_n^mu(-r_l), [.., n, mu]
    qx, qy, qz = (np.asarray(moment)[:, k][:, None, None] for k in range(3))
    # entry (n, m) needs mu = -m: R_{n-1}^{-m+1}, R_{n-1}^{-m-1}, R_{n-1}^{-m}
    Rneg = _neg_m(Rm, p - 1)                                             # [.., n, m] = R_n^{-m}
    out = -(0.5 * ((qy + 1j * qx) * C(Rneg, -1, -1) - (qy - 1j * qx) * C(Rneg, -1, +1))
            - qz * C(Rneg, -1, 0))
    return out * _valid(p)


def p2m_method1(x, w, centre, p):
    """Sec. 4.3.1, Eqs. eve5-eve10: psi is a dipole of moment r_l x w_l, varpi a
    dipole of moment -w_l, and phi_n^m = -psi_n^m/(n+1), chi_n^m = -varpi_n^m/n
    (chi_0^0 = 0)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    w = np.asarray(w, dtype=np.float64).reshape(-1, 3)
    r_l = x - np.asarray(centre, dtype=np.float64)
    psi = _dipole_coefficients(r_l, np.cross(r_l, w), p)
    varpi = _dipole_coefficients(r_l, -w, p)
    n, m = _grid(p)
    phi = -psi / (n + 1)
    chi = -np.where(n > 0, 1.0 / np.maximum(n, 1), 0.0) * varpi
    return phi.sum(axis=0), chi.sum(axis=0)


def eval_R(c, r):
    """sum_{n,m} c_n^m R_n^m(r) at points r (..., 3) (Eq. rsbf6, F = R)."""
    p = c.shape[-2]
    return np.einsum("...nm,nm->...", R_table(p - 1, r), c)


def eval_S(c, r):
    """sum_{n,m} c_n^m S_n^m(r) at points r (..., 3) (Eq. rsbf6, F = S)."""
    p = c.shape[-2]
    return np.einsum("...nm,nm->...", S_table(p - 1, r), c)


def velocity_coefficients(phi, chi):
    """Eq. evf3: R-expansion coefficients v_{kn}^m of the three velocity
    components, from the local expansions of phi and chi.

    v_x = 1/2 [ i phi_{n+1}^{m-1} + i phi_{n+1}^{m+1} + (n-m) chi_n^{m+1} - (n+m) chi_n^{m-1} ]
    v_y = 1/2 [ phi_{n+1}^{m-1} - phi_{n+1}^{m+1} + i (n-m) chi_n^{m+1} + i (n+m) chi_n^{m-1} ]
    v_z = -phi_{n+1}^m - i m chi_n^m"""
    p = phi.shape[-2]
    n, m = _grid(p)
    vx = 0.5 * (1j * C(phi, 1, -1) + 1j * C(phi, 1, +1)
                + (n - m) * C(chi, 0, +1) - (n + m) * C(chi, 0, -1))
    vy = 0.5 * (C(phi, 1, -1) - C(phi, 1, +1)
                + 1j * (n - m) * C(chi, 0, +1) + 1j * (n + m) * C(chi, 0, -1))
    vz = -C(phi, 1, 0) - 1j * m * C(chi, 0, 0)
    v = _valid(p)
    return np.stack([vx * v, vy * v, vz * v])                            # (3, p, 2p-1)


def gradient_coefficients(vcoef):
    """Sec. 4.5.2: u_{lk} = D_{i_l} v_k, by the R-basis matrix of D_t (Eq. dt3)
    with t = i_l.  Returns (3, 3, p, 2p-1) indexed [l, k]."""
    units = np.eye(3)
    return np.stack([np.stack([apply_Dt(vcoef[k], units[l], "R") for k in range(3)])
                     for l in range(3)])


def l2p(phi, chi, r, w):
    """Evaluate the local expansion (phi, chi) at points r (N, 3) relative to
    the box centre: velocity v (Eq. evf3), gradient u_{lk} = d_l v_k and the
    stretching s_k = sum_l w_l u_{lk} (Eqs. evf4-evf6), for strengths w (N, 3)."""
    p = phi.shape[-2]
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    Rt = R_table(p - 1, r)                                               # (N, p, 2p-1)
    vc = velocity_coefficients(phi, chi)
    uc = gradient_coefficients(vc)
    v = np.einsum("inm,knm->ik", Rt, vc).real
    grad = np.einsum("inm,lknm->ilk", Rt, uc).real
    s = np.einsum("il,ilk->ik", np.asarray(w, dtype=np.float64).reshape(-1, 3), grad)
    return v, grad, s
