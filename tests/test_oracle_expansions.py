"""Pins of the oracle's P2M (Sec. 4.3) and local-expansion evaluation (Sec. 4.5)."""
import numpy as np

from oracle import expansions, operators
from tests.lh_util import biot_savart, fd_grad, lh_velocity, potential, real_coeffs


def test_p2m_methods_agree(rng):
    """Eq. eve4 (method 2) equals Eqs. eve5-eve10 (method 1, dipoles)."""
    p = 12
    x = rng.uniform(-0.2, 0.2, (7, 3))
    w = rng.normal(size=(7, 3))
    c = np.array([0.01, -0.02, 0.015])
    a = expansions.p2m_method2(x, w, c, p)
    b = expansions.p2m_method1(x, w, c, p)
    scale = max(np.abs(a[0]).max(), np.abs(a[1]).max())
    np.testing.assert_allclose(a[0], b[0], atol=1e-12 * scale)
    np.testing.assert_allclose(a[1], b[1], atol=1e-12 * scale)
    assert np.all(a[1][0] == 0)               # chi_0^0 = 0 (Eq. eve4)


def test_p2m_single_element_far_field(rng):
    """One element: the S-expansion's Lamb-Helmholtz velocity equals Eq. 1."""
    p = 30
    x = np.array([[0.12, -0.07, 0.09]])
    w = np.array([[0.3, -1.1, 0.6]])
    phi, chi = expansions.p2m_method2(x, w, np.zeros(3), p)
    y = np.array([[1.5, 0.7, -0.4], [-0.9, 1.2, 1.1]])
    v = lh_velocity(phi, chi, y, "S", h=1e-4).real
    want = biot_savart(x, w, y)
    assert np.abs(v - want).max() < 3e-10 * np.abs(want).max()


def test_p2m_coefficients_are_real_symmetric(rng):
    p = 9
    x = rng.uniform(-0.2, 0.2, (5, 3))
    w = rng.normal(size=(5, 3))
    for c in expansions.p2m_method2(x, w, np.zeros(3), p):
        for n in range(p):
            for m in range(n + 1):
                assert abs(c[n, -m + p - 1] - (-1) ** m * np.conj(c[n, m + p - 1])) < 1e-14
            assert abs(c[n, p - 1].imag) < 1e-15


def test_velocity_coefficients_match_field(rng):
    """Eq. evf3: sum_k v_{kn}^m R_n^m equals grad phi + curl(r chi) (finite differences)."""
    p = 9
    phi = real_coeffs(p, rng)
    chi = real_coeffs(p, rng)
    r = rng.normal(size=(5, 3)) * 0.3
    vc = expansions.velocity_coefficients(phi, chi)
    got = np.stack([potential(vc[k], r, "R") for k in range(3)], axis=1)
    want = lh_velocity(phi, chi, r, "R", h=1e-3)
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()


def test_gradient_and_stretching(rng):
    """u_{lk} = d_l v_k (Eq. dt3 with t = i_l), trace u = 0 (Eq. 3), s = w . u (Eq. evf6)."""
    p = 9
    phi = real_coeffs(p, rng)
    chi = real_coeffs(p, rng)
    r = rng.normal(size=(4, 3)) * 0.3
    w = rng.normal(size=(4, 3))
    v, u, s = expansions.l2p(phi, chi, r, w)
    vc = expansions.velocity_coefficients(phi, chi)
    for k in range(3):
        g = fd_grad(lambda q: potential(vc[k], q, "R"), r, 1e-3).real
        np.testing.assert_allclose(u[:, :, k], g, atol=1e-8 * np.abs(g).max())
    assert np.abs(np.trace(u, axis1=1, axis2=2)).max() < 1e-12 * np.abs(u).max()
    np.testing.assert_allclose(s, np.einsum("il,ilk->ik", w, u), rtol=1e-14)
    # evf5 form: s_k = sum (D_w v_k) R, D_w applied per point
    for i in range(4):
        sk = [potential(operators.apply_Dt(vc[k], w[i], "R"), r[i:i + 1], "R")[0].real for k in range(3)]
        np.testing.assert_allclose(s[i], sk, rtol=1e-11, atol=1e-12 * np.abs(s).max())
