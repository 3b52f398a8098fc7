"""Pins of the oracle's translation, differential and conversion operators."""
import numpy as np
import pytest

from oracle import basis, expansions, operators
from tests.lh_util import fd_grad, lh_velocity, lh_velocity_shifted, potential, real_coeffs


def _green(x0, p):
    """S coefficients of |r - x0|^{-1} about the origin (Eq. rsbf5): R_n^{-m}(-x0)."""
    tab = basis.R_table(p - 1, -np.asarray(x0))
    return tab[..., ::-1]


def test_RR_exact_on_polynomials(rng):
    """Eq. mr3 (R|R): a truncated local expansion is a polynomial; its translate is exact."""
    p = 8
    c = real_coeffs(p, rng)
    t = np.array([0.21, -0.13, 0.32])
    ch = operators.translate("RR", c, t)
    r = rng.normal(size=(12, 3)) * 0.3
    np.testing.assert_allclose(potential(ch, r, "R"), potential(c, r + t, "R"), rtol=1e-12, atol=1e-13)


def test_SS_exact_on_green_function():
    """Eq. mr3 (S|S) is lower triangular in n: translating the Green's-function
    coefficients gives, degree by degree, the coefficients about the new centre."""
    p = 10
    x0 = np.array([0.05, -0.08, 0.11])
    t = np.array([-0.25, 0.25, 0.25])          # new centre - old centre
    got = operators.translate("SS", _green(x0, p), t)
    want = _green(x0 - t, p)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def test_SR_converges_with_p():
    """Eq. mr3 (S|R): local expansion of a distant multipole, error falls with p."""
    x0 = np.array([0.1, -0.05, 0.12])
    t = np.array([2.0, 0.5, -1.0])             # target centre - source centre
    r = np.array([[0.2, 0.1, -0.25], [-0.3, 0.2, 0.1]])
    exact = 1.0 / np.linalg.norm(r + t - x0, axis=1)
    errs = []
    for p in (4, 8, 12, 16, 20):
        loc = operators.translate("SR", _green(x0, p), t)
        errs.append(np.abs(potential(loc, r, "R") - exact).max() / np.abs(exact).max())
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-11, errs


def _elements(rng, k=5, spread=0.15):
    x = rng.uniform(-spread, spread, (k, 3))
    w = rng.normal(size=(k, 3))
    return x, w


def test_S_conversion_restores_p2m_about_new_centre(rng):
    """Eq. drt11 after (S|S): identical coefficients to a direct P2M about the new
    centre (only chi_0^0 is free, Eq. dr3); without the conversion they differ O(1)."""
    p = 10
    x, w = _elements(rng)
    t = np.array([0.25, -0.25, 0.25])
    phi0, chi0 = expansions.p2m_method2(x, w, np.zeros(3), p)
    phi1, chi1 = expansions.p2m_method2(x, w, t, p)
    ph = operators.translate("SS", phi0, t)
    ch = operators.translate("SS", chi0, t)
    pt, ct = operators.convert_S(ph, ch, t)
    ct[0, p - 1] = chi1[0, p - 1]
    scale = max(np.abs(phi1).max(), np.abs(chi1).max())
    np.testing.assert_allclose(pt, phi1, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(ct, chi1, rtol=0, atol=1e-12 * scale)
    assert np.abs(ph - phi1).max() > 1e-2 * scale


def test_S_conversion_far_field_velocity(rng):
    """The converted multipole reproduces the Biot-Savart field (Eq. 1) about the new centre."""
    from tests.lh_util import biot_savart
    p = 18
    x, w = _elements(rng)
    t = np.array([0.25, 0.25, -0.25])
    phi0, chi0 = expansions.p2m_method2(x, w, np.zeros(3), p)
    pt, ct = operators.convert_S(operators.translate("SS", phi0, t), operators.translate("SS", chi0, t), t)
    y = np.array([[2.0, 1.0, 0.5], [-1.5, 2.2, 0.3]])
    v = lh_velocity(pt, ct, y - t, "S", h=1e-4).real
    want = biot_savart(x, w, y)
    assert np.abs(v - want).max() < 1e-8 * np.abs(want).max()


def test_R_conversion_on_polynomial_pair(rng):
    """Eq. drt10 after (R|R): v~(r) = v(r + t) exactly for a pair of degree <= p-2;
    with the conversion omitted the field is wrong at O(1)."""
    p = 8
    phi = real_coeffs(p, rng)
    chi = real_coeffs(p, rng)
    phi[p - 1] = 0
    chi[p - 1] = 0
    t = np.array([0.3, -0.2, 0.15])
    ph, ch = operators.translate("RR", phi, t), operators.translate("RR", chi, t)
    pt, ct = operators.convert_R(ph, ch, t)
    r = rng.normal(size=(6, 3)) * 0.2
    want = lh_velocity_shifted(phi, chi, r, t, "R", h=1e-3)
    got = lh_velocity(pt, ct, r, "R", h=1e-3)
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()
    bad = lh_velocity(ph, ch, r, "R", h=1e-3)
    assert np.abs(bad - want).max() > 1e-2 * np.abs(want).max()


def test_M2L_with_conversion_reproduces_field(rng):
    """(S|R) then Eq. drt10: the local pair about a distant centre gives the
    Biot-Savart velocity of the source elements, error falling with p."""
    from tests.lh_util import biot_savart
    x, w = _elements(rng, spread=0.1)
    t = np.array([0.0, 0.0, 1.0]) * 1.0 + np.array([0.6, -0.4, 0.0])   # target centre
    y = t + np.array([[0.1, -0.05, 0.08], [-0.09, 0.1, -0.02]])
    want = biot_savart(x, w, y)
    errs = []
    for p in (6, 10, 14):
        phi0, chi0 = expansions.p2m_method2(x, w, np.zeros(3), p)
        pt, ct = operators.convert_R(operators.translate("SR", phi0, t), operators.translate("SR", chi0, t), t)
        v = lh_velocity(pt, ct, y - t, "R", h=1e-4).real
        errs.append(np.abs(v - want).max() / np.abs(want).max())
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-6, errs


@pytest.mark.parametrize("b", ["R", "S"])
def test_Dt_matches_directional_derivative(rng, b):
    """Eq. dt3: coefficients of t . grad f."""
    p = 7
    c = real_coeffs(p, rng)
    t = np.array([0.4, -0.7, 0.3])
    r = np.array([[0.3, 0.2, -0.1]]) if b == "R" else np.array([[1.3, 0.9, -1.1]])
    if b == "S":
        c[p - 1] = 0          # D_t raises the degree in the S basis (Eq. dt2): keep it representable
    d = operators.apply_Dt(c, t, b)
    g = fd_grad(lambda q: potential(c, q, b), r, 1e-4)
    want = (g * t).sum(axis=1)
    np.testing.assert_allclose(potential(d, r, b), want, rtol=1e-8, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("b", ["R", "S"])
def test_Drxt_matches_rotational_derivative(rng, b):
    """Eq. drt7: coefficients of (r x t) . grad f."""
    p = 7
    c = real_coeffs(p, rng)
    t = np.array([-0.2, 0.5, 0.8])
    r = np.array([[0.3, 0.2, -0.1]]) if b == "R" else np.array([[1.3, 0.9, -1.1]])
    d = operators.apply_Drxt(c, t, b)
    g = fd_grad(lambda q: potential(c, q, b), r, 1e-4)
    want = (g * np.cross(r, t)).sum(axis=1)
    np.testing.assert_allclose(potential(d, r, b), want, rtol=1e-8, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("b", ["R", "S"])
def test_Dr_matches_radial_derivative(rng, b):
    p = 7
    c = real_coeffs(p, rng)
    r = np.array([[0.3, 0.2, -0.1]]) if b == "R" else np.array([[1.3, 0.9, -1.1]])
    d = operators.apply_Dr(c, b)
    g = fd_grad(lambda q: potential(c, q, b), r, 1e-4)
    want = (g * r).sum(axis=1)
    np.testing.assert_allclose(potential(d, r, b), want, rtol=1e-8, atol=1e-9 * np.abs(want).max())


def test_conversion_matches_CVL14_operator_form(rng):
    """Eq. CVL14 with the matrices of App. A (Eqs. dr4, dt3, drt7) gives the same
    result as the compact forms of Eqs. drt10 and drt11."""
    p = 7
    phi = real_coeffs(p, rng)
    chi = real_coeffs(p, rng)
    t = np.array([0.3, -0.6, 0.2])
    n = np.arange(p)[:, None]
    # R basis: C12 = -D_r^{-1} D_{r x t}, C22 = I + (I + D_r)^{-1} D_t, D_r^{-1} = 1/n (0 at n = 0)
    inv_dr = np.where(n > 0, 1.0 / np.maximum(n, 1), 0.0)
    pt = phi - inv_dr * operators.apply_Drxt(chi, t, "R")
    ct = chi + operators.apply_Dt(chi, t, "R") / (n + 1)
    got = operators.convert_R(phi, chi, t)
    np.testing.assert_allclose(got[0], pt, atol=1e-13)
    np.testing.assert_allclose(got[1], ct, atol=1e-13)
    # S basis: D_r^{-1} = -1/(n+1), (I + D_r)^{-1} = -1/n (0 at n = 0)
    pt = phi + operators.apply_Drxt(chi, t, "S") / (n + 1)
    ct = chi - np.where(n > 0, 1.0 / np.maximum(n, 1), 0.0) * operators.apply_Dt(chi, t, "S")
    got = operators.convert_S(phi, chi, t)
    np.testing.assert_allclose(got[0], pt, atol=1e-13)
    np.testing.assert_allclose(got[1], ct, atol=1e-13)


def test_coaxial_special_case(rng):
    """With t = t i_z the conversions reduce to Eq. rcr1."""
    p = 7
    phi = real_coeffs(p, rng)
    chi = real_coeffs(p, rng)
    tz = 0.37
    g = operators.get
    pr, cr = operators.convert_R(phi, chi, (0.0, 0.0, tz))
    ps, cs = operators.convert_S(phi, chi, (0.0, 0.0, tz))
    for n in range(p):
        for m in range(-n, n + 1):
            i = m + p - 1
            want = g(phi, n, m) + (1j * tz * m / n * g(chi, n, m) if n > 0 else 0)
            assert abs(pr[n, i] - want) < 1e-13
            assert abs(cr[n, i] - (g(chi, n, m) - tz / (n + 1) * g(chi, n + 1, m))) < 1e-13
            assert abs(ps[n, i] - (g(phi, n, m) - 1j * tz * m / (n + 1) * g(chi, n, m))) < 1e-13
            want = g(chi, n, m) + (tz / n * g(chi, n - 1, m) if n > 0 else 0)
            assert abs(cs[n, i] - want) < 1e-13
