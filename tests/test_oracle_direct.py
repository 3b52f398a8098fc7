"""Pins of the direct smoothed Biot-Savart sum (O1): Eqs. 1, 2, vem1, s1.1."""
import math

import numpy as np
import pytest

from oracle import direct


def test_singular_closed_form():
    """Eq. 1 for one source: v = w x (y - x) / |y - x|^3."""
    x = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 1.2]])
    w = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, -0.5]])
    v, u, s = direct.direct(x, w, 0.0)
    d = x[0] - x[1]
    np.testing.assert_allclose(v[0], np.cross(w[1], d) / np.linalg.norm(d) ** 3, rtol=1e-15)
    np.testing.assert_allclose(v[1], 0.0)


def test_core_limits():
    """Eq. vem1: K -> 1 for r >> a; K ~ sqrt(2/pi) x^3 / 3 for x = r/a -> 0; dK/dr by differences."""
    a = 0.01
    assert abs(direct.core_K(12 * a, a) - 1.0) < 1e-20 + 1e-15
    x = 1e-3
    assert direct.core_K(x * a, a) == pytest.approx(math.sqrt(2 / math.pi) * x ** 3 / 3, rel=1e-5)
    for r in (0.3 * a, a, 2.5 * a, 5 * a):
        h = 1e-3 * a
        K = lambda q: direct.core_K(q, a)
        fd = (-K(r + 2 * h) + 8 * K(r + h) - 8 * K(r - h) + K(r - 2 * h)) / (12 * h)
        assert direct.core_dK(r, a) == pytest.approx(fd, rel=1e-8)


def test_core_series_to_high_precision():
    """Eq. vem1 against a 40-digit evaluation (mpmath)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    a = 0.02
    for x in (0.5, 1.0, 3.0, 6.0):
        want = mp.erf(mp.mpf(x) / mp.sqrt(2)) - mp.sqrt(2 / mp.pi) * x * mp.exp(-mp.mpf(x) ** 2 / 2)
        assert float(direct.core_K(x * a, a)) == pytest.approx(float(want), rel=1e-14)


@pytest.mark.parametrize("a", [0.0, 0.05])
def test_gradient_by_differences(rng, a):
    """u_{lk} = d_l v_k of Eq. 2 at a target, by central differences of the sum."""
    x = rng.uniform(0, 0.3, (6, 3))
    w = rng.normal(size=(6, 3))
    v, u, s = direct.direct(x, w, a)
    h = 1e-6
    for l in range(3):
        xp, xm = x.copy(), x.copy()
        xp[0, l] += h
        xm[0, l] -= h
        vp = direct.direct_at(xp, w, a, [0])[0][0]
        vm = direct.direct_at(xm, w, a, [0])[0][0]
        np.testing.assert_allclose(u[0, l], (vp - vm) / (2 * h), rtol=1e-6, atol=1e-6 * np.abs(u[0]).max())


@pytest.mark.parametrize("a", [0.0, 0.05])
def test_divergence_free_and_stretching(rng, a):
    """div v = trace(u) = 0 (Eq. 3) and s = w_i . grad v (Eq. s1.1)."""
    x = rng.uniform(0, 0.3, (30, 3))
    w = rng.normal(size=(30, 3))
    v, u, s = direct.direct(x, w, a)
    assert np.abs(np.trace(u, axis1=1, axis2=2)).max() < 1e-12 * np.abs(u).max()
    np.testing.assert_allclose(s, np.einsum("il,ilk->ik", w, u), rtol=1e-13)


def test_smoothed_equals_singular_beyond_core(rng):
    """Eq. 2: K = 1 + O(eps) for r >> a."""
    x = rng.uniform(0, 1, (40, 3))
    w = rng.normal(size=(40, 3))
    a = 1e-4
    v0, u0, s0 = direct.direct(x, w, 0.0)
    v1, u1, s1 = direct.direct(x, w, a)
    np.testing.assert_allclose(v1, v0, rtol=1e-12)
    np.testing.assert_allclose(s1, s0, rtol=1e-10)


def test_coincident_distinct_elements_are_regular():
    """With a > 0, two distinct elements at one point interact through K (finite);
    the element itself is excluded by index."""
    x = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3 + 1e-3]])
    w = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    v, u, s = direct.direct(x, w, 0.01)
    assert np.all(np.isfinite(v)) and np.all(np.isfinite(u))


def test_coincident_limit_is_continuous():
    """f = K/r^3 and f'/r at r = 0 (Eq. vem1 limits) continue the values at tiny r."""
    a = 0.05
    w = np.array([[0.3, -0.2, 0.9]])
    v0, u0 = direct.pair_terms(np.zeros((1, 3)), w, a)
    v1, u1 = direct.pair_terms(np.array([[1e-4 * a, 0.0, 0.0]]), w, a)
    assert np.all(v0 == 0)
    np.testing.assert_allclose(u0, u1, rtol=1e-6, atol=1e-9 * np.abs(u1).max())
