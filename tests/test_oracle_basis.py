"""Pins of the oracle's solid harmonics (Sec. 3.3, Eqs. rsbf1-rsbf7)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import basis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "low_order_harmonics.txt")


def _rodrigues_poly(n, m):
    """Exact coefficients (low to high) of d^{n+m}/dmu^{n+m} (mu^2 - 1)^n / (2^n n!)."""
    coeffs = [Fraction(0)] * (2 * n + 1)
    for k in range(n + 1):      # (mu^2 - 1)^n = sum_k C(n,k) mu^{2k} (-1)^{n-k}
        coeffs[2 * k] = Fraction(math.comb(n, k) * (-1) ** (n - k))
    for _ in range(n + m):
        coeffs = [coeffs[i] * i for i in range(1, len(coeffs))] or [Fraction(0)]
    scale = Fraction(1, 2 ** n * math.factorial(n))
    return [c * scale for c in coeffs]


@pytest.mark.parametrize("n", range(0, 9))
def test_legendre_matches_rodrigues_exactly(n):
    """Eq. rsbf3 in exact rational arithmetic against the library routine."""
    for m in range(0, n + 1):
        poly = _rodrigues_poly(n, m)
        for mu in (Fraction(-7, 9), Fraction(-1, 3), Fraction(0), Fraction(2, 5), Fraction(5, 6)):
            val = sum(c * mu ** i for i, c in enumerate(poly))
            exact = (-1) ** m * float(val) * float(1 - mu * mu) ** (m / 2.0)
            got = float(basis.legendre(n, m, float(mu)))
            assert got == pytest.approx(exact, rel=1e-12, abs=1e-14)


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, n, m, expr = line.split(None, 3)
            rows.append((kind, int(n), int(m), expr))
    return rows


def test_low_order_closed_forms(rng):
    """Hand-derived Cartesian forms of R_n^m, S_n^m (n <= 2) fix the phase conventions."""
    pts = rng.normal(size=(20, 3))
    rows = _golden()
    assert len(rows) == 18
    for kind, n, m, expr in rows:
        for p in pts:
            x, y, z = p
            r = math.sqrt(x * x + y * y + z * z)
            want = complex(eval(expr, {}, dict(x=x, y=y, z=z, r=r)))
            got = complex((basis.R_nm if kind == "R" else basis.S_nm)(n, m, p))
            assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (kind, n, m)


def test_S_R_relation(rng):
    """Eq. rsbf4: S_n^m = (-1)^{n+m} (n-m)! (n+m)! r^{-2n-1} R_n^m."""
    pts = rng.normal(size=(10, 3))
    r = np.linalg.norm(pts, axis=1)
    R = basis.R_table(10, pts)
    S = basis.S_table(10, pts)
    for n in range(11):
        for m in range(-n, n + 1):
            want = (-1) ** (n + m) * basis.fact(n - m) * basis.fact(n + m) * r ** (-2 * n - 1) * R[:, n, m + 10]
            np.testing.assert_allclose(S[:, n, m + 10], want, rtol=1e-12, atol=0)


def test_real_symmetry(rng):
    """R_n^{-m} = (-1)^m conj(R_n^m), likewise for S (from Eq. rsbf2)."""
    pts = rng.normal(size=(10, 3))
    for tab in (basis.R_table(8, pts), basis.S_table(8, pts)):
        for n in range(9):
            for m in range(0, n + 1):
                np.testing.assert_allclose(tab[:, n, -m + 8], (-1) ** m * np.conj(tab[:, n, m + 8]),
                                           rtol=1e-13, atol=1e-300)


def test_green_expansion(rng):
    """Eq. rsbf5: |r - r0|^{-1} = sum R_n^{-m}(-r0) S_n^m(r), r > r0."""
    P = 45
    for _ in range(5):
        r0 = rng.normal(size=3)
        r0 *= 0.3 / np.linalg.norm(r0)
        r = rng.normal(size=3)
        r *= 1.0 / np.linalg.norm(r)
        Rm = basis.R_table(P, -r0)
        S = basis.S_table(P, r)
        total = 0.0
        for n in range(P + 1):
            for m in range(-n, n + 1):
                total += Rm[n, -m + P] * S[n, m + P]
        assert abs(total - 1.0 / np.linalg.norm(r - r0)) < 1e-13
        assert abs(total.imag) < 1e-14


def _laplacian(f, p, h=1e-3):
    """Five-point second differences per axis: (sum, largest single |d^2 f/dx_k^2|)."""
    out, big = 0.0, 0.0
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        d2 = (-f(p + 2 * e) + 16 * f(p + e) - 30 * f(p) + 16 * f(p - e) - f(p - 2 * e)) / (12 * h * h)
        out = out + d2
        big = max(big, abs(d2))
    return out, big


def test_harmonic(rng):
    """R_n^m and S_n^m solve the Laplace equation (finite differences)."""
    p = np.array([0.7, -0.4, 0.55])
    for n in range(0, 6):
        for m in range(-n, n + 1):
            for fn in (basis.R_nm, basis.S_nm):
                lap, big = _laplacian(lambda q: fn(n, m, q), p)
                assert abs(lap) < 1e-6 * big + 1e-8 * (1 + abs(fn(n, m, p))), (fn.__name__, n, m)


def _grad(f, p, h=1e-6):
    g = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        g.append((f(p + e) - f(p - e)) / (2 * h))
    return g


def test_derivative_relations():
    """Eq. mr4: D_z R_n^m = -R_{n-1}^m, D_{x+-iy} R_n^m = i R_{n-1}^{m+-1};
    D_z S_n^m = -S_{n+1}^m, D_{x+-iy} S_n^m = i S_{n+1}^{m+-1}."""
    p = np.array([0.3, 0.8, -0.45])
    for n in range(0, 7):
        for m in range(-n, n + 1):
            gx, gy, gz = _grad(lambda q: basis.R_nm(n, m, q), p)
            scale = 1.0 + abs(basis.R_nm(max(n - 1, 0), m, p))
            assert abs(gz - (-basis.R_nm(n - 1, m, p) if n > 0 else 0)) < 1e-8 * scale
            assert abs(gx + 1j * gy - (1j * basis.R_nm(n - 1, m + 1, p) if n > 0 else 0)) < 1e-8 * scale
            assert abs(gx - 1j * gy - (1j * basis.R_nm(n - 1, m - 1, p) if n > 0 else 0)) < 1e-8 * scale
            gx, gy, gz = _grad(lambda q: basis.S_nm(n, m, q), p)
            scale = 1.0 + abs(basis.S_nm(n + 1, m, p))
            assert abs(gz - (-basis.S_nm(n + 1, m, p))) < 1e-7 * scale
            assert abs(gx + 1j * gy - 1j * basis.S_nm(n + 1, m + 1, p)) < 1e-7 * scale
            assert abs(gx - 1j * gy - 1j * basis.S_nm(n + 1, m - 1, p)) < 1e-7 * scale


def test_Dr_eigenvalues():
    """Eq. dr1: r d/dr R_n^m = n R_n^m and r d/dr S_n^m = -(n+1) S_n^m."""
    p = np.array([0.5, -0.2, 0.9])
    h = 1e-6
    for n in range(6):
        for m in range(-n, n + 1):
            for fn, lam in ((basis.R_nm, n), (basis.S_nm, -(n + 1))):
                d = (fn(n, m, p * (1 + h)) - fn(n, m, p * (1 - h))) / (2 * h)
                assert abs(d - lam * fn(n, m, p)) < 1e-7 * (1 + abs(fn(n, m, p)))
