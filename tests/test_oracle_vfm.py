"""Pins of the vortex filament oracle (Sec. 5.3, App. B): Eq. dis2 against the line integral
of Eq. dis1, the Gauss-Legendre S-expansion of Eqs. vf5-vf7 (exact for n < p, and not with one
point fewer), its far field against Eq. dis2, O2f -> O1f with p, exclusion of a node's own
segments, and the ring speed of Eq. dis6."""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from oracle import vfm
from tests.lh_util import lh_velocity


def _line_integral(y, x1, x2, gamma, nq=400):
    """Eq. dis1 (v = Gamma/4pi int dl x (y - x) / |y - x|^3) by a 400-point Gauss-Legendre rule
    on each of 8 sub-intervals."""
    xi, w = leggauss(nq)
    v = np.zeros(3)
    for k in range(8):
        a, b = k / 8.0, (k + 1) / 8.0
        t = 0.5 * (b - a) * xi + 0.5 * (a + b)
        pts = x1[None, :] + t[:, None] * (x2 - x1)[None, :]
        d = y[None, :] - pts
        r3 = np.linalg.norm(d, axis=1) ** 3
        integrand = np.cross(np.broadcast_to(x2 - x1, d.shape), d) / r3[:, None]
        v += 0.5 * (b - a) * (w[:, None] * integrand).sum(axis=0)
    return gamma / (4.0 * math.pi) * v


def test_closed_form_against_the_line_integral(rng):
    for _ in range(6):
        x1, x2 = rng.normal(size=3), rng.normal(size=3)
        y = rng.normal(size=3) * 2.0
        g = rng.normal()
        got = vfm.segment_velocity(y[None], x1[None], x2[None], [g])[0, 0]
        want = _line_integral(y, x1, x2, g)
        assert np.linalg.norm(got - want) < 1e-11 * np.linalg.norm(want)
    # on the segment's line, outside it: no velocity (r1 x r2 = 0)
    x1, x2 = np.zeros(3), np.array([1.0, 0.0, 0.0])
    assert np.all(vfm.segment_velocity(np.array([[2.5, 0.0, 0.0]]), x1[None], x2[None], [1.0]) == 0.0)


def test_quadrature_rule_of_eq_vf7(rng):
    p = 12
    x1, x2 = rng.normal(size=(3, 3)) * 0.05, rng.normal(size=(3, 3)) * 0.05
    g = rng.normal(size=3)
    c = rng.normal(size=3) * 0.02
    exact = vfm.p2m_segment(x1, x2, g, c, p, nq=40)
    got = vfm.p2m_segment(x1, x2, g, c, p)
    fewer = vfm.p2m_segment(x1, x2, g, c, p, nq=vfm.n_quad(p) - 1)
    for k in range(2):
        scale = np.abs(exact[k]).max()
        assert np.abs(got[k] - exact[k]).max() < 1e-14 * scale
    worst = max(np.abs(fewer[k][p - 1] - exact[k][p - 1]).max() / np.abs(exact[k][p - 1]).max() for k in range(2))
    assert worst > 1e-8, worst   # one point fewer misses the top degree


def test_segment_expansion_far_field(rng):
    """The S-expansion of a segment about its centre gives Eq. dis2 at distance 10 l (p = 20)."""
    x1, x2 = np.array([-0.05, 0.02, 0.0]), np.array([0.05, -0.01, 0.03])
    phi, chi = vfm.p2m_segment(x1[None], x2[None], [1.3], np.zeros(3), 20)
    y = rng.normal(size=(6, 3))
    y *= 1.2 / np.linalg.norm(y, axis=1)[:, None]
    got = lh_velocity(phi, chi, y, "S", h=1e-5).real
    want = vfm.segment_velocity(y, x1[None], x2[None], [1.3])[:, 0]
    assert np.abs(got - want).max() < 1e-8 * np.abs(want).max()


def _ring(n, radius=1.0, jitter=0.0, seed=0):
    rng = np.random.default_rng(seed)
    th = 2 * math.pi * np.arange(n) / n
    r = radius + jitter * rng.standard_normal(n)
    z = jitter * rng.standard_normal(n)
    return np.stack([r * np.cos(th), r * np.sin(th), z], axis=1).astype(np.float32)


def test_own_segments_are_excluded():
    """A closed triangle: each node gets only the opposite segment's velocity."""
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    g = np.array([1.0, 2.0, 3.0], np.float32)
    v = vfm.direct_filaments(x, g, [0, 3], [True])
    want0 = vfm.segment_velocity(x[:1].astype(np.float64), x[1:2].astype(np.float64), x[2:3].astype(np.float64),
                                 [2.0])[0, 0]
    assert np.allclose(v[0], want0, rtol=1e-14, atol=0)


def test_fmm_filaments_converge_with_p():
    x = np.concatenate([_ring(3000, jitter=0.002, seed=1), _ring(2000, radius=0.8, jitter=0.002, seed=2) +
                        np.float32([0, 0, 0.3])])
    g = np.concatenate([np.full(3000, 1.0), np.full(2000, -0.7)]).astype(np.float32)
    off, closed = [0, 3000, 5000], [True, True]
    v0 = vfm.direct_filaments(x, g, off, closed)
    errs = []
    for p in (6, 10, 14):
        r = vfm.fmm_filaments(x, g, off, closed, p, leaf_max=32)
        assert r.tree.L >= 3
        errs.append(np.linalg.norm(r.v - v0) / np.linalg.norm(v0))
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.2 * errs[1] and errs[2] < 5e-6, errs


def test_ring_speed_of_eq_dis6():
    """A closed ring of N segments moves along its axis with about Gamma/(4 pi R) ln(2N/pi)."""
    n = 4000
    x = _ring(n)
    v = vfm.direct_filaments(x, np.ones(n, np.float32), [0, n], [True])
    vz = v[:, 2].mean()
    want = 1.0 / (4.0 * math.pi) * math.log(2 * n / math.pi)
    assert np.abs(v[:, :2]).max() < 1e-3 * abs(vz)
    assert abs(vz - want) < 0.02 * want, (vz, want)
