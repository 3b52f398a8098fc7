"""Pins of the scalar harmonic FMM oracle (the paper's phi, grad phi reference case,
Sec. 5.2) against closed forms, finite differences, brute force and convergence in p."""
import math

import numpy as np

import workloads
from oracle import scalar
from oracle.expansions import eval_S
from oracle.operators import translation_matrix, flatten, unflatten
from tests.lh_util import fd_grad


def test_direct_scalar_brute_force(rng):
    """O1s against a pure-Python double loop on 7 elements (two coincident, j != i by index)."""
    x = rng.random((7, 3)).astype(np.float32)
    x[3] = x[1]
    q = rng.standard_normal(7).astype(np.float32)
    phi, grad = scalar.direct_scalar(x, q)
    xd, qd = x.astype(np.float64), q.astype(np.float64)
    for i in range(7):
        ph, g = 0.0, [0.0, 0.0, 0.0]
        for j in range(7):
            if j == i:
                continue
            d = [xd[i][k] - xd[j][k] for k in range(3)]
            r = math.sqrt(sum(v * v for v in d))
            if r == 0.0:
                continue  # the singular kernel has no value there (coincident distinct elements)
            ph += qd[j] / r
            for k in range(3):
                g[k] -= qd[j] * d[k] / r ** 3
        assert abs(phi[i] - ph) <= 1e-13 * max(1.0, abs(ph))
        assert np.allclose(grad[i], g, rtol=1e-13, atol=1e-13)


def test_p2m_scalar_is_the_green_expansion(rng):
    """One charge: the S-expansion about the origin reproduces q / |r - x0| at |r| = 1
    (Eq. rsbf5) to 1e-12 at p = 30, and a sum of charges is the sum of their expansions."""
    x0 = rng.normal(size=(3, 3))
    x0 *= 0.3 / np.linalg.norm(x0, axis=1)[:, None]
    q = np.array([1.5, -0.7, 0.2])
    c = scalar.p2m_scalar(x0, q, np.zeros(3), 30)
    r = rng.normal(size=(20, 3))
    r /= np.linalg.norm(r, axis=1)[:, None]
    got = eval_S(c, r).real
    want = sum(q[k] / np.linalg.norm(r - x0[k], axis=1) for k in range(3))
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    # no imaginary part: the coefficients of a real function
    assert np.max(np.abs(eval_S(c, r).imag)) < 1e-13


def test_l2p_scalar_gradient_of_a_translated_charge(rng):
    """A far charge, expanded about c0 (Eq. rsbf5), translated to c1 by (S|R) (Eq. mr3):
    l2p_scalar gives q/|y - x0| and its gradient -q (y - x0)/|y - x0|^3 near c1, and the
    gradient also matches finite differences of the evaluated potential."""
    p = 24
    x0 = np.array([0.1, -0.05, 0.08])
    q = 0.9
    c0 = np.zeros(3)
    c1 = np.array([2.0, 1.0, -1.5])
    mp = scalar.p2m_scalar(x0[None], [q], c0, p)
    T = translation_matrix("SR", c1 - c0, p)
    loc = unflatten(T @ flatten(mp), p)
    y = c1 + 0.2 * rng.uniform(-1, 1, size=(12, 3))
    phi, grad = scalar.l2p_scalar(loc, y - c1)
    d = y - x0
    r = np.linalg.norm(d, axis=1)
    assert np.max(np.abs(phi - q / r)) < 1e-10 * np.max(q / r)
    want = -q * d / r[:, None] ** 3
    assert np.max(np.abs(grad - want)) < 1e-9 * np.max(np.abs(want))
    fd = fd_grad(lambda pts: scalar.l2p_scalar(loc, pts - c1)[0], y, 1e-3).real
    assert np.max(np.abs(grad - fd)) < 1e-8 * np.max(np.abs(want))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_fmm_scalar_converges_with_p():
    """O2s -> O1s: the error falls with p and is at the rounding level of the
    truncation at p = 16 (Sec. 5.1: spectral convergence)."""
    x, _ = workloads.cube(2000, 11)
    q = np.random.default_rng(12).standard_normal(2000).astype(np.float32)
    phi0, g0 = scalar.direct_scalar(x, q)
    errs = []
    for p in (4, 8, 12, 16):
        r = scalar.fmm_scalar(x, q, p, leaf_max=32)
        assert r.tree.L >= 3
        errs.append((_rel(r.phi, phi0), _rel(r.grad, g0)))
    for k in range(3):
        assert errs[k + 1][0] < 0.3 * errs[k][0] and errs[k + 1][1] < 0.3 * errs[k][1], errs
    assert errs[-1][0] < 1e-7 and errs[-1][1] < 1e-6, errs


def test_fmm_scalar_without_far_field_is_the_direct_sum():
    """A tree with no separated boxes (L < 2): the near field is every pair, exactly."""
    x, _ = workloads.cube(300, 13)
    q = np.random.default_rng(14).standard_normal(300).astype(np.float32)
    r = scalar.fmm_scalar(x, q, 8, leaf_max=400)
    assert r.tree.L < 2
    phi0, g0 = scalar.direct_scalar(x, q)
    assert _rel(r.phi, phi0) < 1e-14 and _rel(r.grad, g0) < 1e-14


def test_fmm_scalar_near_far_split_and_partition():
    """far + near = the whole, and the near part alone is the direct sum over the
    colleague leaves (each pair counted once in one of the two parts)."""
    x, _ = workloads.cube(1500, 15)
    q = np.random.default_rng(16).standard_normal(1500).astype(np.float32)
    r = scalar.fmm_scalar(x, q, 10, leaf_max=24)
    assert np.allclose(r.phi, r.phi_far + r.phi_near, rtol=0, atol=1e-12)
    tr = r.tree
    lv = tr.levels[tr.L]
    inv = np.empty_like(tr.perm)
    inv[tr.perm] = np.arange(x.shape[0])
    for i in (0, 77, 901):
        b = np.searchsorted(lv["begin"], inv[i], side="right") - 1
        src = np.concatenate([tr.perm[lv["begin"][c]:lv["end"][c]] for c in lv["colleagues"][b]])
        src = src[src != i]
        d = x[i].astype(np.float64) - x[src].astype(np.float64)
        want = (q[src].astype(np.float64) / np.linalg.norm(d, axis=1)).sum()
        assert abs(r.phi_near[i] - want) < 1e-12 * abs(want) + 1e-12
