"""Pins of the plain FP64 Lamb-Helmholtz FMM (O2) against the direct sum (O1)."""
import numpy as np
import pytest

from oracle import direct, fmm
from oracle import tree as T
from workloads import cube, ring


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_error_falls_with_p():
    """Spectral convergence in p (Sec. 5.1); p = 12 reaches the paper's ~1e-5 range."""
    x, w = cube(1200, 11)
    a = 0.01
    v0, u0, s0 = direct.direct(x, w, a)
    tr = T.build_tree(x, leaf_max=16, a=a)
    assert tr.L == 4  # the core-aligned cube (side 1.906) puts 16 or fewer per box at level 4
    ev, es = [], []
    for p in (3, 6, 9, 12):
        r = fmm.fmm(x, w, p, tree=tr, a=a)
        ev.append(_rel(r.v, v0))
        es.append(_rel(r.s, s0))
    assert all(ev[i + 1] < 0.5 * ev[i] for i in range(3)), ev
    assert all(es[i + 1] < 0.5 * es[i] for i in range(3)), es
    assert ev[-1] < 3e-5 and es[-1] < 1e-4, (ev, es)


def test_shallow_tree_is_exact():
    """With fewer than 3 levels no box is well separated: O2 is the direct sum."""
    x, w = cube(150, 5)
    x = (x * np.float32(0.9)).astype(np.float32)  # a tight cube (side 0.953 = 8 r_q), level 1 splits evenly
    r = fmm.fmm(x, w, 6, leaf_max=64, a=0.02)
    assert r.tree.L < 2
    v0, u0, s0 = direct.direct(x, w, 0.02)
    np.testing.assert_allclose(r.v, v0, rtol=1e-12, atol=1e-12 * np.abs(v0).max())
    np.testing.assert_allclose(r.s, s0, rtol=1e-12, atol=1e-12 * np.abs(s0).max())


def test_far_field_divergence_free():
    """Every R_n^m is harmonic, so trace(grad v) of the far field vanishes (Eq. 3)."""
    x, w = cube(900, 2)
    r = fmm.fmm(x, w, 8, leaf_max=8, a=0.0, near=False)
    assert np.abs(np.trace(r.grad, axis1=1, axis2=2)).max() < 1e-10 * np.abs(r.grad).max()


def test_core_rule_is_needed():
    """Smoothing with r_K > h at the leaf level: the FMM with the L_K rule switched
    off keeps an error set by 1 - K, not by p; with the rule it converges."""
    x, w = cube(1500, 9)
    a = 0.04
    v0, u0, s0 = direct.direct(x, w, a)
    good = fmm.fmm(x, w, 16, leaf_max=8, a=a)
    bad = fmm.fmm(x, w, 16, tree=T.build_tree(x, leaf_max=8, a=a, L_override=good.tree.L + 1), a=a)
    eg, eb = _rel(good.s, s0), _rel(bad.s, s0)
    assert eg < 1e-4 and eb > 10 * eg, (eg, eb)


def test_ring_accuracy():
    """A thin ring (Sec. 5.3 geometry) at p = 12 against the direct sum.  The
    stretching of a ring is a small residual of cancelling terms, so its relative
    error is larger than that of v (about 3e-4 here, falling ~10x per 3 orders)."""
    x, w = ring(3000, 1)
    a = 0.02
    r = fmm.fmm(x, w, 12, leaf_max=16, a=a)
    assert r.tree.L >= 3
    v0, u0, s0 = direct.direct(x, w, a)
    assert _rel(r.v, v0) < 2e-5 and _rel(r.s, s0) < 1e-3
