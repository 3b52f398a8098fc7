"""Pins of the complex Psi = phi + i chi oracle (Sec. 4.2, Eq. chf1): the split back
into real potentials, complex linearity of the translations (one complex translation of
Psi is the two real ones), and the whole FMM equal to the two-potential FMM O2."""
import numpy as np
import pytest

import workloads
from oracle import complex_psi as cp
from oracle import fmm as ofmm
from oracle.expansions import eval_R, eval_S
from oracle.operators import flatten, translation_matrix, unflatten
from tests.lh_util import real_coeffs


def test_split_inverts_eq_chf1(rng):
    for p in (1, 4, 9):
        phi, chi = real_coeffs(p, rng), real_coeffs(p, rng)
        ph, ch = cp.split_psi(cp.psi_of(phi, chi))
        assert np.max(np.abs(ph - phi)) < 1e-15 and np.max(np.abs(ch - chi)) < 1e-15


def test_psi_is_the_complex_function(rng):
    """sum Psi_n^m F_n^m(r) = phi(r) + i chi(r) at points, for F = S and F = R."""
    p = 8
    phi, chi = real_coeffs(p, rng), real_coeffs(p, rng)
    psi = cp.psi_of(phi, chi)
    r = rng.normal(size=(10, 3))
    for ev in (eval_S, eval_R):
        a, b, c = ev(psi, r), ev(phi, r), ev(chi, r)
        assert np.max(np.abs(b.imag)) < 1e-12 and np.max(np.abs(c.imag)) < 1e-12  # real functions
        assert np.max(np.abs(a - (b.real + 1j * c.real))) < 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("kind", ["SS", "SR", "RR"])
def test_one_complex_translation_is_two_real_ones(rng, kind):
    p = 7
    phi, chi = real_coeffs(p, rng), real_coeffs(p, rng)
    t = np.array([2.1, -1.3, 0.7]) if kind == "SR" else np.array([0.2, -0.1, 0.15])
    T = translation_matrix(kind, t, p)
    tr = lambda c: unflatten(T @ flatten(c), p)
    got = tr(cp.psi_of(phi, chi))
    want = cp.psi_of(tr(phi), tr(chi))
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    # the translated pair is still a pair of real functions: the split recovers them
    ph, ch = cp.split_psi(got)
    assert np.max(np.abs(ph - tr(phi))) < 1e-12 * np.max(np.abs(want))
    assert np.max(np.abs(ch - tr(chi))) < 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("case", ["cube", "ring"])
def test_fmm_psi_equals_the_two_potential_fmm(case):
    if case == "cube":
        x, w = workloads.cube(1500, 31)
        a, leaf, p = 0.01, 24, 8
    else:
        x, w = workloads.ring(3000, 32)
        a, leaf, p = workloads.RING_CORE_A, 64, 10
    ref = ofmm.fmm(x, w, p, leaf_max=leaf, a=a)
    got = cp.fmm_psi(x, w, p, leaf_max=leaf, a=a)
    assert ref.tree.L >= 3
    rel = lambda a_, b_: np.linalg.norm(a_ - b_) / np.linalg.norm(b_)
    assert rel(got.v, ref.v) < 1e-12 and rel(got.s, ref.s) < 1e-12, (rel(got.v, ref.v), rel(got.s, ref.s))
