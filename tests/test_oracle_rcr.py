"""Pins of the RCR oracle (Sec. 4.4, Eq. rcr1): rotations of coefficients against the rotated
functions, their inverse, the coaxial conversions of Eq. rcr1 against the general ones of
Eqs. drt10 / drt11 at t = t i_z, RCR translation + conversion against the dense one for all
three kinds, and the whole FMM against O2."""
import numpy as np
import pytest

import workloads
from oracle import fmm as ofmm
from oracle import rcr
from oracle.expansions import eval_R, eval_S
from oracle.operators import convert_R, convert_S, flatten, translation_matrix, unflatten
from tests.lh_util import real_coeffs


def _rand_rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


@pytest.mark.parametrize("basis", ["R", "S"])
def test_rotation_reproduces_the_rotated_function(rng, basis):
    p = 12
    Q = _rand_rotation(rng)
    c = real_coeffs(p, rng)
    blocks = rcr.rotation_blocks(p, Q, basis)
    c2 = rcr.rotate(c, blocks)
    ev = eval_R if basis == "R" else eval_S
    r = rng.normal(size=(10, 3))
    if basis == "S":
        r *= 2.0 / np.linalg.norm(r, axis=1)[:, None]
    want = ev(c, r @ Q.T)
    got = ev(c2, r)
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))
    back = rcr.rotate(c2, rcr.rotation_blocks(p, Q.T, basis))
    assert np.max(np.abs(back - c)) < 1e-11 * np.max(np.abs(c))


def test_frame_takes_z_to_t(rng):
    for _ in range(5):
        t = rng.normal(size=3)
        Q = rcr.frame_of(t)
        assert np.allclose(Q @ np.array([0, 0, 1.0]), t / np.linalg.norm(t), atol=1e-15)
        assert np.allclose(Q.T @ Q, np.eye(3), atol=1e-15) and np.linalg.det(Q) > 0


def test_coaxial_conversions_of_eq_rcr1(rng):
    p, d = 9, 0.37
    phi, chi = real_coeffs(p, rng), real_coeffs(p, rng)
    for mine, general in ((rcr.coax_convert_R, convert_R), (rcr.coax_convert_S, convert_S)):
        a = mine(phi, chi, d)
        b = general(phi, chi, np.array([0.0, 0.0, d]))
        for k in range(2):
            assert np.max(np.abs(a[k] - b[k])) < 1e-13 * np.max(np.abs(b[k]))


@pytest.mark.parametrize("kind", ["SS", "SR", "RR"])
def test_rcr_equals_the_dense_translation_and_conversion(rng, kind):
    p = 10
    phi, chi = real_coeffs(p, rng), real_coeffs(p, rng)
    t = rng.normal(size=3)
    t *= (2.5 if kind == "SR" else 0.4) / np.linalg.norm(t)
    T = translation_matrix(kind, t, p)
    ph, cc = unflatten(T @ flatten(phi), p), unflatten(T @ flatten(chi), p)
    want = (convert_S if kind == "SS" else convert_R)(ph, cc, t)
    got = rcr.translate_convert_rcr(kind, phi, chi, t)
    for k in range(2):
        assert np.max(np.abs(got[k] - want[k])) < 1e-10 * np.max(np.abs(want[k])), kind


def test_fmm_rcr_equals_o2():
    x, w = workloads.cube(1200, 51)
    ref = ofmm.fmm(x, w, 8, leaf_max=24, a=0.01)
    got = rcr.fmm_rcr(x, w, 8, leaf_max=24, a=0.01)
    assert ref.tree.L >= 3
    rel = lambda a_, b_: np.linalg.norm(a_ - b_) / np.linalg.norm(b_)
    assert rel(got.v, ref.v) < 1e-10 and rel(got.s, ref.s) < 1e-10, (rel(got.v, ref.v), rel(got.s, ref.s))
