"""Pins of the oracle's variable truncation number (one p per octree level).

Translations between levels of different p are the square maps of Eq. mr3
restricted to n' < p_out, n < p_in; each result is truncated to p_out before
its conversion (Eqs. drt10, drt11), as in the uniform case."""
import numpy as np

import workloads
from oracle import direct, expansions, operators
from oracle.fmm import fmm
from oracle.tree import build_tree
from tests.lh_util import potential, real_coeffs


def test_resize_pads_and_truncates(rng):
    c = real_coeffs(6, rng)
    big = operators.resize(c, 9)
    assert big.shape == (9, 17)
    np.testing.assert_array_equal(operators.resize(big, 6), c)
    assert np.all(big[6:] == 0)
    small = operators.resize(c, 4)
    for n in range(4):
        for m in range(-n, n + 1):
            assert operators.get(small, n, m) == operators.get(c, n, m)


def test_RR_to_more_terms_is_exact(rng):
    """A local expansion with 6 terms is a polynomial of degree 5: its (R|R)
    translate into 9 terms reproduces it exactly (Eq. mr3)."""
    c = real_coeffs(6, rng)
    t = np.array([0.17, -0.22, 0.09])
    out = operators.resize(operators.translate("RR", operators.resize(c, 9), t), 9)
    r = rng.normal(size=(10, 3)) * 0.3
    np.testing.assert_allclose(potential(out, r, "R"), potential(c, r + t, "R"), rtol=1e-12, atol=1e-13)
    assert np.abs(out[6:]).max() == 0.0    # degree cannot grow under (R|R)


def test_SS_between_truncations_keeps_the_exact_degrees(rng):
    """(S|S) is lower triangular in n, and Eq. drt11 reads chi at degrees <= n:
    a multipole of p_in terms moved to a centre with p_out terms and converted
    equals the direct P2M about that centre in every degree < min(p_in, p_out)."""
    x = rng.uniform(-0.12, 0.12, (6, 3))
    w = rng.normal(size=(6, 3))
    t = np.array([0.25, -0.25, 0.25])
    for p_in, p_out in ((6, 10), (10, 6)):
        phi0, chi0 = expansions.p2m_method2(x, w, np.zeros(3), p_in)
        pm = max(p_in, p_out)
        ph = operators.resize(operators.translate("SS", operators.resize(phi0, pm), t), p_out)
        ch = operators.resize(operators.translate("SS", operators.resize(chi0, pm), t), p_out)
        pt, ct = operators.convert_S(ph, ch, t)
        phi1, chi1 = expansions.p2m_method2(x, w, t, p_out)
        k = min(p_in, p_out)
        scale = np.abs(phi1).max()
        np.testing.assert_allclose(pt[:k], phi1[:k], rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(ct[1:k], chi1[1:k], rtol=0, atol=1e-12 * scale)   # chi_0^0 is free (Eq. dr3)
        if p_out > p_in:
            high = np.abs(phi1[p_in:]).max()   # the moments of degree >= p_in the input lacks
            assert np.abs(pt[p_in:] - phi1[p_in:]).max() > 1e-4 * high


def test_fmm_with_level_p_lies_between_the_uniform_runs():
    """Against the direct sum (O1): a schedule mixing p = 4 and p = 10 is less
    accurate than p = 10 everywhere and more accurate than p = 4 everywhere; the
    schedule with 10 at every far-field level reproduces p = 10 exactly."""
    x, w = workloads.cube(700, 7)
    tree = build_tree(x, 6, 0.0, 1e-6)
    assert tree.L == 3
    v_ref, _, s_ref = direct.direct(x.astype(np.float64), w.astype(np.float64), 0.0)

    def err(r):
        return (np.linalg.norm(r.v - v_ref) / np.linalg.norm(v_ref),
                np.linalg.norm(r.s - s_ref) / np.linalg.norm(s_ref))

    r4 = fmm(x, w, 4, leaf_max=6, tree=tree)
    r10 = fmm(x, w, 10, leaf_max=6, tree=tree)
    e4, e10 = err(r4), err(r10)
    for sched in ([0, 0, 4, 10], [0, 0, 10, 4]):
        r = fmm(x, w, 8, leaf_max=6, tree=tree, level_p=sched)
        assert r.level_p == [8, 8] + sched[2:]
        e = err(r)
        for k in range(2):
            assert e10[k] < e[k] < e4[k], (sched, e, e4, e10)
    same = fmm(x, w, 8, leaf_max=6, tree=tree, level_p=[0, 0, 10, 10])
    np.testing.assert_array_equal(same.v, r10.v)
    np.testing.assert_array_equal(same.s, r10.s)
