"""Pins of the oracle's Morton keys, octree and FMM lists."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import tree as T
from workloads import cube, ring


def _brute_key(x, x0, side):
    """Exact rational quantisation and a string-built bit interleave (x lowest)."""
    q = []
    for k in range(3):
        v = (Fraction(float(x[k])) - Fraction(float(x0[k]))) * (1 << 21) / Fraction(side)
        qi = int(v // 1)
        q.append(min(max(qi, 0), (1 << 21) - 1))
    bx, by, bz = (format(v, "021b") for v in q)
    return int("".join(bz[i] + by[i] + bx[i] for i in range(21)), 2)


def test_keys_match_brute_force(rng):
    x, _ = cube(300, 3)
    x = (x * np.float32(2.7) - np.float32(0.4)).astype(np.float32)
    keys, x0, side = T.morton_keys(x)
    assert side == 4.0
    for i in range(300):
        assert int(keys[i]) == _brute_key(x[i], x0, side)


def test_cube_side_is_power_of_two():
    for ext in (0.7, 1.0, 1.0000001, 3.9, 4.0, 4.01):
        x = np.array([[0.0, 0, 0], [ext, 0.1, 0.2]], dtype=np.float32)
        x0, side = T.cube(x)
        e = float(np.float32(ext))
        assert side >= e and side / 2 < e
        assert np.log2(side) == int(np.log2(side))
    x0, side = T.cube(np.zeros((3, 3), np.float32))
    assert side == 1.0


def test_core_unit_rounds_up_to_eight_bits():
    for rK in (0.0408, 0.01, 0.0625, 1.0, 3.3e-5, 0.123456789):
        u = T.core_unit(rK)
        assert rK <= u < rK * (1.0 + 1.0 / 128.0)
        mant, e = math.frexp(u)
        assert mant * 256.0 == int(mant * 256.0)  # an 8-bit mantissa
    assert T.core_unit(0.0) == 0.0


def test_cube_side_with_core_unit():
    u = T.core_unit(0.0408)
    for ext in (0.05, 0.7, 2.2, 2.75, 2.7500001, 10.0):
        x = np.array([[0.0, 0, 0], [ext, 0.01, 0.02]], dtype=np.float32)
        x0, side = T.cube(x, u)
        e = float(np.float32(ext))
        assert side >= e and side / 2 < e
        r = side / u
        assert r == 2.0 ** round(math.log2(r))  # a power of two times the unit


def test_leaf_side_lies_just_above_rK():
    """With the core rule binding (many elements per leaf), the leaf box side is the unit."""
    x, _ = ring(20000, 4)  # a thin ring: 4 elements per leaf needs a far deeper tree than L_K
    for a in (0.002, 0.005, 0.0063):
        rK = T.core_cutoff(a, 1e-6)
        tr = T.build_tree(x, leaf_max=4, a=a, eps=1e-6)
        h = tr.h(tr.L)
        assert rK <= h < (1.0 + 1.0 / 128.0) * rK, (a, rK, h)
        assert tr.h(tr.L + 1) < rK


def test_keys_match_brute_force_with_core_unit():
    """The keys are floor((x - x0) 2^21 / side) in FP64: equal to the exact rational value
    wherever it is not within FP64 rounding of an integer."""
    x, _ = cube(300, 5)
    x = (x * np.float32(2.2) - np.float32(1.1)).astype(np.float32)
    u = T.core_unit(T.core_cutoff(0.0063, 1e-6))
    keys, x0, side = T.morton_keys(x, u)
    assert side == u * 64.0
    near = 0
    for i in range(300):
        q = []
        for k in range(3):
            v = (Fraction(float(x[i, k])) - Fraction(float(x0[k]))) * (1 << 21) / Fraction(side)
            if abs(v - round(v)) < Fraction(1, 10 ** 6):
                near += 1
            q.append(min(max(math.floor(v), 0), (1 << 21) - 1))
        key = 0
        for b in range(21):
            for k in range(3):
                key |= ((q[k] >> b) & 1) << (3 * b + k)
        if near == 0:
            assert int(keys[i]) == key


def test_batch_side_is_the_largest_and_gives_leaves_at_the_unit():
    """A batch with a core: every system takes the largest own side; the core-capped leaf
    level of that side has leaves of the unit for every system."""
    a = 0.01
    u = T.core_unit(T.core_cutoff(a, 1e-6))
    xs = [(ring(3000, s)[0] * np.float32(f)).astype(np.float32) for s, f in ((1, 0.2), (2, 0.45), (3, 0.9))]
    own = [T.cube(x, u)[1] for x in xs]
    assert len(set(own)) > 1
    bs = T.batch_side(xs, a)
    assert bs == max(own)
    lev = round(math.log2(bs / u))
    assert bs / 2 ** lev == u
    for x in xs:
        tr = T.build_tree(x, leaf_max=1, a=a, side=bs)
        assert tr.side == bs and tr.L == lev and tr.h(tr.L) == u
    assert T.batch_side(xs, 0.0) is None and T.batch_side(xs[:1], a) is None


def test_sort_is_stable_permutation():
    x = np.array([[0.1, 0.1, 0.1]] * 5 + [[0.9, 0.9, 0.9]] * 3 + [[0.1, 0.1, 0.1]] * 2, dtype=np.float32)
    tr = T.build_tree(x, leaf_max=2)
    assert sorted(tr.perm.tolist()) == list(range(10))
    assert np.all(np.diff(tr.keys.astype(np.float64)) >= 0)
    assert tr.perm.tolist() == [0, 1, 2, 3, 4, 8, 9, 5, 6, 7]


def _check_structure(tr):
    for lev, d in enumerate(tr.levels):
        assert d["begin"][0] == 0 and d["end"][-1] == tr.n
        assert np.all(d["begin"][1:] == d["end"][:-1])
        for i, col in enumerate(d["colleagues"]):
            assert i in col and len(col) <= 27
            for j in col:
                assert i in d["colleagues"][j]
                assert np.abs(d["coords"][i] - d["coords"][j]).max() <= 1
        for i, il in enumerate(d["il"]):
            assert len(il) <= 189
            for j in il:
                assert i in d["il"][j]
                diff = np.abs(d["coords"][i] - d["coords"][j]).max()
                assert 2 <= diff <= 3
        if lev < tr.L:
            for i, ch in enumerate(d["children"]):
                assert ch and d["begin"][i] == tr.levels[lev + 1]["begin"][ch[0]]
                assert d["end"][i] == tr.levels[lev + 1]["end"][ch[-1]]


def _covered_once(tr):
    """Every (target, source != target) pair is handled exactly once: by the
    near field (colleague leaves) or by one M2L at the first separated level."""
    L = tr.L
    box_of = []
    for d in tr.levels:
        b = np.empty(tr.n, dtype=np.int64)
        for i in range(d["begin"].shape[0]):
            b[d["begin"][i]:d["end"][i]] = i
        box_of.append(b)
    col = [set(c) for c in tr.levels[L]["colleagues"]]
    ils = [[set(c) for c in d["il"]] for d in tr.levels]
    for i in range(tr.n):
        for j in range(tr.n):
            if i == j:
                continue
            count = int(box_of[L][j] in col[box_of[L][i]])
            for lev in range(2, L + 1):
                count += int(box_of[lev][j] in ils[lev][box_of[lev][i]])
            assert count == 1, (i, j, count)


@pytest.mark.parametrize("n,leaf", [(1, 4), (2, 1), (64, 64), (65, 64), (200, 3), (257, 8)])
def test_tree_structure_and_partition(n, leaf):
    x, _ = cube(n, 7)
    tr = T.build_tree(x, leaf_max=leaf)
    _check_structure(tr)
    _covered_once(tr)
    counts = [e - b for b, e in zip(tr.levels[-1]["begin"], tr.levels[-1]["end"])]
    assert max(counts) <= leaf or tr.L == T.KEY_BITS
    if tr.L > 0:
        prev = [e - b for b, e in zip(tr.levels[-2]["begin"], tr.levels[-2]["end"])]
        assert max(prev) > leaf


def test_ring_tree_partition():
    x, _ = ring(600, 1)
    tr = T.build_tree(x, leaf_max=8)
    assert tr.L >= 3
    _check_structure(tr)
    _covered_once(tr)


def test_core_rule_limits_depth():
    """L_K: the leaf boxes are no smaller than r_K, where 1 - K = eps/10 (Eq. vem1)."""
    mp = pytest.importorskip("mpmath")
    a, eps = 0.01, 1e-6
    rK = T.core_cutoff(a, eps)
    x = mp.mpf(rK / a)
    one_minus_K = mp.erfc(x / mp.sqrt(2)) + mp.sqrt(2 / mp.pi) * x * mp.exp(-x * x / 2)
    assert float(one_minus_K) == pytest.approx(eps / 10, rel=1e-9)
    xs, _ = cube(20000, 0)
    tr = T.build_tree(xs, leaf_max=4, a=a, eps=eps)
    assert tr.h(tr.L) >= rK and tr.h(tr.L + 1) < rK
    tr0 = T.build_tree(xs, leaf_max=4, a=0.0)
    assert tr0.L > tr.L
