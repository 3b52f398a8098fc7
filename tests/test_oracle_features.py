"""Pins of the oracle's selector features on inputs whose values are known in
closed form: a full grid (one element per leaf cell) and strengths that are all
equal or cancel in pairs."""
import math

import numpy as np

from oracle.features import level_features
from oracle.tree import build_tree


def _grid(L):
    m = 2 ** L
    g = (np.arange(m) + 0.5) / m
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    return x.astype(np.float32)


def test_full_grid_counts_in_closed_form():
    L = 3
    x = _grid(L)
    w = np.tile([[0.0, 0.0, 1.0]], (x.shape[0], 1))
    tree = build_tree(x, leaf_max=1)
    assert tree.L == L
    f = level_features(tree, w, 1e-6, 0.0)
    assert f.shape == (L - 1, 12)
    for r, lev in enumerate(range(2, L + 1)):
        m, mp = 2 ** lev, 2 ** (lev - 1)
        col = ((3 * m - 2) / m) ** 3                       # neighbours per axis: 3 inside, 2 at a face
        il = 8 * ((3 * mp - 2) / mp) ** 3 - col            # children of the parent's colleagues minus colleagues
        assert abs(f[r, 8] - col / 27) < 1e-12
        assert abs(f[r, 7] - il / 189) < 1e-12
        assert abs(f[r, 3] - 1.0) < 1e-12                  # every box has 8 children: log2 8 / 3
        assert abs(f[r, 2] - 3 * lev / 20) < 1e-12
        assert abs(f[r, 4] - 3 * (L - lev) / 20) < 1e-12   # 8^(L - l) elements per box
        assert f[r, 9] == 0.0                              # equal strengths never cancel
        assert f[r, 0] == lev / 10 and f[r, 1] == (L - lev) / 10
    assert f[0, 5] == 0.6 and f[0, 6] == -3.0 and abs(f[0, 10] - 9 / 24) < 1e-12


def test_cancelling_strengths_and_core_feature():
    """Pairs of opposite strengths in every leaf cancel at every level: the
    moment feature takes its floor; a = h_2 gives log2(1) = 0."""
    x = np.repeat(_grid(2), 2, axis=0)
    w = np.tile([[1.0, 2.0, -1.0], [-1.0, -2.0, 1.0]], (x.shape[0] // 2, 1))
    tree = build_tree(x, leaf_max=2)
    assert tree.L == 2
    f = level_features(tree, w, 1e-3, tree.side / 4, prec=0.5)
    assert f[0, 9] == -3.0 and f[0, 6] == 0.0 and f[0, 11] == 0.5
    assert abs(f[0, 5] - 0.3) < 1e-15
    assert abs(f[0, 4] - math.log2(2) / 20) < 1e-15
