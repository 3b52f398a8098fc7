"""The ordering argument behind the tree build's short sort, checked on the CPU.

After its first tree a context orders the Morton keys only by their prefix down
to a level S at least as deep as the deepest level its trees may have (L_cap,
from the core rule and the level cap).  The leaf level comes from a window rule
on the ordered keys: the deepest level at which keys leaf_max apart share a box.
Here that rule is restated in integers, and prefix order is compared with full
order: the leaf level capped at L_cap and the sequence of boxes of every level
down to S must be the same."""
import numpy as np
import pytest

import workloads
from oracle import tree as T

BITS = 21


def window_leaf_level(keys, leaf_max):
    """min(deepest shared level + 1, BITS) over windows of leaf_max + 1 keys (-1 + 1 if none)."""
    best = -1
    a, b = keys[:-leaf_max] if leaf_max else keys, keys[leaf_max:]
    for x in (a ^ b).tolist() if keys.shape[0] > leaf_max else []:
        lvl = BITS if x == 0 else BITS - (x.bit_length() - 1 + 3) // 3
        best = max(best, lvl)
    return min(best + 1, BITS)


def _cases():
    xr, _ = workloads.ring(4000, 1)
    xc, _ = workloads.cube(3000, 2)
    xd = np.repeat(workloads.cube(40, 3)[0], 25, axis=0)  # many equal keys
    return {"ring": xr, "cube": xc, "duplicates": xd}


@pytest.mark.parametrize("name", ["ring", "cube", "duplicates"])
@pytest.mark.parametrize("leaf_max", [8, 64])
def test_prefix_order_keeps_capped_leaf_level_and_boxes(name, leaf_max):
    x = _cases()[name]
    keys, _, _ = T.morton_keys(x)
    full = keys[np.argsort(keys, kind="stable")]
    L_full = window_leaf_level(full, leaf_max)
    for L_cap in range(0, 9):
        for S in (L_cap, L_cap + 1, L_cap + 3):
            if S > BITS:
                continue
            pref = keys[np.argsort(keys >> np.uint64(3 * (BITS - S)), kind="stable")]
            assert min(window_leaf_level(pref, leaf_max), L_cap) == min(L_full, L_cap), (L_cap, S)
            for lev in range(S + 1):
                sh = np.uint64(3 * (BITS - lev))
                np.testing.assert_array_equal(pref >> sh, full >> sh)


def test_a_prefix_shorter_than_the_cap_can_change_the_leaf_level():
    """The bound S >= L_cap matters: ordering by a shorter prefix does change the
    window rule's answer here, which is why a tree whose cap grew is re-sorted."""
    x = _cases()["cube"]
    keys, _, _ = T.morton_keys(x)
    full = keys[np.argsort(keys, kind="stable")]
    L_cap, S = 6, 2
    pref = keys[np.argsort(keys >> np.uint64(3 * (BITS - S)), kind="stable")]
    assert min(window_leaf_level(pref, 8), L_cap) != min(window_leaf_level(full, 8), L_cap)
