"""GPU tree construction is bit-exact with the oracle's (keys, permutation, boxes, colleagues)."""
import numpy as np
import pytest

import workloads
from oracle import tree as T
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def _check(x, leaf_max, a=0.0, eps=1e-6, max_level=0):
    from paper_1201_5430_gb300 import LHV
    ctx = LHV(p=4, leaf_max=leaf_max, core_a=a, eps=eps, max_level=max_level)
    ctx.build_tree(dev(x, "fp32"))
    tr = T.build_tree(x, leaf_max=leaf_max, a=a, eps=eps)
    st = ctx.stats()
    if max_level == 0:
        assert st["leaf_level"] == tr.L
    L = st["leaf_level"]
    keys = ctx.export("keys").cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(keys, tr.keys)
    np.testing.assert_array_equal(ctx.export("perm").cpu().numpy(), tr.perm)
    cube = ctx.export("cube").cpu().numpy()
    np.testing.assert_array_equal(cube[:3], tr.x0)
    assert cube[3] == tr.side
    if max_level:
        tr = T.build_tree(x, leaf_max=leaf_max, a=a, eps=eps, L_override=L)
    _boxes_match(ctx, tr, st, L)
    ctx.close()


def _boxes_match(ctx, tr, st, L):
    for lev in range(L + 1):
        d = tr.levels[lev]
        assert st["nbox"][lev] == d["keys"].shape[0]
        bk = ctx.export("box_keys", lev).cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(bk, d["keys"])
        rng = ctx.export("box_range", lev).cpu().numpy().reshape(-1, 2)
        np.testing.assert_array_equal(rng[:, 0], d["begin"])
        np.testing.assert_array_equal(rng[:, 1], d["end"])
        col = ctx.export("colleagues", lev).cpu().numpy().reshape(-1, 27)
        for i in range(col.shape[0]):
            assert sorted(c for c in col[i] if c >= 0) == d["colleagues"][i]


def test_repeated_trees_in_one_context():
    """After a context's first tree the sort orders the keys only down to five levels
    below the previous depth cap (core rule): leaf level, boxes and colleagues stay
    the oracle's, the keys are the oracle's keys of the permuted elements in prefix
    order; a cube that grows (the cap moves six levels deeper) falls back to the full sort."""
    from paper_1201_5430_gb300 import LHV
    x, _ = workloads.ring(20000, 1)
    a = workloads.RING_CORE_A
    ctx = LHV(p=4, leaf_max=64, core_a=a, eps=1e-6)
    for k, xs in enumerate((x, x + np.float32(1e-4), x * np.float32(64.0))):
        ctx.build_tree(dev(xs, "fp32"))
        tr = T.build_tree(xs, leaf_max=64, a=a, eps=1e-6)
        st = ctx.stats()
        L = st["leaf_level"]
        assert L == tr.L
        keys = ctx.export("keys").cpu().numpy().view(np.uint64)
        perm = ctx.export("perm").cpu().numpy()
        np.testing.assert_array_equal(np.sort(perm), np.arange(xs.shape[0]))
        okeys, _, _ = T.morton_keys(xs, T.core_unit(T.core_cutoff(a, 1e-6)))
        np.testing.assert_array_equal(keys, okeys[perm])
        if k != 1:  # a first tree, and the fallback, are fully sorted
            np.testing.assert_array_equal(perm, tr.perm)
        else:       # prefix order down to the previous cap + 5 > L
            pre = keys >> np.uint64(3 * (21 - (L + 1)))
            assert (pre[1:] >= pre[:-1]).all()
        _boxes_match(ctx, tr, st, L)
    ctx.close()
    # fewer elements than leaf_max + 1, first in a tiny region (cap 0), then spread over the
    # unit cube (cap 4): the fallback recomputes the leaf level from scratch, which stays 0
    xt, _ = workloads.cube(10, 5)
    ctx = LHV(p=4, leaf_max=64, core_a=a, eps=1e-6)
    for xs in (xt * np.float32(0.01), xt):
        ctx.build_tree(dev(xs, "fp32"))
        tr = T.build_tree(xs, leaf_max=64, a=a, eps=1e-6)
        st = ctx.stats()
        assert st["leaf_level"] == tr.L == 0
        _boxes_match(ctx, tr, st, 0)
    ctx.close()


@pytest.mark.parametrize("n,leaf", [(1, 64), (2, 1), (64, 64), (65, 64), (4096, 64), (5000, 7)])
def test_cube(n, leaf):
    x, _ = workloads.cube(n, 0)
    _check(x, leaf)


def test_ring_with_core_rule():
    x, _ = workloads.ring(20000, 1)
    _check(x, 64, a=workloads.RING_CORE_A, eps=1e-6)


def test_duplicates_and_ties():
    x = np.repeat(np.array([[0.1, 0.2, 0.3], [0.9, 0.1, 0.5], [0.4, 0.4, 0.4]], np.float32), 40, axis=0)
    x = x[np.random.default_rng(0).permutation(120)]
    _check(x, 8, max_level=5)


def test_full_size_ring_keys():
    x, _ = workloads.ring(262144, 1)
    from paper_1201_5430_gb300 import LHV
    ctx = LHV(p=12, leaf_max=64, core_a=workloads.RING_CORE_A, eps=1e-6)
    ctx.build_tree(dev(x, "fp32"))
    keys, x0, side = T.morton_keys(x, T.core_unit(T.core_cutoff(workloads.RING_CORE_A, 1e-6)))
    perm = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(ctx.export("keys").cpu().numpy().view(np.uint64), keys[perm])
    np.testing.assert_array_equal(ctx.export("perm").cpu().numpy(), perm)
    assert ctx.stats()["leaf_level"] == T.leaf_level(keys[perm], 64, side, workloads.RING_CORE_A, 1e-6)
