"""lhv_morton_sort_noalloc (fixed file-scope scratch, no device allocation)
gives the same sorted Morton keys and permutation as lhv_build_tree followed by
lhv_export, on two calls in a row.  Named to be collected last, so that it also
runs after every other test has used the library; it passes alone too."""

import numpy as np
import pytest

import workloads
from oracle import tree as T
from tests.gpu_util import dev


def _tree_keys(x4):
    from paper_1201_5430_gb300 import LHV
    ctx = LHV(p=4, leaf_max=64)
    ctx.build_tree(x4)
    keys = ctx.export("keys").clone()
    perm = ctx.export("perm").clone()
    ctx.close()
    return keys, perm


def _noalloc(x4, w4=None):
    import torch
    from paper_1201_5430_gb300.api import morton_sort_noalloc
    n = x4.shape[0]
    keys = torch.empty(n, dtype=torch.int64, device=x4.device)
    perm = torch.empty(n, dtype=torch.int32, device=x4.device)
    morton_sort_noalloc(x4, keys, perm, w4)
    return keys, perm


def test_rejects_oversized_input_before_any_device_work():
    from paper_1201_5430_gb300 import _lib
    lib = _lib.load()
    assert lib.lhv_morton_sort_noalloc(_lib.NOALLOC_MAX_N + 1, None, None, None, None, None) == -7
    assert lib.lhv_morton_sort_noalloc(-1, None, None, None, None, None) == -1
    assert lib.lhv_morton_sort_noalloc(0, None, None, None, None, None) == 0
    assert b"no-allocation" in lib.lhv_status_string(-7)


@pytest.mark.gpu
def test_matches_build_tree_on_two_calls_in_a_row():
    from paper_1201_5430_gb300 import _lib
    xr, wr = workloads.ring(200003, 1)
    xc, _ = workloads.cube(_lib.NOALLOC_MAX_N, 3)  # the maximum size
    for x, w in ((xr, wr), (xc, None), (xr, wr)):
        x4 = dev(x, "fp32")
        w4 = dev(w, "fp32") if w is not None else None
        k_ref, p_ref = _tree_keys(x4)
        for _ in range(2):
            k, p = _noalloc(x4, w4)
            assert bool((k == k_ref).all()) and bool((p == p_ref).all())


@pytest.mark.gpu
def test_matches_oracle_keys_on_a_ragged_size():
    x, _ = workloads.cube(5003, 0)
    k, p = _noalloc(dev(x, "fp32"))
    tr = T.build_tree(x, leaf_max=64)
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint64), tr.keys)
    np.testing.assert_array_equal(p.cpu().numpy(), tr.perm)


@pytest.mark.gpu
def test_non_finite_input_is_reported_and_the_next_call_is_clean():
    from paper_1201_5430_gb300 import LHVError
    x, w = workloads.cube(4096, 0)
    w = w.copy()
    w[17, 1] = np.nan
    with pytest.raises(LHVError) as e:
        _noalloc(dev(x, "fp32"), dev(w, "fp32"))
    assert e.value.status == -5
    k, p = _noalloc(dev(x, "fp32"))
    k_ref, p_ref = _tree_keys(dev(x, "fp32"))
    assert bool((k == k_ref).all()) and bool((p == p_ref).all())
