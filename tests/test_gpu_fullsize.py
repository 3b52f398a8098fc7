"""The two colliding offset rings (2,097,152 elements, p = 16) under TF32x3 at full
size: the near field of sampled targets against the oracle's sum over the same
colleague leaves, and v against the oracle's direct sum at sampled targets."""
import numpy as np
import pytest

import workloads
from oracle import direct
from oracle import tree as T
from oracle.direct import pair_terms
from tests.gpu_util import dev, host3, rel

pytestmark = pytest.mark.gpu


def test_offset_rings_full_size_sampled():
    from paper_1201_5430_gb300 import LHV
    x, w, spec = workloads.make("offset_rings_2097152")
    a, p = spec["a"], spec["p"]
    tr = T.build_tree(x, leaf_max=spec["leaf_max"], a=a, eps=spec["eps"])
    near = LHV(p=p, leaf_max=spec["leaf_max"], core_a=a, eps=spec["eps"], precision="tf32x3", terms="near")
    vn, sn = near.evaluate_velocity_stretching(dev(x, "fp32"), dev(w, "fp32"))
    vn, sn = host3(vn), host3(sn)
    assert near.stats()["leaf_level"] == tr.L
    rng = np.random.default_rng(5)
    sample = rng.choice(x.shape[0], 100, replace=False)
    inv = np.empty_like(tr.perm)
    inv[tr.perm] = np.arange(x.shape[0])
    lv = tr.levels[tr.L]
    leaf_of = np.searchsorted(lv["begin"], inv[sample], side="right") - 1
    xs64, ws64 = x.astype(np.float64), w.astype(np.float64)
    for k, i in enumerate(sample):
        b = leaf_of[k]
        src = np.concatenate([tr.perm[lv["begin"][c]:lv["end"][c]] for c in lv["colleagues"][b]])
        src = src[src != i]
        vv, uu = pair_terms(xs64[i] - xs64[src], ws64[src], a)
        v_ref = vv.sum(axis=0)
        s_ref = ws64[i] @ uu.sum(axis=0)
        assert np.linalg.norm(vn[i] - v_ref) <= 2e-6 * np.linalg.norm(v_ref) + 1e-9
        assert np.linalg.norm(sn[i] - s_ref) <= 2e-5 * np.linalg.norm(s_ref) + 1e-9
    full = LHV(p=p, leaf_max=spec["leaf_max"], core_a=a, eps=spec["eps"], precision="tf32x3")
    v, s = full.evaluate_velocity_stretching(dev(x, "fp32"), dev(w, "fp32"))
    v, s = host3(v), host3(s)
    idx = sample[:24]
    v0, _, s0 = direct.direct_at(x, w, a, idx, chunk=4)
    ev, es = rel(v[idx], v0), rel(s[idx], s0)
    print(f"offset rings 2,097,152 p=16 TF32x3 vs direct sum: v {ev:.2e} s {es:.2e}")
    assert ev < 5e-6 and es < 1e-3
