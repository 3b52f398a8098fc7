"""Parity with the oracle O2 at the truncation numbers that reach eps = 1e-6 on the
ring workloads (Sec. 5.1: the error falls with p; Sec. 4.4: translations), element by
element, relative L2 of v and s below 1e-6, same p and same tree on both sides:

* plain FP32 at uniform p = 15 and p = 16 (the equal-accuracy arm of plain FP32);
* TF32x3 at uniform p = 16 (one 256-row N range per half of the 2p^2 outputs) and
  p = 20 (each half of the 800 outputs in a 256-row and a 144-row N range, so the
  tensor-core kernel walks four ranges per work item);
* TF32x3 under the per-level schedule (20, 20, 20, 16, 16, 16, 16) that the selector
  network picks on the leapfrogging ring pair, on a scaled-down pair of coaxial rings.
"""
import pytest

import workloads
from oracle import fmm as ofmm
from tests.gpu_util import dev, host3, rel

pytestmark = pytest.mark.gpu

N_RING = 8000
A = workloads.RING_CORE_A
TOL = 1e-6


@pytest.fixture(scope="module")
def ring8k():
    return workloads.ring(N_RING, 1)


_refs = {}


def _ref(x, w, p, level_p=None, key=None):
    k = key or p
    if k not in _refs:
        _refs[k] = ofmm.fmm(x, w, p, leaf_max=64, a=A, level_p=level_p)
    return _refs[k]


def _gpu(x, w, p, prec, level_p=None):
    from paper_1201_5430_gb300 import LHV
    ctx = LHV(p=p, leaf_max=64, core_a=A, eps=1e-6, precision=prec)
    if level_p is not None:
        ctx.set_level_p(level_p)
    v4, s4 = ctx.evaluate_velocity_stretching(dev(x, "fp32"), dev(w, "fp32"))
    st = ctx.stats()  # raises if a tensor-core wait timed out
    return st, host3(v4), host3(s4)


@pytest.mark.parametrize("p", [15, 16])
def test_fp32_parity_at_eps_p(ring8k, p):
    x, w = ring8k
    ref = _ref(x, w, p)
    st, v, s = _gpu(x, w, p, "fp32")
    assert st["leaf_level"] == ref.tree.L and ref.tree.L >= 3
    assert st["launch_shape"]["m2l_tensor_cores"] == 0
    ev, es = rel(v, ref.v), rel(s, ref.s)
    print(f"fp32 ring {N_RING} p={p}: rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < TOL and es < TOL, (ev, es)


@pytest.mark.parametrize("p", [16, 20])
def test_tf32x3_parity_at_eps_p(ring8k, p):
    """p = 20 runs the multi-range path of the tensor-core kernel (2 x (256 + 144) rows)."""
    x, w = ring8k
    ref = _ref(x, w, p)
    st, v, s = _gpu(x, w, p, "tf32x3")
    assert st["leaf_level"] == ref.tree.L and ref.tree.L >= 3
    assert st["launch_shape"]["m2l_tensor_cores"] == 1  # the products ran on the tensor cores
    assert st["level_p"][2:] == [p] * (ref.tree.L - 1)
    ev, es = rel(v, ref.v), rel(s, ref.s)
    print(f"tf32x3 ring {N_RING} p={p}: rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < TOL and es < TOL, (ev, es)


def test_tf32x3_learned_leapfrog_schedule():
    """The schedule the network chose on the leapfrogging pair, on two coaxial rings of
    4096 elements (z = 0 and 0.1, the same core and leaf rule): p = 20 on levels 0..2
    (the tensor-core multi-range path at level 2), p = 16 below."""
    x, w = workloads.ring_pair(4096, 6, "leapfrog")
    sched = [20, 20, 20, 16, 16, 16, 16]
    ref = ofmm.fmm(x, w, 12, leaf_max=64, a=A, level_p=sched)
    L = ref.tree.L
    assert L >= 4
    st, v, s = _gpu(x, w, 12, "tf32x3", level_p=sched)
    assert st["leaf_level"] == L
    assert st["level_p"][2:] == ref.level_p[2:L + 1]
    assert st["launch_shape"]["m2l_tensor_cores"] == 1
    ev, es = rel(v, ref.v), rel(s, ref.s)
    print(f"tf32x3 leapfrog pair 2x4096 schedule {ref.level_p[:L + 1]}: rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < TOL and es < TOL, (ev, es)
