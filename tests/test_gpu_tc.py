"""Tensor-core (tcgen05, TF32) path: descriptor self-test and split-precision parity."""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import fmm as ofmm
from tests.gpu_util import dev, host3, rel

pytestmark = pytest.mark.gpu


def _tf32(a):
    """Round FP32 to TF32 (10 mantissa bits), to nearest, ties away from zero."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("N,K", [(16, 32), (144, 64), (256, 96)])
def test_tc_selftest_matches_reference(N, K):
    import torch
    from paper_1201_5430_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(N + K)
    X = rng.normal(size=(128, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32)
    Xd, Bd = torch.from_numpy(X).cuda(), torch.from_numpy(B).cuda()
    Dd = torch.zeros(128, N, device="cuda")
    torch.cuda.synchronize()
    st = lib.lhv_tc_selftest(ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(Bd.data_ptr()),
                             ctypes.c_void_p(Dd.data_ptr()), N, K)
    assert st == 0
    want = _tf32(X).astype(np.float64) @ _tf32(B).astype(np.float64).T
    got = Dd.cpu().numpy()
    scale = np.abs(_tf32(X)).astype(np.float64) @ np.abs(_tf32(B)).astype(np.float64).T
    assert np.max(np.abs(got - want) / scale) < 1e-6


@pytest.mark.parametrize("case", ["cube", "ring"])
def test_tf32x3_parity(case):
    from paper_1201_5430_gb300 import LHV
    if case == "cube":
        x, w = workloads.cube(6000, 5)
        a, leaf = 0.01, 32
    else:
        x, w = workloads.ring(12000, 1)
        a, leaf = workloads.RING_CORE_A, 64
    p = 12
    ref = ofmm.fmm(x, w, p, leaf_max=leaf, a=a)
    ctx = LHV(p=p, leaf_max=leaf, core_a=a, precision="tf32x3")
    v4, s4 = ctx.evaluate_velocity_stretching(dev(x, "fp32"), dev(w, "fp32"))
    ctx.stats()  # raises if a tensor-core wait timed out
    ev, es = rel(host3(v4), ref.v), rel(host3(s4), ref.s)
    print(f"tf32x3 {case} p=12: rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < 1e-6 and es < 1e-6, (ev, es)
