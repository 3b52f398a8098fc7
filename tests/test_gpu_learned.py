"""What the trained selector network (paper_1201_5430_gb300/selector_weights.npz)
gains over the method without it, on workloads held out of its training set: the
262,144-element ring (seed 1) and a 262,144-element cube (seed 0).  Accuracy is
the relative L2 error of v against FP64 direct sums at 1000 sampled elements
(Sec. 5.1), the target eps = 1e-6 of the learned form."""
import time

import numpy as np
import pytest
import torch

import workloads
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu

EPS = 1e-6


def _case(name):
    if name == "ring":
        x, w = workloads.ring(262144, 1)
        return x, w, workloads.RING_CORE_A
    x, w = workloads.cube(262144, 0)
    return x, w, 0.01


def _err(v, v0, idx):
    return float(torch.linalg.norm(v[idx].double()[:, :3] - v0[:, :3]) / torch.linalg.norm(v0[:, :3]))


def _ms(ctx, x4, w4, reps=5):
    ctx.evaluate_velocity_stretching(x4, w4)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        t = time.perf_counter()
        ctx.evaluate_velocity_stretching(x4, w4)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t)
    return float(np.median(ts)) * 1e3


@pytest.fixture(scope="module")
def net():
    from paper_1201_5430_gb300 import selector
    W, b, meta = selector.load()
    assert meta["train_within1_p"] > 0.9
    return W, b


@pytest.mark.parametrize("name", ["ring", "cube"])
def test_network_meets_the_target_the_fixed_p_misses(net, name):
    """Without the network the context's fixed p = 12 misses eps = 1e-6 by a wide
    margin; with it every evaluation meets eps on the sampled direct sums, with
    no fallback."""
    from paper_1201_5430_gb300 import LHV
    x, w, a = _case(name)
    x4, w4 = dev(x, "fp32"), dev(w, "fp32")
    idx = torch.from_numpy(np.random.default_rng(0).choice(x.shape[0], 1000, replace=False).astype(np.int32)).cuda()
    v0, _ = LHV(p=4, leaf_max=64, core_a=a).direct_sampled(x4, w4, idx)
    fixed = LHV(p=12, leaf_max=64, core_a=a)
    v, _ = fixed.evaluate_velocity_stretching(x4, w4)
    e_fixed = _err(v, v0, idx.long())
    for prec in ("fp32", "tf32x3"):
        ctx = LHV(p=12, leaf_max=64, core_a=a, precision=prec)
        ctx.set_selector(*net, eps=EPS, check_every=1, check_samples=1000)
        v, _ = ctx.evaluate_velocity_stretching(x4, w4)
        st = ctx.stats()
        e = _err(v, v0, idx.long())
        print(f"{name} {prec}: fixed p=12 err {e_fixed:.2e}; learned p {st['level_p']} err {e:.2e}")
        assert st["selector"]["fallbacks"] == 0
        assert e <= EPS and 0 <= st["selector"]["err_v"] <= EPS  # this sample and the library's own
    assert e_fixed > 4 * EPS


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_network_against_the_best_uniform_p_at_equal_precision(net, prec):
    """The method without the network needs the fastest uniform p that reaches eps, found
    by trial evaluations against direct sums, in the same arithmetic as the learned form
    (so the tensor cores are credited to neither).  On the held-out cube the network's
    one-pass schedule is faster than that best uniform p in plain FP32; under TF32x3,
    where the uniform arm already runs its M2L on the tensor cores (p a multiple of 4),
    it is not slower by more than 10 % (a measured outcome, printed)."""
    from paper_1201_5430_gb300 import LHV
    x, w, a = _case("cube")
    x4, w4 = dev(x, "fp32"), dev(w, "fp32")
    idx = torch.from_numpy(np.random.default_rng(0).choice(x.shape[0], 1000, replace=False).astype(np.int32)).cuda()
    v0, _ = LHV(p=4, leaf_max=64, core_a=a).direct_sampled(x4, w4, idx)
    cands = []
    for p in range(14, 21):
        ctx = LHV(p=p, leaf_max=64, core_a=a, precision=prec)
        v, _ = ctx.evaluate_velocity_stretching(x4, w4)
        if _err(v, v0, idx.long()) <= EPS:
            cands.append((_ms(ctx, x4, w4), p))
            if prec == "fp32" or p % 4 == 0:
                break  # the next p costs more on the same pipes
    assert cands
    best = min(cands)
    ctx = LHV(p=12, leaf_max=64, core_a=a, precision=prec)
    ctx.set_selector(*net, eps=EPS, check_every=0)
    t_learned = _ms(ctx, x4, w4)
    print(f"cube {prec}: best uniform p {best[1]} {best[0]:.1f} ms; learned {ctx.stats()['level_p']} "
          f"{t_learned:.1f} ms ({best[0] / t_learned:.2f}x)")
    if prec == "fp32":
        assert t_learned < best[0]
    else:
        assert t_learned < 1.10 * best[0]
