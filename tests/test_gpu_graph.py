"""Whole RK4 steps as one CUDA graph (lhv_set_graph): replays equal the uncaptured steps
(same kernels, captured layout) for one system and for a batch, the guard sends a step
whose tree no longer fits the captured layout back to the uncaptured path, and a
non-finite input is still reported."""
import numpy as np
import pytest

import workloads
from tests.gpu_util import dev, host3, rel

pytestmark = pytest.mark.gpu


def _pair(p=12, prec="tf32x3", a=workloads.RING_CORE_A, leaf=64, max_level=0):
    import torch
    from paper_1201_5430_gb300 import LHV
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = LHV(p=p, leaf_max=leaf, core_a=a, eps=1e-6, precision=prec, max_level=max_level)
        e = LHV(p=p, leaf_max=leaf, core_a=a, eps=1e-6, precision=prec, max_level=max_level)
    g.set_graph(True)
    return s, g, e


def _steps(s, ctx, x, w, k, dt, offsets=None):
    import torch
    out = []
    with torch.cuda.stream(s):
        x4, w4 = dev(x, "fp32"), dev(w, "fp32")
        for _ in range(k):
            if offsets is None:
                ctx.step(x4, w4, dt)
            else:
                ctx.step_batched(offsets, x4, w4, dt)
            out.append((host3(x4), host3(w4)))
    s.synchronize()
    return out


def _close(a, b, x0, w0):
    """The changes of x and w over the steps agree to 2e-6 (the far field's atomic additions
    run in another order), above the FP32 resolution of the states themselves (a last-bit
    difference in x = x0 + dt v is all a rounding difference in v can leave)."""
    for (xg, wg), (xe, we) in zip(a, b):
        for g, e, o in ((xg, xe, x0), (wg, we, w0)):
            ulp = 4.0 * np.linalg.norm(np.spacing(np.abs(e).astype(np.float32)).astype(np.float64))
            assert np.linalg.norm(g - e) <= 2e-6 * np.linalg.norm(e - o) + ulp, (np.linalg.norm(g - e), ulp)


def test_graph_replays_equal_uncaptured_steps():
    x, w = workloads.ring(20000, 1)
    s, g, e = _pair()
    a = _steps(s, g, x, w, 4, 1e-3)
    b = _steps(s, e, x, w, 4, 1e-3)
    _close(a, b, x.astype(np.float64), w.astype(np.float64))
    st = g.stats()["graph"]
    assert st["captures"] == 1 and st["replays"] == 3 and st["fallbacks"] == 0, st
    assert st["kernels"] > 50


def test_graph_batched_systems():
    systems = workloads.blob_systems(5, 9, n_lo=3000, n_hi=20000)
    x = np.concatenate([q[0] for q in systems])
    w = np.concatenate([q[1] for q in systems])
    off = [0] + list(np.cumsum([q[0].shape[0] for q in systems]))
    # the captured layout keeps one leaf level for the whole step; a level cap that every
    # stage's tree reaches makes the uncaptured steps use the same one (the same FMM)
    s, g, e = _pair(a=0.01, max_level=3)
    a = _steps(s, g, x, w, 3, 1e-3, off)
    b = _steps(s, e, x, w, 3, 1e-3, off)
    _close(a, b, x.astype(np.float64), w.astype(np.float64))
    st = g.stats()["graph"]
    assert st["captures"] == 1 and st["replays"] == 2, st


def test_guard_sends_a_changed_tree_back_uncaptured():
    """The same buffers refilled with a cube 64 times smaller: the core rule no longer
    allows the captured leaf level, so the replay writes nothing and the step runs
    uncaptured (equal to a context that never captured)."""
    import torch
    x, w = workloads.ring(12000, 2)
    s, g, e = _pair()
    with torch.cuda.stream(s):
        x4, w4 = dev(x, "fp32"), dev(w, "fp32")
        g.step(x4, w4, 1e-3)          # uncaptured + captured layout, then captured
        xs = (x / np.float32(64.0)).astype(np.float32)
        x4.copy_(dev(xs, "fp32"))
        w4.copy_(dev(w, "fp32"))
        g.step(x4, w4, 1e-3)          # replay: the guard fires, the step is redone
        xr, wr = host3(x4), host3(w4)
        x5, w5 = dev(xs, "fp32"), dev(w, "fp32")
        e.step(x5, w5, 1e-3)
        xe, we = host3(x5), host3(w5)
    st = g.stats()["graph"]
    assert st["fallbacks"] == 1, st
    _close([(xr, wr)], [(xe, we)], xs.astype(np.float64), w.astype(np.float64))


def test_nonfinite_input_under_a_graph():
    import torch
    from paper_1201_5430_gb300 import LHVError
    x, w = workloads.ring(8000, 4)
    s, g, _ = _pair()
    with torch.cuda.stream(s):
        x4, w4 = dev(x, "fp32"), dev(w, "fp32")
        g.step(x4, w4, 1e-3)
        w4[17, 1] = float("nan")
        before = host3(x4)
        with pytest.raises(LHVError) as ei:
            g.step(x4, w4, 1e-3)
        assert ei.value.status == -5
        assert np.array_equal(host3(x4), before)   # nothing written


def test_graph_needs_a_stream():
    from paper_1201_5430_gb300 import LHV, LHVError
    c = LHV(p=8, leaf_max=32, core_a=0.01)
    if c.stream.cuda_stream == 0:
        with pytest.raises(LHVError) as ei:
            c.set_graph(True)
        assert ei.value.status == -6
    assert c.lib.lhv_set_graph(c.h, 3) == -1
