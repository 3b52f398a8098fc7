"""Variable truncation number (lhv_set_level_p) against the oracle with the same
per-level p: FP64 within 1e-10, FP32 and TF32x3 within 1e-6 (relative L2 of v, s),
and the exported expansions of each level against the oracle's."""
import numpy as np
import pytest

import workloads
from oracle import fmm as ofmm
from tests.gpu_util import dev, host3, rel, to_complex

pytestmark = pytest.mark.gpu


def _run(x, w, p, leaf, a, prec, sched):
    from paper_1201_5430_gb300 import LHV
    ctx = LHV(p=p, leaf_max=leaf, core_a=a, precision=prec)
    ctx.set_level_p(sched)
    dt = "fp64" if prec == "fp64" else "fp32"
    v4, s4 = ctx.evaluate_velocity_stretching(dev(x, dt), dev(w, dt))
    return ctx, host3(v4), host3(s4)


def _coeffs(ctx, ref, what, lev, basis):
    p = ref.level_p[lev]
    got = ctx.export(what, lev).cpu().numpy().reshape(-1, 2 * p * p)
    want = (ref.multipole if what == "multipole" else ref.local)[lev]
    worst = 0.0
    for b in range(got.shape[0]):
        phi, chi = to_complex(got[b], p, ref.tree.h(lev), basis)
        for g, wv in ((phi, want[b][0]), (chi, want[b][1])):
            worst = max(worst, float(np.abs(g - wv).max() / (np.abs(wv).max() + 1e-300)))
    return worst


@pytest.mark.parametrize("sched", [[0, 0, 4, 10], [0, 0, 10, 4], [0, 0, 7, 9]])
def test_fp64_level_p_parity(sched):
    x, w = workloads.cube(700, 7)
    ref = ofmm.fmm(x, w, 8, leaf_max=6, a=0.0, level_p=sched)
    ctx, v, s = _run(x, w, 8, 6, 0.0, "fp64", sched)
    st = ctx.stats()
    assert st["leaf_level"] == ref.tree.L == 3
    assert st["level_p"][2:] == sched[2:]
    assert rel(v, ref.v) < 1e-10 and rel(s, ref.s) < 1e-10, (rel(v, ref.v), rel(s, ref.s))
    assert _coeffs(ctx, ref, "multipole", 3, "S") < 1e-12    # P2M at p[3]
    assert _coeffs(ctx, ref, "multipole", 2, "S") < 1e-11    # M2M p[3] -> p[2] + Eq. drt11
    assert _coeffs(ctx, ref, "local", 2, "R") < 1e-11        # M2L at p[2] + Eq. drt10
    assert _coeffs(ctx, ref, "local", 3, "R") < 1e-11        # L2L p[2] -> p[3] + M2L at p[3]


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_fp32_ring_level_p_parity(prec):
    x, w = workloads.ring(12000, 1)
    a = workloads.RING_CORE_A
    sched = [0, 0, 8, 12, 16, 12, 10, 8]
    ref = ofmm.fmm(x, w, 12, leaf_max=64, a=a, level_p=sched)
    ctx, v, s = _run(x, w, 12, 64, a, prec, sched)
    L = ref.tree.L
    assert ctx.stats()["level_p"][2:] == ref.level_p[2:L + 1]
    ev, es = rel(v, ref.v), rel(s, ref.s)
    print(f"{prec} ring level p {ref.level_p}: rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < 1e-6 and es < 1e-6, (ev, es)


def test_reset_and_uniform_schedule_match_config_p():
    """A schedule equal to p at every level, and the reset, give the uniform result."""
    x, w = workloads.cube(3000, 2)
    from paper_1201_5430_gb300 import LHV
    ctx = LHV(p=8, leaf_max=16, core_a=0.01, precision="fp64")
    x4, w4 = dev(x, "fp64"), dev(w, "fp64")
    v0, s0 = ctx.evaluate_velocity_stretching(x4, w4)
    v0, s0 = host3(v0), host3(s0)
    ctx.set_level_p([8] * 10)
    v1, s1 = ctx.evaluate_velocity_stretching(x4, w4)
    assert rel(host3(v1), v0) < 1e-14 and rel(host3(s1), s0) < 1e-14
    ctx.set_level_p([0, 0, 6, 6, 6])
    v2, _ = ctx.evaluate_velocity_stretching(x4, w4)
    assert rel(host3(v2), v0) > 1e-9
    ctx.set_level_p(None)
    v3, s3 = ctx.evaluate_velocity_stretching(x4, w4)
    assert rel(host3(v3), v0) < 1e-14 and rel(host3(s3), s0) < 1e-14


def test_rejects_out_of_range():
    from paper_1201_5430_gb300 import LHV, LHVError
    ctx = LHV(p=8, leaf_max=16)
    for bad in ([0, 0, 25], [-1]):
        with pytest.raises(LHVError):
            ctx.set_level_p(bad)
