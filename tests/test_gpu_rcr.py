"""M2L by rotation - coaxial translation - back rotation (Sec. 4.4, Eq. rcr1) on the GPU,
against the oracle's FMM with every translation by RCR (same p and tree): FP32 within
1e-6 relative L2 of v and s; the form against the fused-table form on the same inputs at
p = 12, 16, 20 (multi-level trees with full interaction lists); an RK4 step and a CUDA
graph replay of it equal to the uncaptured step; the unsupported configurations."""
import numpy as np
import pytest

import workloads
from oracle import rcr
from tests.gpu_util import dev, host3, rel

pytestmark = pytest.mark.gpu


def _ctx(p, leaf, a, prec="fp32", form="rcr", terms="all"):
    from paper_1201_5430_gb300 import LHV
    c = LHV(p=p, leaf_max=leaf, core_a=a, eps=1e-6, precision=prec, terms=terms)
    c.set_form(form)
    return c


@pytest.mark.parametrize("case", ["cube", "ring"])
def test_parity_with_oracle_rcr(case):
    if case == "cube":
        x, w = workloads.cube(2500, 41)
        a, p, leaf = 0.01, 8, 24
    else:
        x, w = workloads.ring(8000, 1)
        a, p, leaf = workloads.RING_CORE_A, 12, 64
    ref = rcr.fmm_rcr(x, w, p, leaf_max=leaf, a=a)
    c = _ctx(p, leaf, a)
    v4, s4 = c.evaluate_velocity_stretching(dev(x, "fp32"), dev(w, "fp32"))
    assert c.stats()["leaf_level"] == ref.tree.L >= 3
    ev, es = rel(host3(v4), ref.v), rel(host3(s4), ref.s)
    print(f"rcr {case} p={p}: rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < 1e-6 and es < 1e-6, (ev, es)


@pytest.mark.parametrize("p", [12, 16, 20])
def test_equals_fused_form(p):
    x, w = workloads.cube(60000, 7)
    out = {}
    for form in ("phi_chi", "rcr"):
        c = _ctx(p, 32, 0.002, "fp32", form, terms="far")
        v4, s4 = c.evaluate_velocity_stretching(dev(x, "fp32"), dev(w, "fp32"))
        out[form] = (host3(v4), host3(s4))
        assert c.stats()["leaf_level"] >= 4
    ev = rel(out["rcr"][0], out["phi_chi"][0])
    es = rel(out["rcr"][1], out["phi_chi"][1])
    print(f"rcr vs fused p={p}: far field rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < 2e-6 and es < 2e-6, (ev, es)


def test_step_and_graph_replay():
    import torch
    from paper_1201_5430_gb300 import LHV
    x, w = workloads.ring(6000, 3)
    a = workloads.RING_CORE_A
    res = []
    for form, graph in (("phi_chi", False), ("rcr", False), ("rcr", True)):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            c = LHV(p=12, leaf_max=64, core_a=a, eps=1e-6, precision="fp32")
            c.set_form(form)
            if graph:
                c.set_graph(True)
            x4, w4 = dev(x, "fp32"), dev(w, "fp32")
            for _ in range(3):
                c.step(x4, w4, 1e-3)
        s.synchronize()
        res.append((host3(x4), host3(w4)))
        if graph:
            assert c.stats()["graph"]["replays"] >= 1
    x0 = x.astype(np.float64)
    assert rel(res[1][0] - x0, res[0][0] - x0) < 1e-5
    assert rel(res[1][1], res[0][1]) < 1e-6
    assert rel(res[2][0] - x0, res[1][0] - x0) < 1e-5
    assert rel(res[2][1], res[1][1]) < 1e-6


def test_unsupported():
    from paper_1201_5430_gb300 import LHVError
    x, w = workloads.cube(3000, 2)
    for kw, lp in ((dict(p=8, prec="fp64"), None), (dict(p=22, prec="fp32"), None), (dict(p=8, prec="fp32"), [0, 0, 6, 8])):
        c = _ctx(kw["p"], 16, 0.01, kw["prec"])
        if lp:
            c.set_level_p(lp)
        with pytest.raises(LHVError) as e:
            c.evaluate_velocity_stretching(dev(x, kw["prec"]), dev(w, kw["prec"]))
        assert e.value.status == -6
