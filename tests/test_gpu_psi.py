"""The complex form Psi = phi + i chi (Sec. 4.2, Eq. chf1) on the GPU, against the
oracle's one-complex-FMM (O2 in the Psi form) at the same p and tree: FP64 within 1e-10,
FP32 and TF32x3 within 1e-6 relative L2 of v and s; the exported Psi coefficients of a
level against the oracle's; an RK4 step equal to the two-potential form's."""
import numpy as np
import pytest

import workloads
from oracle import complex_psi as cp
from tests.gpu_util import dev, host3, rel, to_complex

pytestmark = pytest.mark.gpu


def _ctx(p, leaf, a, prec):
    from paper_1201_5430_gb300 import LHV
    c = LHV(p=p, leaf_max=leaf, core_a=a, eps=1e-6, precision=prec)
    c.set_form("psi")
    return c


def _psi_rows_to_phichi(rows, p):
    """Inverse of the layout in include/lhv.h (lhv_set_form), per row: Psi -> (phi, chi)."""
    P = p * p
    out = np.array(rows, dtype=np.float64, copy=True)
    for n in range(p):
        for m in range(1, n + 1):
            re, im = n * n + 2 * m - 1, n * n + 2 * m
            s = -1.0 if m % 2 else 1.0
            x0, x1, x2, x3 = rows[:, re], rows[:, im], rows[:, P + re], rows[:, P + im]
            out[:, re] = 0.5 * (x0 + s * x2)
            out[:, im] = 0.5 * (x1 - s * x3)
            out[:, P + re] = 0.5 * (x1 + s * x3)
            out[:, P + im] = 0.5 * (s * x2 - x0)
    return out


def test_fp64_parity_and_exported_psi():
    x, w = workloads.cube(2500, 41)
    a, p, leaf = 0.01, 8, 24
    ref = cp.fmm_psi(x, w, p, leaf_max=leaf, a=a)
    c = _ctx(p, leaf, a, "fp64")
    v4, s4 = c.evaluate_velocity_stretching(dev(x, "fp64"), dev(w, "fp64"))
    assert c.stats()["leaf_level"] == ref.tree.L >= 3
    ev, es = rel(host3(v4), ref.v), rel(host3(s4), ref.s)
    assert ev < 1e-10 and es < 1e-10, (ev, es)
    for what, lev, basis, tab in (("multipole", 2, "S", ref.multipole), ("local", 2, "R", ref.local),
                                  ("local", ref.tree.L, "R", ref.local)):
        rows = c.export(what, lev).cpu().numpy().reshape(-1, 2 * p * p)
        pc = _psi_rows_to_phichi(rows, p)
        worst = 0.0
        for b in range(rows.shape[0]):
            phi, chi = to_complex(pc[b], p, ref.tree.h(lev), basis)
            want = tab[lev][b]
            got = cp.psi_of(phi, chi)
            worst = max(worst, float(np.abs(got - want).max() / (np.abs(want).max() + 1e-300)))
        assert worst < 1e-11, (what, lev, worst)


@pytest.mark.parametrize("prec,p", [("fp32", 12), ("tf32x3", 12), ("tf32x3", 16)])
def test_fp32_ring_parity(prec, p):
    x, w = workloads.ring(8000, 1)
    a = workloads.RING_CORE_A
    ref = cp.fmm_psi(x, w, p, leaf_max=64, a=a)
    c = _ctx(p, 64, a, prec)
    v4, s4 = c.evaluate_velocity_stretching(dev(x, "fp32"), dev(w, "fp32"))
    st = c.stats()
    assert st["leaf_level"] == ref.tree.L
    ev, es = rel(host3(v4), ref.v), rel(host3(s4), ref.s)
    print(f"psi {prec} ring p={p}: rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < 1e-6 and es < 1e-6, (ev, es)


def test_step_equals_two_potential_form():
    import torch
    from paper_1201_5430_gb300 import LHV
    x, w = workloads.ring(6000, 3)
    a = workloads.RING_CORE_A
    res = []
    for form in ("phi_chi", "psi"):
        c = LHV(p=12, leaf_max=64, core_a=a, eps=1e-6, precision="tf32x3")
        c.set_form(form)
        x4, w4 = dev(x, "fp32"), dev(w, "fp32")
        c.step(x4, w4, 1e-3)
        torch.cuda.synchronize()
        res.append((host3(x4), host3(w4)))
    x0 = x.astype(np.float64)
    assert rel(res[1][0] - x0, res[0][0] - x0) < 1e-5   # the displacement over the step
    assert rel(res[1][1], res[0][1]) < 1e-6


def test_form_errors():
    from paper_1201_5430_gb300 import LHV, LHVError
    c = LHV(p=8, leaf_max=16, core_a=0.01)
    with pytest.raises(KeyError):
        c.set_form("quaternion")
    assert c.lib.lhv_set_form(c.h, 7) == -1
    c.set_form("psi")
    c.set_level_p([0, 0, 6, 8])
    x, w = workloads.cube(3000, 2)
    with pytest.raises(LHVError) as e:
        c.evaluate_velocity_stretching(dev(x, "fp32"), dev(w, "fp32"))
    assert e.value.status == -6
