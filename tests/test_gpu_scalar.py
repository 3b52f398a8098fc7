"""The scalar reference case (Sec. 5.2, phi and grad phi of monopoles) on the GPU against
the oracle's scalar FMM (O2s) at the same p and tree: FP64 within 1e-10, FP32 and TF32x3
within 1e-6 relative L2 of phi and of grad phi; the near and far parts separately; the
full result against the direct sum (O1s)."""
import numpy as np
import pytest

import workloads
from oracle import scalar
from tests.gpu_util import dev, rel

pytestmark = pytest.mark.gpu


def _run(x, q, p, leaf, prec, terms="all"):
    import torch
    from paper_1201_5430_gb300 import LHV
    ctx = LHV(p=p, leaf_max=leaf, core_a=0.0, precision=prec, terms=terms)
    dt = torch.float64 if prec == "fp64" else torch.float32
    pg = ctx.evaluate_potential_gradient(dev(x, "fp64" if prec == "fp64" else "fp32"),
                                         torch.from_numpy(np.asarray(q, np.float64)).to("cuda", dt))
    pg = pg.double().cpu().numpy()
    return ctx, pg[:, 3], pg[:, :3]


@pytest.fixture(scope="module")
def cube3k():
    x, _ = workloads.cube(3000, 21)
    q = workloads.charges(3000, 22)
    return x, q, scalar.fmm_scalar(x, q, 10, leaf_max=16)


def test_fp64_parity(cube3k):
    x, q, ref = cube3k
    ctx, phi, grad = _run(x, q, 10, 16, "fp64")
    assert ctx.stats()["leaf_level"] == ref.tree.L >= 3
    assert rel(phi, ref.phi) < 1e-10 and rel(grad, ref.grad) < 1e-10, (rel(phi, ref.phi), rel(grad, ref.grad))


@pytest.mark.parametrize("terms", ["near", "far"])
def test_fp64_terms_split(cube3k, terms):
    x, q, ref = cube3k
    _, phi, grad = _run(x, q, 10, 16, "fp64", terms=terms)
    wp = ref.phi_near if terms == "near" else ref.phi_far
    wg = ref.grad_near if terms == "near" else ref.grad_far
    assert rel(phi, wp) < 1e-10 and rel(grad, wg) < 1e-10


@pytest.mark.parametrize("prec,p", [("fp32", 12), ("tf32x3", 12), ("tf32x3", 16), ("fp32", 15)])
def test_fp32_parity(prec, p):
    """p = 12 and 16 run the M2L products on the tensor cores (p^2 a multiple of 16) under
    TF32x3; p = 15 on the CUDA cores."""
    x, _ = workloads.cube(6000, 23)
    q = workloads.charges(6000, 24)
    ref = scalar.fmm_scalar(x, q, p, leaf_max=32)
    ctx, phi, grad = _run(x, q, p, 32, prec)
    assert ctx.stats()["leaf_level"] == ref.tree.L
    ep, eg = rel(phi, ref.phi), rel(grad, ref.grad)
    print(f"scalar {prec} p={p}: rel L2 phi {ep:.2e} grad {eg:.2e}")
    assert ep < 1e-6 and eg < 1e-6, (ep, eg)


def test_sphere_surface_and_direct_sum():
    """Table 2's distribution: parity with O2s, and accuracy against the direct sum that
    falls with p (Sec. 5.1)."""
    x, _ = workloads.sphere(5000, 25)
    q = workloads.charges(5000, 26)
    phi0, g0 = scalar.direct_scalar(x, q)
    errs = []
    for p in (8, 12):
        ref = scalar.fmm_scalar(x, q, p, leaf_max=32)
        _, phi, grad = _run(x, q, p, 32, "fp32")
        assert rel(phi, ref.phi) < 1e-6 and rel(grad, ref.grad) < 1e-6
        errs.append((rel(phi, phi0), rel(grad, g0)))
    assert errs[1][0] < 0.2 * errs[0][0] and errs[1][1] < 0.2 * errs[0][1], errs


def test_coincident_elements_contribute_nothing():
    x, _ = workloads.cube(2001, 27)
    x = x.copy()
    x[5] = x[4]
    x[9:12] = x[8]
    q = workloads.charges(2001, 28)
    ref = scalar.fmm_scalar(x, q, 8, leaf_max=16)
    for prec, tol in (("fp32", 1e-6), ("fp64", 1e-10)):
        _, phi, grad = _run(x, q, 8, 16, prec)
        assert np.isfinite(phi).all() and np.isfinite(grad).all()
        assert rel(phi, ref.phi) < tol and rel(grad, ref.grad) < tol


def test_rejects_a_smoothed_context():
    import torch
    from paper_1201_5430_gb300 import LHV, LHVError
    ctx = LHV(p=8, leaf_max=16, core_a=0.01)
    x = dev(np.zeros((4, 3), np.float32), "fp32")
    with pytest.raises(LHVError) as e:
        ctx.evaluate_potential_gradient(x, torch.zeros(4, device="cuda"))
    assert e.value.status == -6
