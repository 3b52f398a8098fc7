"""lhv_direct_sampled (FP64 direct sums at sampled targets) against the oracle's
direct sum O1, element by element."""
import numpy as np
import pytest
import torch

import workloads
from oracle import direct
from tests.gpu_util import dev, rel

pytestmark = pytest.mark.gpu


def _ctx(a, prec="fp32"):
    from paper_1201_5430_gb300 import LHV
    return LHV(p=4, leaf_max=64, core_a=a, precision=prec)


def _with_duplicates(n, seed):
    x, w = workloads.cube(n, seed)
    x = x.copy()
    x[1] = x[0]          # coincident distinct elements: r = 0, j != i
    x[7] = x[5]
    return x, w


@pytest.mark.parametrize("a", [0.0, 0.01, 0.2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_matches_oracle_direct_sum(a, prec):
    x, w = _with_duplicates(3001, 4)
    if a == 0.0:
        x, w = workloads.cube(3001, 4)  # the singular kernel has no value at r = 0
    rng = np.random.default_rng(0)
    idx = np.concatenate([[0, 1, 5, 7], rng.choice(np.arange(8, 3001), 157, replace=False)]).astype(np.int32)
    ctx = _ctx(a, prec)
    v, s = ctx.direct_sampled(dev(x, prec), dev(w, prec), torch.from_numpy(idx).cuda())
    v0, _, s0 = direct.direct_at(x, w, a, idx)
    v, s = v[:, :3].cpu().numpy(), s[:, :3].cpu().numpy()
    assert rel(v, v0) < 1e-12 and rel(s, s0) < 1e-12, (rel(v, v0), rel(s, s0))
    for k in range(idx.shape[0]):
        assert np.linalg.norm(v[k] - v0[k]) <= 1e-11 * np.linalg.norm(v0[k]) + 1e-300


def test_full_size_ring_sample():
    x, w, spec = workloads.make("ring_262144")
    rng = np.random.default_rng(1)
    idx = rng.choice(x.shape[0], 1000, replace=False).astype(np.int32)
    ctx = _ctx(spec["a"])
    v, s = ctx.direct_sampled(dev(x, "fp32"), dev(w, "fp32"), torch.from_numpy(idx).cuda())
    v0, _, s0 = direct.direct_at(x, w, spec["a"], idx[:12], chunk=2)
    v, s = v[:12, :3].cpu().numpy(), s[:12, :3].cpu().numpy()
    assert rel(v, v0) < 1e-12 and rel(s, s0) < 1e-11, (rel(v, v0), rel(s, s0))


def test_rejects_bad_index():
    from paper_1201_5430_gb300 import LHVError
    x, w = workloads.cube(100, 0)
    ctx = _ctx(0.01)
    with pytest.raises(LHVError):
        ctx.direct_sampled(dev(x, "fp32"), dev(w, "fp32"), torch.tensor([3, 100], dtype=torch.int32).cuda())
    v, s = ctx.direct_sampled(dev(x, "fp32"), dev(w, "fp32"), torch.tensor([3, 99], dtype=torch.int32).cuda())
    v0, _, s0 = direct.direct_at(x, w, 0.01, [3, 99])
    assert rel(v[:, :3].cpu().numpy(), v0) < 1e-12
