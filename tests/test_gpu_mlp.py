"""Selector network kernels (lhv_mlp_*) against the FP64 oracle of oracle/mlp.py:
forward logits, loss and gradient, and the Adam step."""
import numpy as np
import pytest
import torch

from oracle import mlp

pytestmark = pytest.mark.gpu


def _params(seed):
    rng = np.random.default_rng(seed)
    w, b = mlp.init(seed)
    b = (rng.normal(size=b.shape) * 0.1).astype(np.float32)
    return w, b


def _dev(w, b):
    W = torch.from_numpy(w).cuda().to(torch.bfloat16)
    return W, torch.from_numpy(b).cuda()


def _batch(rows, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(rows, 12)).astype(np.float32)
    yp = rng.integers(-1, mlp.N_P, rows).astype(np.int32)
    yl = rng.integers(-1, mlp.N_LEAF, rows).astype(np.int32)
    return x, yp, yl


@pytest.mark.parametrize("rows", [1, 64, 1000, 20000])
def test_forward_matches_oracle(rows):
    from paper_1201_5430_gb300.api import mlp_forward
    w, b = _params(1)
    x, _, _ = _batch(rows, 2)
    W, B = _dev(w, b)
    z = mlp_forward(torch.from_numpy(x).cuda(), W, B).cpu().numpy()
    want = mlp.forward(x, w, b)
    assert np.abs(z - want).max() <= 1e-5 * (np.abs(want).max() + 1.0)


@pytest.mark.parametrize("rows", [64, 777, 20000])
def test_gradient_matches_oracle(rows):
    from paper_1201_5430_gb300.api import mlp_loss_grad
    w, b = _params(3)
    x, yp, yl = _batch(rows, 4)
    W, B = _dev(w, b)
    loss, gW, gb = mlp_loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(yp).cuda(), torch.from_numpy(yl).cuda(),
                                 W, B)
    l0, gw0, gb0 = mlp.loss_and_grad(x, yp, yl, w, b)
    assert abs(float(loss) - l0) <= 1e-5 * abs(l0)
    gw, gbb = gW.cpu().numpy(), gb.cpu().numpy()
    assert np.linalg.norm(gw - gw0) <= 1e-4 * np.linalg.norm(gw0), np.linalg.norm(gw - gw0) / np.linalg.norm(gw0)
    assert np.linalg.norm(gbb - gb0) <= 1e-4 * np.linalg.norm(gb0)


def test_adam_step_matches_oracle():
    from paper_1201_5430_gb300.api import mlp_adam
    rng = np.random.default_rng(7)
    w, b = _params(5)
    gw = rng.normal(size=w.shape).astype(np.float32)
    gb = rng.normal(size=b.shape).astype(np.float32)
    mw, vw = (rng.normal(size=w.shape) * 0.01).astype(np.float32), (rng.random(w.shape) * 0.01).astype(np.float32)
    mb, vb = np.zeros_like(b), np.zeros_like(b)
    cuda = lambda a: torch.from_numpy(a.copy()).cuda()  # noqa: E731
    W32, Gw, Mw, Vw, B, Gb, Mb, Vb = map(cuda, (w, gw, mw, vw, b, gb, mb, vb))
    W = W32.to(torch.bfloat16)
    mlp_adam(W32, W, Gw, Mw, Vw, B, Gb, Mb, Vb, 3, 1e-3)
    w64, mw64, vw64 = w.astype(np.float64), mw.astype(np.float64), vw.astype(np.float64)
    mlp.adam(w64, gw.astype(np.float64), mw64, vw64, 3, 1e-3)
    np.testing.assert_allclose(W32.cpu().numpy(), w64, rtol=1e-6, atol=1e-7)
    # FP32 rounding of 0.9 m + 0.1 g: absolute, on the scale of 0.1 |g| ~ 0.1
    np.testing.assert_allclose(Mw.cpu().numpy(), mw64, rtol=1e-6, atol=1e-7)
    assert np.array_equal(W.float().cpu().numpy(), mlp.bf16_round(W32.cpu().numpy()))


def test_training_lowers_the_loss():
    """A few hundred Adam steps of the GPU kernels fit a separable toy labelling."""
    from paper_1201_5430_gb300.api import mlp_adam, mlp_loss_grad
    rng = np.random.default_rng(11)
    x = rng.normal(size=(4096, 12)).astype(np.float32)
    yp = np.clip((x[:, 0] * 4 + 8).astype(np.int32), 0, 16)
    yl = (x[:, 1] > 0).astype(np.int32) + 2 * (x[:, 2] > 0).astype(np.int32)
    w, b = mlp.init(0)
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    X, YP, YL = cuda(x), cuda(yp), cuda(yl)
    W32, B = cuda(w), cuda(b)
    W = W32.to(torch.bfloat16)
    Mw, Vw, Mb, Vb = (torch.zeros_like(W32), torch.zeros_like(W32), torch.zeros_like(B), torch.zeros_like(B))
    first = None
    for t in range(1, 301):
        loss, gW, gb = mlp_loss_grad(X, YP, YL, W, B)
        if first is None:
            first = float(loss)
        mlp_adam(W32, W, gW, Mw, Vw, B, gb, Mb, Vb, t, 3e-3)
    last = float(mlp_loss_grad(X, YP, YL, W, B)[0])
    assert last < 0.35 * first, (first, last)
