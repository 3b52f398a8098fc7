"""Pins of the oracle's selector network: bfloat16 rounding, the analytic
backward pass against finite differences, one Adam step in closed form."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_round_closed_form_values():
    one = 1.0
    assert mlp.bf16_round([one])[0] == 1.0
    assert mlp.bf16_round([1 + 2.0 ** -8])[0] == 1.0                  # halfway: ties to the even mantissa
    assert mlp.bf16_round([1 + 3 * 2.0 ** -8])[0] == 1 + 2.0 ** -6     # halfway: rounds up to even
    assert mlp.bf16_round([1 + 2.0 ** -8 + 2.0 ** -20])[0] == 1 + 2.0 ** -7
    assert mlp.bf16_round([-3.0])[0] == -3.0


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.random.default_rng(0).normal(size=4096).astype(np.float32) * 10.0 ** np.random.default_rng(1).uniform(
        -8, 8, 4096).astype(np.float32)
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(a), want)


def _batch(rng, rows=40):
    x = rng.normal(size=(rows, 12))
    yp = rng.integers(-1, mlp.N_P, rows)
    yl = rng.integers(-1, mlp.N_LEAF, rows)
    return x, yp, yl


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    w, b = mlp.init(3)
    w = w.astype(np.float64)
    b = rng.normal(size=b.shape) * 0.1
    x, yp, yl = _batch(rng)
    ident = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
    loss, gw, gb = mlp.loss_and_grad(x, yp, yl, w, b, rnd=ident)
    assert np.isfinite(loss)
    h = 1e-6
    for k in rng.choice(w.size, 60, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (mlp.loss_and_grad(x, yp, yl, wp, b, rnd=ident)[0] - mlp.loss_and_grad(x, yp, yl, wm, b, rnd=ident)[0]) / (2 * h)
        assert abs(fd - gw[k]) <= 1e-6 * max(1.0, abs(gw[k])) + 1e-8, (k, fd, gw[k])
    for k in range(b.size):
        bp, bm = b.copy(), b.copy()
        bp[k] += h
        bm[k] -= h
        fd = (mlp.loss_and_grad(x, yp, yl, w, bp, rnd=ident)[0] - mlp.loss_and_grad(x, yp, yl, w, bm, rnd=ident)[0]) / (2 * h)
        assert abs(fd - gb[k]) <= 1e-6 * max(1.0, abs(gb[k])) + 1e-8, (k, fd, gb[k])


def test_loss_is_mean_cross_entropy_of_uniform_scores():
    """All-zero weights: every softmax is uniform, the loss is log 17 + log 4."""
    x, yp, yl = _batch(np.random.default_rng(5))
    yp[0], yl[0] = 3, 1
    w = np.zeros(mlp.n_weights())
    b = np.zeros(mlp.n_biases())
    loss, gw, gb = mlp.loss_and_grad(x, yp, yl, w, b)
    assert abs(loss - (np.log(17) + np.log(4))) < 1e-12
    assert np.all(gw == 0.0)  # no signal reaches the weights through zero activations


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    mlp.adam(theta, g, m, v, 1, 0.01)
    # bias-corrected m = g and v = g^2 after one step: theta -= lr g / (|g| + eps)
    np.testing.assert_allclose(theta, [1.0 - 0.01 * 0.3 / (0.3 + 1e-8), -2.0 + 0.01 * 4 / (4 + 1e-8),
                                       0.5 - 0.01 * 1e-3 / (1e-3 + 1e-8)], rtol=1e-14)
