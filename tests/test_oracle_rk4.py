"""Pins of the RK4 step (Eq. s1.1 integrated at a constant step)."""
import numpy as np

from oracle import direct, rk4


def test_constant_rate_is_exact():
    x = np.array([[0.1, 0.2, 0.3], [1.0, -1.0, 0.5]])
    w = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 1.0]])
    vel = np.array([[0.5, -0.25, 2.0], [1.0, 1.0, 1.0]])
    xn, wn = rk4.rk4_step(x, w, 0.1, lambda xx, ww: (vel, np.zeros_like(ww)))
    np.testing.assert_allclose(xn, x + 0.1 * vel, rtol=1e-15)
    np.testing.assert_allclose(wn, w)


def test_fourth_order_convergence():
    """Two interacting smoothed elements: the one-step error scales as dt^5."""
    x0 = np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.05]])
    w0 = 0.02 * np.array([[0.2, -0.4, 1.0], [-0.7, 0.5, 0.3]])

    def rate(x, w):
        v, u, s = direct.direct(x, w, 0.1)
        return v, s

    def run(dt, steps):
        x, w = x0.copy(), w0.copy()
        for _ in range(steps):
            x, w = rk4.rk4_step(x, w, dt, rate)
        return x, w

    ref = run(0.0025, 32)
    errs = []
    for dt, steps in ((0.04, 2), (0.02, 4)):
        x, w = run(dt, steps)
        errs.append(np.abs(np.concatenate([x - ref[0], w - ref[1]])).max())
    ratio = errs[0] / errs[1]
    assert 12.0 < ratio < 20.0, (errs, ratio)
