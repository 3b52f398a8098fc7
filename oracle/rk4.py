"""Classical fourth-order Runge-Kutta step for Eq. s1.1, FP64.

Test infrastructure (see ``oracle/__init__``).

The state is y = (x, w); its rate is F(y) = (v, s) with v the velocity at each
element and s = w . grad v the stretching (Eq. s1.1).  The paper integrates
with RK4 at a constant step (Sec. 5.3); the classical tableau is used:
  k1 = F(y), k2 = F(y + dt/2 k1), k3 = F(y + dt/2 k2), k4 = F(y + dt k3),
  y <- y + dt/6 (k1 + 2 k2 + 2 k3 + k4).
"""
import numpy as np

__all__ = ["rk4_step"]


def rk4_step(x, w, dt, rate):
    """One step.  ``rate(x, w) -> (v, s)``; x, w are (N, 3) arrays."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    v1, s1 = rate(x, w)
    v2, s2 = rate(x + 0.5 * dt * v1, w + 0.5 * dt * s1)
    v3, s3 = rate(x + 0.5 * dt * v2, w + 0.5 * dt * s2)
    v4, s4 = rate(x + dt * v3, w + dt * s3)
    x_new = x + dt / 6.0 * (v1 + 2.0 * v2 + 2.0 * v3 + v4)
    w_new = w + dt / 6.0 * (s1 + 2.0 * s2 + 2.0 * s3 + s4)
    return x_new, w_new
