"""Seeded synthetic vortex-element inputs shared by the tests, the bench and the oracle.

This module holds none of the method's arithmetic: it only draws positions x and
strengths w (FP64 with ``numpy.random.default_rng(seed)``, then rounded once to
FP32, so that every consumer sees identical FP32 values) and names the run
parameters of each workload.

Workloads (shapes follow the paper's test problems, Sec. 5):

* ``cube``   -- N elements uniform in [0, 1]^3, w ~ N(0, 1) per component
                (the error and timing tests of Sec. 5.1-5.2, Table 1).
* ``sphere`` -- N elements uniform on the unit sphere surface (normalised Gaussian
                vectors), w ~ N(0, 1) per component (Table 2).
* ``charges`` -- monopole strengths q ~ N(0, 1) for the scalar reference case.
* ``ring``   -- a thin vortex ring of radius R: theta_i = 2 pi i / N, radial and
                axial jitter ~ N(0, sigma^2); w_i = Gamma (2 pi R / N) / (4 pi) t_i
                with t_i the unit tangent (the element field of Eq. 1 carries no
                1/(4 pi), Eq. 7 puts it into the strengths).
* ``ring_pair`` -- two rings (Sec. 5.3.2): coaxial leapfrogging pair, or an
                offset pair whose second ring is tilted and reversed.
* ``blob_systems`` -- independent systems of Gaussian blob clouds of uneven size,
                strengths xi / (4 pi N_s) with xi ~ N(0, 1) (quadrature weight 1/N_s).
"""
import math

import numpy as np

__all__ = [
    "cube", "sphere", "charges", "ring", "ring_pair", "blob_systems", "WORKLOADS", "make", "make_spec", "to_f4",
    "RING_CORE_A",
]

# Gaussian core of the ring workloads: a = 2 pi R / N_c with N_c = 1000 (Sec. 5.3).
RING_CORE_A = 2.0 * math.pi / 1000.0


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def cube(n, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3))
    w = rng.standard_normal((n, 3))
    return _f32(x), _f32(w)


def sphere(n, seed=0):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 3))
    x = g / np.linalg.norm(g, axis=1)[:, None]
    w = rng.standard_normal((n, 3))
    return _f32(x), _f32(w)


def charges(n, seed=0):
    return np.ascontiguousarray(np.random.default_rng(seed).standard_normal(n).astype(np.float32))


def _rot_x(deg):
    c, s = math.cos(math.radians(deg)), math.sin(math.radians(deg))
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def _ring64(n, rng, radius=1.0, sigma=0.03, gamma=1.0, centre=(0.0, 0.0, 0.0), tilt_deg=0.0):
    theta = 2.0 * math.pi * np.arange(n) / n
    rho = radius + sigma * rng.standard_normal(n)
    z = sigma * rng.standard_normal(n)
    p = np.stack([rho * np.cos(theta), rho * np.sin(theta), z], axis=1)
    tangent = np.stack([-np.sin(theta), np.cos(theta), np.zeros(n)], axis=1)
    w = gamma * (2.0 * math.pi * radius / n) / (4.0 * math.pi) * tangent
    Q = _rot_x(tilt_deg)
    return p @ Q.T + np.asarray(centre), w @ Q.T


def ring(n, seed=1, radius=1.0, sigma=0.03, gamma=1.0):
    rng = np.random.default_rng(seed)
    x, w = _ring64(n, rng, radius, sigma, gamma)
    return _f32(x), _f32(w)


def ring_pair(n_per_ring, seed, kind="leapfrog"):
    """kind="leapfrog": coaxial rings at z = 0 and z = 0.1, Gamma_1 = Gamma_2 = 1.
    kind="offset": ring A at the origin (Gamma = +1); ring B centred at (0, 0, 1.5),
    its normal tilted 30 degrees about the x-axis and its circulation reversed."""
    rng = np.random.default_rng(seed)
    xa, wa = _ring64(n_per_ring, rng)
    if kind == "leapfrog":
        xb, wb = _ring64(n_per_ring, rng, centre=(0.0, 0.0, 0.1))
    elif kind == "offset":
        xb, wb = _ring64(n_per_ring, rng, gamma=-1.0, centre=(0.0, 0.0, 1.5), tilt_deg=30.0)
    else:
        raise ValueError(kind)
    return _f32(np.concatenate([xa, xb])), _f32(np.concatenate([wa, wb]))


def blob_systems(nsys=64, seed=4, n_lo=1e4, n_hi=5e5, blobs=8, sigma=0.05):
    """List of (x, w) per system: sizes log-uniform in [n_lo, n_hi]; each system
    is ``blobs`` Gaussian clouds (centres ~ U[0.2, 0.8]^3, std ``sigma``).
    Strengths w = xi / (4 pi N_s), xi ~ N(0, 1) per component: a unit-strength
    random vorticity field sampled with quadrature weight 1/N_s, the weight and
    the 1/(4 pi) entering w as in Eq. 7."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), nsys))).astype(np.int64)
    out = []
    for ns in sizes:
        counts = np.full(blobs, ns // blobs)
        counts[: ns % blobs] += 1
        xs, ws = [], []
        for c in counts:
            centre = rng.uniform(0.2, 0.8, 3)
            xs.append(centre + sigma * rng.standard_normal((c, 3)))
            ws.append(rng.standard_normal((c, 3)) / (4.0 * math.pi * ns))
        out.append((_f32(np.concatenate(xs)), _f32(np.concatenate(ws))))
    return out


# Named workloads: generator + the run parameters that go with it.
#   p: truncation number (n = 0 .. p-1), leaf_max: elements per leaf bound,
#   a: Gaussian core of Eq. vem1, eps: target accuracy, dt: RK4 step, n: elements.
WORKLOADS = {
    "cube_4096": dict(gen=lambda: cube(4096, 0), n=4096, p=8, leaf_max=64, a=0.01, eps=1e-6, dt=1e-3),
    "ring_262144": dict(gen=lambda: ring(262144, 1), n=262144, p=12, leaf_max=64, a=RING_CORE_A, eps=1e-6,
                        dt=1e-3),
    "offset_rings_2097152": dict(gen=lambda: ring_pair(1 << 20, 2, "offset"), n=1 << 21, p=16, leaf_max=64,
                                 a=RING_CORE_A, eps=1e-6, dt=1e-3),
    "leapfrog_rings_4194304": dict(gen=lambda: ring_pair(1 << 21, 5, "leapfrog"), n=1 << 22, p=12, leaf_max=64,
                                   a=RING_CORE_A, eps=1e-6, dt=5e-4),
}


def make(name):
    spec = dict(WORKLOADS[name])
    x, w = spec.pop("gen")()
    return x, w, spec


def make_spec(name):
    """The run parameters of a named workload without drawing its elements: (None, None, spec)."""
    spec = dict(WORKLOADS[name])
    spec.pop("gen")
    return None, None, spec


def to_f4(a3, dtype=np.float32):
    """(N, 3) -> (N, 4) with a zero fourth lane (the library's element layout)."""
    a3 = np.asarray(a3)
    out = np.zeros((a3.shape[0], 4), dtype=dtype)
    out[:, :3] = a3
    return out
