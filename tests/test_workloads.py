"""The seeded input generators are deterministic and have the stated shapes."""
import math

import numpy as np

import workloads as W


def test_deterministic_and_f32():
    a = W.cube(100, 0)
    b = W.cube(100, 0)
    assert a[0].dtype == np.float32 and a[1].dtype == np.float32
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_ring_geometry():
    x, w = W.ring(4096, 1)
    rho = np.hypot(x[:, 0], x[:, 1])
    assert abs(rho.mean() - 1.0) < 3e-3 and abs(rho.std() - 0.03) < 3e-3
    assert abs(x[:, 2].std() - 0.03) < 3e-3
    # w = Gamma (2 pi R / N) / (4 pi) along the tangent
    np.testing.assert_allclose(np.linalg.norm(w, axis=1), 1.0 / (2 * 4096), rtol=1e-6)
    assert np.abs((w * x).sum(axis=1)).max() < 1e-4 * 0.1


def test_ring_pairs():
    x, w = W.ring_pair(1000, 5, "leapfrog")
    assert x.shape == (2000, 3)
    assert abs(x[1000:, 2].mean() - 0.1) < 5e-3
    x, w = W.ring_pair(1000, 2, "offset")
    assert abs(x[1000:, 2].mean() - 1.5) < 5e-3
    # reversed circulation: ring B rotates the other way about its own normal
    nb = np.array([0.0, -math.sin(math.radians(30)), math.cos(math.radians(30))])
    lb = np.cross(x[1000:] - x[1000:].mean(axis=0), w[1000:]).sum(axis=0)
    assert np.dot(lb, nb) < 0


def test_blob_systems():
    sys_ = W.blob_systems(nsys=4, seed=4, n_lo=100, n_hi=1000)
    assert len(sys_) == 4
    for x, w in sys_:
        assert 100 <= x.shape[0] <= 1000 and x.shape == w.shape


def test_named_workloads_have_parameters():
    for name, spec in W.WORKLOADS.items():
        for k in ("p", "leaf_max", "a", "eps", "dt"):
            assert k in spec
    assert W.WORKLOADS["ring_262144"]["p"] == 12
