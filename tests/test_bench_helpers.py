"""Host-side helpers of bench.py (no GPU): the near-field core accounting of the roofline."""
import numpy as np


def test_core_pair_fraction_against_brute_force():
    """The bench's share of near-field pairs inside r_K, on a small synthetic tree."""
    import bench
    rng = np.random.default_rng(0)
    xs = rng.random((200, 3))
    begin, end = np.array([0, 50, 120]), np.array([50, 120, 200])
    col = np.full((3, 27), -1)
    col[0, :2], col[1, :3], col[2, :2] = (0, 1), (0, 1, 2), (1, 2)
    close = total = 0
    for i in range(200):
        b = np.searchsorted(begin, i, side="right") - 1
        for c in col[b][col[b] >= 0]:
            for j in range(begin[c], end[c]):
                if j != i:
                    total += 1
                    close += int(((xs[j] - xs[i]) ** 2).sum() < 0.09)
    assert bench.core_pair_fraction(xs, begin, end, col, 0.3, np.arange(200)) == close / total


def test_core_cutoff_matches_the_oracle():
    import bench
    from oracle import tree as T
    for a, eps in ((0.0063, 1e-6), (0.01, 1e-6), (0.002, 1e-9)):
        assert abs(bench.core_cutoff(a, eps) - T.core_cutoff(a, eps)) < 1e-12 * a
    assert bench.core_cutoff(0.0, 1e-6) == 0.0
