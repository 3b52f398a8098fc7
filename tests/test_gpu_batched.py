"""Batched form: independent systems in one call give the per-system results."""
import numpy as np
import pytest

import workloads
from oracle import fmm as ofmm
from oracle import tree as T
from tests.gpu_util import dev, host3, rel

pytestmark = pytest.mark.gpu


def _systems(k=4, lo=1500, hi=6000, seed=7):
    return workloads.blob_systems(nsys=k, seed=seed, n_lo=lo, n_hi=hi)


def _batch(systems):
    x = np.concatenate([s[0] for s in systems])
    w = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([s[0].shape[0] for s in systems])])
    return x, w, off


def _same_extent(systems, ext=0.9):
    """The systems scaled to one extent, so that each one's own cube side is the batch's."""
    out = []
    for xs, ws in systems:
        lo = xs.min(axis=0)
        e = float((xs.max(axis=0) - lo).max())
        out.append((((xs - lo) * np.float32(ext / e) + lo).astype(np.float32), ws))
    return out


def test_batched_matches_single_systems():
    from paper_1201_5430_gb300 import LHV
    a, p = 0.01, 8
    systems = _same_extent(_systems())
    sides = {T.cube(xs, T.core_unit(T.core_cutoff(a, 1e-6)))[1] for xs, _ in systems}
    assert len(sides) == 1  # each system's own side is the batch's
    x, w, off = _batch(systems)
    ctx = LHV(p=p, leaf_max=64, core_a=a, precision="fp32")
    v4, s4 = ctx.evaluate_batched(off, dev(x, "fp32"), dev(w, "fp32"))
    L = ctx.stats()["leaf_level"]
    v, s = host3(v4), host3(s4)
    for k, (xs, ws) in enumerate(systems):
        single = LHV(p=p, leaf_max=1, core_a=a, precision="fp32", max_level=L)
        vk, sk = single.evaluate_velocity_stretching(dev(xs, "fp32"), dev(ws, "fp32"))
        assert single.stats()["leaf_level"] == L
        sl = slice(off[k], off[k + 1])
        assert rel(v[sl], host3(vk)) < 1e-6 and rel(s[sl], host3(sk)) < 1e-6


def test_batched_against_oracle():
    from paper_1201_5430_gb300 import LHV
    systems = _systems(k=3, lo=1500, hi=3000, seed=11)
    x, w, off = _batch(systems)
    a, p = 0.01, 8
    ctx = LHV(p=p, leaf_max=64, core_a=a, precision="fp32")
    v4, s4 = ctx.evaluate_batched(off, dev(x, "fp32"), dev(w, "fp32"))
    L = ctx.stats()["leaf_level"]
    # per-system leaf levels of the oracle's rule with the batch's common cube side; the batch
    # uses the deepest, within the core cap
    bs = T.batch_side([xs for xs, _ in systems], a)
    Ls = [T.build_tree(xs, leaf_max=64, a=a, side=bs).L for xs, _ in systems]
    assert L == max(Ls)
    v, s = host3(v4), host3(s4)
    for k, (xs, ws) in enumerate(systems):
        ref = ofmm.fmm(xs, ws, p, a=a, tree=T.build_tree(xs, leaf_max=64, a=a, L_override=L, side=bs))
        sl = slice(off[k], off[k + 1])
        assert rel(v[sl], ref.v) < 1e-6 and rel(s[sl], ref.s) < 1e-6, (k, rel(v[sl], ref.v), rel(s[sl], ref.s))


def test_batched_step_identical_copies_and_empty_system():
    """Two copies of one system advance identically (to rounding); an empty
    system in the batch is allowed."""
    from paper_1201_5430_gb300 import LHV
    (xs, ws), = _systems(k=1, lo=3000, hi=3001, seed=3)
    x = np.concatenate([xs, xs])
    w = np.concatenate([ws, ws])
    n = xs.shape[0]
    off = [0, n, n, 2 * n]
    ctx = LHV(p=8, leaf_max=64, core_a=0.01, precision="tf32x3")
    x4, w4 = dev(x, "fp32"), dev(w, "fp32")
    ctx.step_batched(off, x4, w4, 1e-3)
    gx, gw = host3(x4), host3(w4)
    assert np.abs(gx[:n] - gx[n:]).max() <= 4 * 2.0 ** -24 * np.abs(gx).max()
    assert np.abs(gw[:n] - gw[n:]).max() <= 1e-6 * np.abs(gw).max()
    assert rel(gx[:n] - xs, gx[n:] - xs) < 1e-4
