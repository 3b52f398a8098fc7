"""GPU FMM against the oracle: stage outputs and v, s, element by element.

Parity (same p, same tree) is the contract: FP64 within 1e-10 and FP32 within
1e-6 relative L2 for v and s.  Accuracy against the direct sum is checked as well."""
import numpy as np
import pytest

import workloads
from oracle import direct, fmm as ofmm
from oracle import tree as T
from tests.gpu_util import dev, host3, rel, to_complex

pytestmark = pytest.mark.gpu


def _run(x, w, p, leaf, a, prec, terms="all", eps=1e-6):
    from paper_1201_5430_gb300 import LHV
    ctx = LHV(p=p, leaf_max=leaf, core_a=a, eps=eps, precision=prec, terms=terms)
    v4, s4 = ctx.evaluate_velocity_stretching(dev(x, prec), dev(w, prec))
    return ctx, host3(v4), host3(s4)


@pytest.fixture(scope="module")
def cube_fp64():
    x, w, spec = workloads.make("cube_4096")
    ref = ofmm.fmm(x, w, spec["p"], leaf_max=spec["leaf_max"], a=spec["a"], eps=spec["eps"])
    ctx, v, s = _run(x, w, spec["p"], spec["leaf_max"], spec["a"], "fp64")
    return x, w, spec, ref, ctx, v, s


def test_fp64_cube_parity(cube_fp64):
    x, w, spec, ref, ctx, v, s = cube_fp64
    assert ctx.stats()["leaf_level"] == ref.tree.L == 4
    assert rel(v, ref.v) < 1e-10, rel(v, ref.v)
    assert rel(s, ref.s) < 1e-10, rel(s, ref.s)
    v0, _, s0 = direct.direct(x, w, spec["a"])
    assert rel(v, v0) < 1e-3 and rel(s, s0) < 3e-3


def _stage_compare(ctx, ref, what, lev, p, basis, tol):
    tr = ref.tree
    h = tr.h(lev)
    got = ctx.export(what, lev).cpu().numpy().reshape(-1, 2 * p * p)
    want = (ref.multipole if what == "multipole" else ref.local)[lev]
    assert got.shape[0] == len(want)
    worst = 0.0
    for b in range(got.shape[0]):
        phi, chi = to_complex(got[b], p, h, basis)
        for g, wv in ((phi, want[b][0]), (chi, want[b][1])):
            scale = np.abs(wv).max() + 1e-300
            worst = max(worst, float(np.abs(g - wv).max() / scale))
    assert worst < tol, (what, lev, worst)


def test_fp64_stage_outputs(cube_fp64):
    x, w, spec, ref, ctx, v, s = cube_fp64
    p, L = spec["p"], ref.tree.L
    _stage_compare(ctx, ref, "multipole", L, p, "S", 1e-12)   # P2M, Eq. eve4
    _stage_compare(ctx, ref, "multipole", 2, p, "S", 1e-11)   # M2M + Eq. drt11
    _stage_compare(ctx, ref, "local", 2, p, "R", 1e-11)       # M2L + Eq. drt10
    _stage_compare(ctx, ref, "local", L, p, "R", 1e-11)       # M2L + L2L + Eq. drt10


def test_fp64_p20_parity():
    x, w = workloads.cube(1500, 3)
    a = 0.01
    ref = ofmm.fmm(x, w, 20, leaf_max=16, a=a)
    ctx, v, s = _run(x, w, 20, 16, a, "fp64")
    assert ref.tree.L >= 2
    assert rel(v, ref.v) < 1e-10 and rel(s, ref.s) < 1e-10, (rel(v, ref.v), rel(s, ref.s))


@pytest.mark.parametrize("terms", ["near", "far"])
def test_fp64_terms_split(cube_fp64, terms):
    x, w, spec, ref, ctx, v, s = cube_fp64
    ctx2, v2, s2 = _run(x, w, spec["p"], spec["leaf_max"], spec["a"], "fp64", terms=terms)
    want_v = ref.v_near if terms == "near" else ref.v_far
    want_s = ref.s_near if terms == "near" else ref.s_far
    assert rel(v2, want_v) < 1e-10 and rel(s2, want_s) < 1e-10


def test_fp32_cube_parity():
    x, w = workloads.cube(6000, 5)
    a, p = 0.01, 12
    ref = ofmm.fmm(x, w, p, leaf_max=32, a=a)
    ctx, v, s = _run(x, w, p, 32, a, "fp32")
    ev, es = rel(v, ref.v), rel(s, ref.s)
    print(f"fp32 cube p=12: rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < 1e-6 and es < 1e-6, (ev, es)


def test_fp32_ring_parity():
    x, w = workloads.ring(12000, 1)
    a, p = workloads.RING_CORE_A, 12
    ref = ofmm.fmm(x, w, p, leaf_max=64, a=a)
    ctx, v, s = _run(x, w, p, 64, a, "fp32")
    assert ctx.stats()["leaf_level"] == ref.tree.L
    ev, es = rel(v, ref.v), rel(s, ref.s)
    print(f"fp32 ring p=12: rel L2 v {ev:.2e} s {es:.2e}")
    assert ev < 1e-6 and es < 1e-6, (ev, es)


def test_singular_kernel_parity():
    x, w = workloads.cube(3000, 8)
    ref = ofmm.fmm(x, w, 10, leaf_max=16, a=0.0)
    ctx, v, s = _run(x, w, 10, 16, 0.0, "fp64")
    assert rel(v, ref.v) < 1e-10 and rel(s, ref.s) < 1e-10


@pytest.mark.parametrize("tpt", [1, 2, 4])
def test_fp32_singular_kernel_parity(tpt):
    """a = 0: the FP32 pair loop without the core correction, in each warp-tile
    width (32, 64 and 128 targets), against the oracle."""
    from paper_1201_5430_gb300 import LHV
    x, w = workloads.cube(3001, 8)
    ref = ofmm.fmm(x, w, 10, leaf_max=16, a=0.0)
    ctx = LHV(p=10, leaf_max=16, core_a=0.0, precision="fp32")
    ctx.set_launch_shape(tpt, 0, 1, p2p_sources_per_stage=128)
    v4, s4 = ctx.evaluate_velocity_stretching(dev(x, "fp32"), dev(w, "fp32"))
    ev, es = rel(host3(v4), ref.v), rel(host3(s4), ref.s)
    assert ev < 1e-6 and es < 1e-6, (ev, es)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_coincident_elements(prec):
    """Distinct elements at one point (r = 0, j != i) take the limits of the
    smoothed kernel in the near field, in both precisions."""
    x, w = workloads.cube(3001, 4)
    x = x.copy()
    x[1] = x[0]
    x[7] = x[5]
    x[100:104] = x[99]
    a = 0.01
    ref = ofmm.fmm(x, w, 10, leaf_max=32, a=a)
    ctx, v, s = _run(x, w, 10, 32, a, prec)
    assert np.isfinite(v).all() and np.isfinite(s).all()
    tol = 1e-6 if prec == "fp32" else 1e-10
    ev, es = rel(v, ref.v), rel(s, ref.s)
    assert ev < tol and es < tol, (ev, es)


def test_full_size_ring_sampled():
    """The bench workload (262,144-element ring, p = 12, FP32) in the bench's
    launch configuration: the near field of sampled targets against the oracle's
    sum over the same colleague leaves, and v, s against the direct sum."""
    x, w, spec = workloads.make("ring_262144")
    a, p = spec["a"], spec["p"]
    tr = T.build_tree(x, leaf_max=64, a=a, eps=1e-6)
    ctx, vn, sn = _run(x, w, p, 64, a, "fp32", terms="near")
    rng = np.random.default_rng(3)
    sample = rng.choice(x.shape[0], 200, replace=False)
    inv = np.empty_like(tr.perm)
    inv[tr.perm] = np.arange(x.shape[0])
    lv = tr.levels[tr.L]
    leaf_of = np.searchsorted(lv["begin"], inv[sample], side="right") - 1
    from oracle.direct import pair_terms
    xs64, ws64 = x.astype(np.float64), w.astype(np.float64)
    for k, i in enumerate(sample):
        b = leaf_of[k]
        src = np.concatenate([tr.perm[lv["begin"][c]:lv["end"][c]] for c in lv["colleagues"][b]])
        src = src[src != i]
        vv, uu = pair_terms(xs64[i] - xs64[src], ws64[src], a)
        v_ref = vv.sum(axis=0)
        s_ref = ws64[i] @ uu.sum(axis=0)
        assert np.linalg.norm(vn[i] - v_ref) <= 2e-6 * np.linalg.norm(v_ref) + 1e-9
        assert np.linalg.norm(sn[i] - s_ref) <= 2e-5 * np.linalg.norm(s_ref) + 1e-9
    ctx2, v, s = _run(x, w, p, 64, a, "fp32")
    v0, _, s0 = direct.direct_at(x, w, a, sample[:64])
    ev, es = rel(v[sample[:64]], v0), rel(s[sample[:64]], s0)
    print(f"ring 262144 p=12 vs direct sum: v {ev:.2e} s {es:.2e}")
    assert ev < 1e-4 and es < 1e-3
