"""Throughput of the GB300 Lamb-Helmholtz vortex FMM at equal accuracy eps = 1e-6.

Headline workload: the leapfrogging coaxial ring pair, N = 4,194,304 (two rings of
2^21 at z = 0 and 0.1, R = 1, radial and axial jitter sigma = 0.03, Gaussian core
a = 2 pi / 1000, <= 64 per leaf, dt = 5e-4), the largest single-system workload.
One step = one classical RK4 step (four evaluations of v and s = (w . grad) v, each
with its own octree); consecutive steps of the trajectory from the initial state.
Metric: element evaluations (v and s at one element) per second = 4 N / step time.

Forms compared at equal accuracy, eps_2(v) <= 1e-6 against FP64 direct sums at
1000 sampled elements (relative L2):
  plain_fp32   -- every kernel on the CUDA cores in FP32, the smallest uniform p
                  that reaches eps;
  tf32x3       -- M2L products on the tcgen05 tensor cores in split TF32, the smallest
                  uniform p with tensor-core shapes (a multiple of 4) that reaches eps;
  learned      -- TF32x3 with p per level chosen by the selector network every step
                  (its sampled direct-sum check every 10th step);
  tf32x3_graph -- the tf32x3 arm with each RK4 step as one CUDA graph replay.
`value` is the fastest form that reached eps.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload leapfrog|ring_262144|offset_rings|blobs64]

Multi-GPU (torchrun): every rank advances its own replica (a single system has no
data exchange to shard); value = all ranks' evaluations / the slowest rank's time
("replicas", weak scaling).  blobs64 shards its independent systems over ranks.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "vortex-element v+stretching evals/sec at ε=1e-6 vs plain FP32 GPU FMM; % roofline"
UNIT = "evals/s"
EPS = 1e-6
SINGLE = {"leapfrog": "leapfrog_rings_4194304", "ring_262144": "ring_262144"}
# algorithmic FP32 work of one near-field pair (singular kernel): d (3), r^2 (5), 1/r^3 (3),
# g = f'/r (2), w_j x d (9), v += f (w_j x d) (6), sum f w_j (6), (w_i . d) and g (w_i . d) (6),
# s += g (w_i . d)(w_j x d) (6) = 46 flops
P2P_FLOPS_PER_PAIR = 46
# extra FP32 flops of a pair inside the core radius r_K (the evaluation of K, Eq. vem1, on top of
# the singular terms, in the form K / r^3 = 1/r^3 - exp(-x^2/2) G(a/r) / (a r^2)): t 2, degree-7
# polynomial 14, exp argument 2 (the exp on the SFU), f 3, g 3
P2P_CORE_FLOPS_PER_PAIR = 24
# the oracle sample of the CPU legs: the headline geometry at 2 x 2048 elements
CPU_SAMPLE_PER_RING = 2048


# ---------------------------------------------------------------------------------------
# host-side helpers (tested on the CPU)
# ---------------------------------------------------------------------------------------
def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _traffic_record(name, kernel_file):
    """dram bytes per launch from a committed ncu summary, if it was taken on the current
    source of the kernel and of the tree that sets its work (null otherwise)."""
    path = os.path.join(ROOT, "profiles", name)
    csrc = os.path.join(ROOT, "paper_1201_5430_gb300", "csrc")
    src, tree = os.path.join(csrc, kernel_file), os.path.join(csrc, "tree.cu")
    if not (os.path.exists(path) and os.path.exists(src) and os.path.exists(tree)):
        return None
    rec = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()

    def sha(f):
        return hashlib.sha256(open(f, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != sha(src) or rec.get("tree_sha256_16") != sha(tree):
        return None
    try:
        return float(rec["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def core_cutoff(a, eps):
    """r_K = x_K a with 1 - K(x_K a; a) = eps / 10 (Eq. vem1), by bisection (0 without a core)."""
    import math
    if a <= 0.0:
        return 0.0

    def g(x):
        return math.erfc(x / math.sqrt(2.0)) + math.sqrt(2.0 / math.pi) * x * math.exp(-0.5 * x * x) - eps / 10.0
    lo, hi = 0.0, 60.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if g(mid) > 0.0 else (lo, mid)
    return 0.5 * (lo + hi) * a


def core_pair_fraction(xs, begin, end, colleagues, rK, sample):
    """Of the near-field pairs (target, colleague-leaf source, j != i) of the sorted targets
    ``sample``, the share closer than r_K: the pairs that need the core evaluation of Eq. vem1.
    xs: sorted positions (N, 3); begin/end: leaf element ranges; colleagues: (leaves, 27) leaf
    indices or -1."""
    leaf = np.searchsorted(begin, sample, side="right") - 1
    close = total = 0
    for i, b in zip(sample, leaf):
        src = np.concatenate([np.arange(begin[c], end[c]) for c in colleagues[b] if c >= 0])
        src = src[src != i]
        d = xs[src] - xs[i]
        close += int(((d * d).sum(axis=1) < rK * rK).sum())
        total += src.shape[0]
    return close / total if total else 0.0


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu model", "hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        return clock_summary(open(self.path).read().splitlines() if self.path and os.path.exists(self.path) else [])


def clock_summary(lines):
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


def max_over_ranks(ms, dist, device="cuda"):
    """The slowest rank's time (every rank gets it); `ms` unchanged without a process group."""
    if not dist:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(nsys, rank, world):
    """Systems of this rank: a contiguous block of about nsys / world (independent
    systems need no collective)."""
    lo = nsys * rank // world
    hi = nsys * (rank + 1) // world
    return list(range(lo, hi))


def throughput(evals_per_rank, world, max_ms):
    """Whole-job evaluations per second: the units all ranks processed over the
    slowest rank's time."""
    return evals_per_rank * world / (max_ms / 1e3)


def pick_at_eps(trials, eps):
    """The smallest p whose error meets eps, from (p, err) trials; None if none does."""
    ok = [p for p, e in trials if e is not None and e <= eps]
    return min(ok) if ok else None


def fastest_form(arms, eps):
    """Name of the fastest arm (lowest ms_per_step) among those whose err_v <= eps."""
    cands = [(a["ms_per_step"], k) for k, a in arms.items() if a and a.get("err_v") is not None
             and a["err_v"] <= eps and a.get("ms_per_step")]
    return min(cands)[1] if cands else None


# ---------------------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------------------
def _o2_job(args):
    """One O2 evaluation (plain FP64 CPU FMM) of the sample with seed `seed`; returns
    (elements, seconds)."""
    seed, n_per_ring, p, leaf, a, kind = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import fmm as ofmm
    x, w = workloads.ring_pair(n_per_ring, seed, kind)
    t0 = time.perf_counter()
    ofmm.fmm(x, w, p, leaf_max=leaf, a=a, eps=EPS)
    return x.shape[0], time.perf_counter() - t0


class OraclePool:
    """Process pool (spawn) running O2 on every host core: one independent sample per
    process per round (replicas of the headline geometry at a bounded size)."""

    def __init__(self, cores=None):
        self.cores = cores or os.cpu_count() or 1
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"  # one BLAS thread per process: the pool is the parallelism
        self.pool = mp.get_context("spawn").Pool(self.cores)
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    def round(self, n_per_ring, p, leaf, a, kind, seed0):
        t0 = time.perf_counter()
        res = self.pool.map(_o2_job, [(seed0 + k, n_per_ring, p, leaf, a, kind) for k in range(self.cores)])
        return sum(r[0] for r in res), time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(p, spec, rounds=2, pool=None):
    """The oracle's FMM (O2) as it stands on all host cores: `rounds` rounds of one
    sample per core; evals/s = elements evaluated / wall seconds."""
    own = pool is None
    pool = pool or OraclePool()
    try:
        pool.round(256, p, spec["leaf_max"], spec["a"], "leapfrog", 900)  # imports and warm-up
        tot_n, tot_s = 0, 0.0
        for r in range(rounds):
            n, s = pool.round(CPU_SAMPLE_PER_RING, p, spec["leaf_max"], spec["a"], "leapfrog", 1000 + 100 * r)
            tot_n += n
            tot_s += s
    finally:
        if own:
            pool.close()
    return {"value": tot_n / tot_s, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"O2 (plain FP64 numpy Lamb-Helmholtz FMM, p = {p}) on {rounds} rounds of {pool.cores} "
                      f"independent leapfrogging ring pairs of 2 x {CPU_SAMPLE_PER_RING} elements (same geometry, "
                      f"core a and leaf rule as the headline workload, seeds 1000+), one process per core, "
                      f"{tot_s:.1f} s wall; per-element cost at this N is below that of the full 4,194,304 "
                      f"(fewer near-field sources per target)"}


def run_reference(args, rank, world):
    """The oracle (O2) timed on the host cores: each step is one round of one sample per
    core (measured wall time, nothing extrapolated)."""
    if rank != 0:
        return
    name = SINGLE.get(args.workload, SINGLE["leapfrog"])
    _, _, spec = workloads.make_spec(name)
    p = 16
    pool = OraclePool()
    try:
        for k in range(args.warmup):
            pool.round(CPU_SAMPLE_PER_RING, p, spec["leaf_max"], spec["a"], "leapfrog", 2000 + k)
        tot_n, walls = 0, []
        for k in range(args.steps):
            n, s = pool.round(CPU_SAMPLE_PER_RING, p, spec["leaf_max"], spec["a"], "leapfrog", 3000 + 100 * k)
            tot_n += n
            walls.append(s)
    finally:
        pool.close()
    val = tot_n / sum(walls) if walls else 0.0
    cb = {"value": val, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "cpu_model": cpu_model(),
          "nproc": os.cpu_count(),
          "sample": f"each step: {pool.cores} O2 evaluations (plain FP64 numpy FMM, p = {p}) of independent "
                    f"leapfrogging ring pairs of 2 x {CPU_SAMPLE_PER_RING} elements, one per core"}
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": statistics.mean(walls) * 1e3 if walls else None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": name, "n": spec["n"], "p": p, "leaf_max": spec["leaf_max"], "core_a": spec["a"],
                      "dt": spec["dt"], "eps": EPS, "sample_elements_per_step": tot_n // max(args.steps, 1)},
           "cpu_baseline": cb,
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------------------
# GPU arms
# ---------------------------------------------------------------------------------------
def measure_peaks(torch, lib, stream):
    """Rates of the pipes the kernels are bound by, measured now (lhv_peak_probe)."""
    import ctypes
    from paper_1201_5430_gb300 import _lib
    out = {}
    plan = {"ffma": (20000, 20), "ffma2": (20000, 20), "mufu": (2500, 10), "tf32_mma": (60000, 10),
            "bf16_mma": (60000, 10)}
    for name, (iters, reps) in plan.items():
        rate, ms = ctypes.c_double(0), ctypes.c_double(0)
        st = lib.lhv_peak_probe(_lib.PEAK[name], iters, reps, ctypes.c_void_p(stream.cuda_stream),
                                ctypes.byref(rate), ctypes.byref(ms))
        out[name] = {"rate": rate.value / 1e12 if st == 0 else None, "ms": ms.value, "status": st}
    out["unit"] = "TFLOP/s (mufu: Tops/s)"
    return out



def scalar_ratio(torch, LHV, n=1 << 20, p=12, leaves=(32, 64, 128, 256)):
    """The paper's central cost ratio (Sec. 5.2, Tables 1-2, Fig. 3): run time of v and s
    (vortex elements, singular kernel) over that of phi and grad phi (the scalar reference
    case, monopoles) on the same distribution, p = 12, each at its fastest leaf size (the
    paper optimises l_max per case); uniform cube and sphere surface.  One evaluation
    each, CUDA events, mean of 3 after a warm-up."""
    out = {"p": p, "n": n, "precision": "tf32x3", "paper_mean_ratio": 1.405}

    def t(c, f):
        f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            f()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / 3

    for dist, gen in (("cube", workloads.cube), ("sphere", workloads.sphere)):
        x, w = gen(n, 7)
        q = workloads.charges(n, 8)
        x0 = torch.from_numpy(workloads.to_f4(x)).cuda()
        w0 = torch.from_numpy(workloads.to_f4(w)).cuda()
        q0 = torch.from_numpy(q).cuda()
        rec = {}
        for form in ("v_s", "phi_grad"):
            best = None
            for leaf in leaves:
                c = LHV(p=p, leaf_max=leaf, core_a=0.0, precision="tf32x3")
                f = (lambda: c.evaluate_velocity_stretching(x0, w0)) if form == "v_s" else \
                    (lambda: c.evaluate_potential_gradient(x0, q0))
                ms = t(c, f)
                if best is None or ms < best["ms"]:
                    best = {"ms": ms, "leaf_max": leaf, "leaf_level": c.stats()["leaf_level"]}
                c.close()
            rec[form] = best
        rec["ratio"] = rec["v_s"]["ms"] / rec["phi_grad"]["ms"]
        out[dist] = rec
    return out



def vfm_ring(torch, LHV, n=1 << 20, p=16, reps=3):
    """Vortex filaments (Sec. 5.3): one closed ring of n segments (R = 1, Gamma = 1), v at the
    n nodes by the FMM (TF32x3, segments in closed form near, Gauss-Legendre S-expansions far).
    Error against the FP64 FMM at p = 20 at every node; the mean axial speed against Eq. dis6,
    Gamma / (4 pi R) ln(2 n / pi)."""
    import math
    th = 2.0 * math.pi * np.arange(n) / n
    x = np.stack([np.cos(th), np.sin(th), np.zeros(n)], axis=1)
    g = np.ones(n)
    out = {"n": n, "p": p, "precision": "tf32x3"}
    ref = LHV(p=20, leaf_max=64, core_a=0.0, precision="fp64")
    x64 = torch.from_numpy(workloads.to_f4(x.astype(np.float32), np.float64)).cuda()
    v64 = ref.evaluate_filaments([0, n], [True], x64, torch.from_numpy(g).cuda())
    ref.close()
    c = LHV(p=p, leaf_max=64, core_a=0.0, precision="tf32x3")
    x32 = torch.from_numpy(workloads.to_f4(x.astype(np.float32))).cuda()
    g32 = torch.ones(n, device="cuda")
    v = c.evaluate_filaments([0, n], [True], x32, g32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        c.evaluate_filaments([0, n], [True], x32, g32, v)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    d = (v[:, :3].double() - v64[:, :3])
    out["ms_per_evaluation"] = ms
    out["evals_per_s"] = n / (ms / 1e3)
    out["err_v_vs_fp64_p20"] = float(torch.linalg.norm(d) / torch.linalg.norm(v64[:, :3]))
    out["mean_axial_speed"] = float(v[:, 2].double().mean())
    out["eq_dis6"] = math.log(2 * n / math.pi) / (4.0 * math.pi)
    out["leaf_level"] = c.stats()["leaf_level"]
    c.close()
    return out


def rcr_macs(p, padded=True):
    """Multiply-adds per M2L pair of the RCR products (Sec. 4.4) as the kernel runs them: the
    z-phases (2 x 2 per order m > 0) and the y-turn blocks (even class n + 1, odd class n per
    degree; output rows padded to 4 in the kernel) both ways for both potentials, the coaxial
    blocks A_m (both potentials, Re and Im) and the conversion of Eq. rcr1."""
    q = (lambda k: (k + 3) // 4 * 4) if padded else (lambda k: k)
    y = sum((n + 1) * q(n + 1) + n * q(n) for n in range(p))
    z = 4 * sum(n for n in range(p))
    cx = sum((2 if m else 1) * (p - m) * q(p - m) for m in range(p))
    conv = sum((2 if m else 0) + ((2 if m else 1) if n + 1 < p else 0) for n in range(p) for m in range(n + 1))
    return 2 * 2 * (y + z) + 2 * cx + conv


def m2l_forms(torch, LHV, n=1 << 20, ps=(12, 16, 20), reps=2, fma_peak=None):
    """M2L products by the fused tables on the tensor cores (TF32x3) against RCR translations
    on the CUDA cores (FP32), uniform cube of n elements, far field only: time per evaluation
    (CUDA events around the products), box pairs, useful flops and agreement of v."""
    x, w = workloads.cube(n, 5)
    X = torch.from_numpy(workloads.to_f4(x)).cuda()
    W = torch.from_numpy(workloads.to_f4(w)).cuda()
    out = {"n": n, "workload": "uniform cube", "rows": []}
    for p in ps:
        row = {"p": p}
        vs = {}
        for form, prec in (("phi_chi", "tf32x3"), ("rcr", "fp32")):
            c = LHV(p=p, leaf_max=64, core_a=0.0005, eps=1e-6, precision=prec, terms="far")
            c.set_form(form)
            v4, s4 = c.evaluate_velocity_stretching(X, W)
            torch.cuda.synchronize()
            c.set_timing(True)
            c.reset_stats()
            for _ in range(reps):
                c.evaluate_velocity_stretching(X, W, v4, s4)
            torch.cuda.synchronize()
            st = c.stats()
            key = "fused_tf32x3" if form == "phi_chi" else "rcr_fp32"
            row[key + "_ms"] = st["stage_ms"]["m2l_products"] / reps
            row["pairs"] = st["m2l_pairs"]
            row["leaf_level"] = st["leaf_level"]
            vs[key] = v4[:, :3].double()
            c.close()
        row["rcr_over_fused"] = row["rcr_fp32_ms"] / row["fused_tf32x3_ms"]
        row["rel_l2_v_rcr_vs_fused"] = float(torch.linalg.norm(vs["rcr_fp32"] - vs["fused_tf32x3"])
                                             / torch.linalg.norm(vs["fused_tf32x3"]))
        row["rcr_useful_flops_per_pair"] = 2 * rcr_macs(p, padded=False)
        row["rcr_issued_flops_per_pair"] = 2 * rcr_macs(p)
        row["fused_useful_flops_per_pair"] = 6 * p ** 4
        tf = row["rcr_issued_flops_per_pair"] * row["pairs"] / (row["rcr_fp32_ms"] / 1e3) / 1e12
        row["rcr_tflops_issued"] = tf
        if fma_peak:
            row["rcr_frac_of_fma_peak"] = tf / fma_peak
        out["rows"].append(row)
    return out


def run_single(args, torch, LHV, local, world, rank, dist):
    from paper_1201_5430_gb300 import _lib, selector
    name = SINGLE[args.workload]
    x, w, spec = workloads.make(name)
    n = x.shape[0]
    x0 = torch.from_numpy(workloads.to_f4(x)).cuda()
    w0 = torch.from_numpy(workloads.to_f4(w)).cuda()
    x4, w4 = x0.clone(), w0.clone()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def ctx(p, prec):
        return LHV(p=p, leaf_max=spec["leaf_max"], core_a=spec["a"], eps=spec["eps"], precision=prec)

    if args.profile:  # ncu target: one warm-up evaluation and one evaluation, nothing else
        c = ctx(16, "tf32x3")
        if args.form == "rcr":
            c = LHV(p=16, leaf_max=spec["leaf_max"], core_a=spec["a"], eps=spec["eps"], precision="fp32")
            c.set_form("rcr")
        for _ in range(2):
            c.evaluate_velocity_stretching(x4, w4)
        torch.cuda.synchronize()
        return

    # reference values at 1000 sampled elements: FP64 direct sums on the GPU
    idx = torch.from_numpy(np.random.default_rng(0).choice(n, 1000, replace=False).astype(np.int32)).cuda()
    il = idx.long()
    ref = LHV(p=4, leaf_max=spec["leaf_max"], core_a=spec["a"])
    v0, s0 = ref.direct_sampled(x0, w0, idx)
    ref.close()

    def errs(v, s):
        ev = float(torch.linalg.norm(v[il].double()[:, :3] - v0[:, :3]) / torch.linalg.norm(v0[:, :3]))
        es = float(torch.linalg.norm(s[il].double()[:, :3] - s0[:, :3]) / torch.linalg.norm(s0[:, :3]))
        return ev, es

    peaks, peak_kind = _measured_peaks()
    with Clocks(local) as pclk:
        probes = measure_peaks(torch, _lib.load(), stream)
    probes["clocks"] = pclk.summary()

    # launch shape of the near field (the same for every form): tuned once, outside the timed regions
    tuner = ctx(16, "tf32x3")
    shape = tuner.autotune(x0, w0)
    tuner.close()

    def configured(p, prec):
        c = ctx(p, prec)
        c.set_launch_shape(shape["p2p_targets_per_thread"], 0, 1 if prec == "tf32x3" else 0,
                           p2p_sources_per_stage=shape["p2p_sources_per_stage"])
        return c

    # the smallest p that reaches eps, per precision (tensor-core shapes: multiples of 4)
    search = {}
    for prec, cand in (("fp32", range(13, 21)), ("tf32x3", (12, 16, 20))):
        trials = []
        for p in cand:
            c = configured(p, prec)
            v, s = c.evaluate_velocity_stretching(x0, w0)
            trials.append((p, *errs(v, s)))
            c.close()
            if trials[-1][1] <= EPS:
                break
        search[prec] = {"trials": [{"p": p, "err_v": ev, "err_s": es} for p, ev, es in trials],
                        "p": pick_at_eps([(p, ev) for p, ev, _ in trials], EPS)}

    def timed(c, steps, warmup, clocks=None):
        """consecutive RK4 steps from the initial state, L2 flushed before each, CUDA events
        on the context stream around each step"""
        x4.copy_(x0)
        w4.copy_(w0)
        for _ in range(max(warmup, 3)):
            c.step(x4, w4, spec["dt"])
        x4.copy_(x0)
        w4.copy_(w0)
        torch.cuda.synchronize()
        c.set_timing(True)
        c.reset_stats()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            flush.zero_()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            c.step(x4, w4, spec["dt"])
            eb.record(stream)
            eb.synchronize()
            times.append(ea.elapsed_time(eb))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        st = c.stats()
        c.set_timing(False)
        return times, st

    def arm_record(times, st, p, ev, es):
        return {"p": p, "err_v": ev, "err_s": es, "ms_per_step": float(np.mean(times)),
                "stage_ms_per_step": {k: v / len(times) for k, v in st["stage_ms"].items() if v > 0}}

    # screening: every form over a few steps; then the fastest one at eps over all the steps
    screen_steps = min(args.steps, 5)
    arms, makers = {}, {}
    for prec, key in (("fp32", "plain_fp32"), ("tf32x3", "tf32x3")):
        p = search[prec]["p"]
        if p is None:
            arms[key] = None
            continue
        ev, es = next((t["err_v"], t["err_s"]) for t in search[prec]["trials"] if t["p"] == p)
        makers[key] = (lambda p=p, prec=prec: configured(p, prec), p, ev, es)
        if prec == "tf32x3":  # the same arm with each RK4 step as one CUDA graph replay
            def graphed(p=p):
                c = configured(p, "tf32x3")
                c.set_graph(True)
                return c
            makers["tf32x3_graph"] = (graphed, p, ev, es)
    W, b, _ = selector.load()

    def learned():
        c = configured(spec["p"], "tf32x3")
        c.set_selector(W, b, eps=EPS, check_every=10, check_samples=1000)
        return c

    c = learned()
    v, s = c.evaluate_velocity_stretching(x0, w0)
    lev, les = errs(v, s)
    lst = c.stats()
    c.close()
    makers["learned_tf32x3"] = (learned, None, lev, les)
    screen_stats = {}
    for key, (mk, p, ev, es) in makers.items():
        c = mk()
        t, st = timed(c, screen_steps, 3)
        screen_stats[key] = st
        arms[key] = arm_record(t, st, p if p else st["level_p"], ev, es)
        if key == "learned_tf32x3":
            arms[key]["initial_selection"] = {"level_p": lst["level_p"], "check_err_v": lst["selector"]["err_v"],
                                              "check_err_s": lst["selector"]["err_s"],
                                              "fallbacks": lst["selector"]["fallbacks"]}
            arms[key]["checks_in_timed_steps"] = st["selector"]["checks"]
            arms[key]["fallbacks_in_timed_steps"] = st["selector"]["fallbacks"]
        c.close()
    head = fastest_form(arms, EPS) or "tf32x3"
    c = makers[head][0]()
    with Clocks(local) as clk:
        times, st = timed(c, args.steps, args.warmup)
    total_ms = max_over_ranks(sum(times), dist)
    value = throughput(4 * n * args.steps, world, total_ms)
    arms[head]["ms_per_step_full_run"] = total_ms / args.steps

    # roofline of the dominant kernel (near field): algorithmic FP32 flops per launch / its mean duration.
    # Captured steps record no stage events: the graph arm's kernels are timed in its uncaptured twin.
    if st["stage_ms"].get("p2p", 0.0) <= 0.0:
        st = dict(screen_stats["tf32x3"], kernel_launches=st["kernel_launches"], graph=st.get("graph"))
    p2p_ms = st["stage_ms"]["p2p"] / max(st["stage_launches"]["p2p"], 1)
    pairs = st["p2p_pairs"]
    # the share of the pairs inside r_K (the core evaluation they need), on 2000 sampled targets of
    # the initial tree (a context that builds it uncaptured, so its lists can be exported)
    rK = core_cutoff(spec["a"], spec["eps"])
    core_frac = 0.0
    if rK > 0.0:
        tc_ = ctx(16, "tf32x3")
        tc_.build_tree(x0)
        L = tc_.stats()["leaf_level"]
        perm = tc_.export("perm").cpu().numpy()
        rng_ = tc_.export("box_range", L).cpu().numpy().reshape(-1, 2)
        col = tc_.export("colleagues", L).cpu().numpy().reshape(-1, 27)
        tc_.close()
        xs_np = x[perm].astype(np.float64)
        samp = np.sort(np.random.default_rng(1).choice(n, 2000, replace=False))
        core_frac = core_pair_fraction(xs_np, rng_[:, 0], rng_[:, 1], col, rK, samp)
    flops_pair = P2P_FLOPS_PER_PAIR + P2P_CORE_FLOPS_PER_PAIR * core_frac
    achieved = flops_pair * pairs / (p2p_ms / 1e3) / 1e12
    achieved_singular = P2P_FLOPS_PER_PAIR * pairs / (p2p_ms / 1e3) / 1e12
    fma_peak = max(probes["ffma"]["rate"] or 0.0, probes["ffma2"]["rate"] or 0.0)
    m2l_ms = st["stage_ms"].get("m2l_products", 0.0) / max(st["stage_launches"].get("m2l_products", 0), 1)
    m2l_p = st["level_p"][-1] if st["level_p"] else spec["p"]
    m2l_flops = 6.0 * m2l_p ** 4 * st["m2l_pairs"]
    tf32_peak = probes["tf32_mma"]["rate"]
    tc = head != "plain_fp32"

    # end to end through the C ABI with host buffers (H2D, step, D2H inside the timed region),
    # L2 flushed before each step as in the device-timed arm
    hx = x0.cpu().pin_memory()
    hw = w0.cpu().pin_memory()
    hx0, hw0 = hx.clone(), hw.clone()
    e2e_times = []
    e2e_steps = min(args.steps, 5)
    for i in range(e2e_steps + 1):
        hx.copy_(hx0)
        hw.copy_(hw0)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.step_host(hx, hw, spec["dt"])
        if i > 0:  # the first is a warm-up of the host copies' buffers
            e2e_times.append(time.perf_counter() - t0)
    e2e_val = 4 * n * world / statistics.mean(e2e_times)
    c.close()
    ratio = None if args.no_scalar_ratio else scalar_ratio(torch, LHV)
    batched = None if args.no_batched else batched_form(torch, LHV, min(args.steps, 3), 3)
    filaments = None if args.no_filaments else vfm_ring(torch, LHV)
    rcr = None if args.no_rcr else m2l_forms(torch, LHV, fma_peak=fma_peak)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cb = None if args.no_cpu_baseline else cpu_baseline(arms[head]["p"] if isinstance(arms[head]["p"], int) else 16,
                                                        spec)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if head == "plain_fp32" else "f32+tf32x3",
        "data": "synthetic",
        "config": {"workload": name, "n": n, "form": head, "p": arms[head]["p"], "leaf_max": spec["leaf_max"],
                   "core_a": spec["a"], "eps": EPS, "dt": spec["dt"], "rk4_evals_per_step": 4,
                   "steps": "consecutive RK4 steps of the trajectory from the initial state",
                   "accuracy": "eps_2(v) vs FP64 direct sums at 1000 sampled elements (err_s reported)",
                   "l2": "flushed before every step (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "leaf_level": st["leaf_level"], "boxes": st["nbox"]},
        "err_v": arms[head]["err_v"], "err_s": arms[head]["err_s"],
        "forms_at_eps_1e-6": {"arms": arms, "p_search": search, "screen_steps": screen_steps,
                              "speedup_vs_plain_fp32": {k: arms["plain_fp32"]["ms_per_step"] / a["ms_per_step"]
                                                        for k, a in arms.items() if a and arms.get("plain_fp32")}},
        "roofline": {"kernel": "k_p2p_x2 (near field, packed FP32x2)", "bound": "alu", "achieved": achieved,
                     "peak": fma_peak, "unit": "TFLOP/s", "frac": achieved / fma_peak if fma_peak else None,
                     "traffic": _traffic_record("p2p_leapfrog_traffic.txt", "p2p.cu"),
                     "peak_kind": "measured in this run: FP32 FMA probe (lhv_peak_probe, max of scalar and "
                                  "packed FP32x2), median of 20 launches at the running clocks",
                     "pairs_per_launch": pairs, "flops_per_pair": flops_pair,
                     "flops_per_pair_parts": {"singular": P2P_FLOPS_PER_PAIR, "core": P2P_CORE_FLOPS_PER_PAIR,
                                              "core_pair_fraction": core_frac, "r_K": rK,
                                              "core_fraction_sample": "2000 targets of the initial tree"},
                     "frac_singular_only": achieved_singular / fma_peak if fma_peak else None,
                     "mean_launch_ms": p2p_ms},
        "roofline_m2l": {"kernel": "M2L products, " + ("tcgen05 TF32 x3 (k_tc_gemm)" if tc else "CUDA cores"),
                         "bound": "tensor" if tc else "alu",
                         "achieved": m2l_flops / (m2l_ms / 1e3) / 1e12 if m2l_ms else None,
                         "peak": tf32_peak if tc else fma_peak, "unit": "TFLOP/s",
                         "frac": (m2l_flops / (m2l_ms / 1e3) / 1e12) / (tf32_peak if tc else fma_peak)
                         if m2l_ms and (tf32_peak if tc else fma_peak) else None,
                         "peak_kind": "measured in this run: tcgen05.mma kind::tf32 probe" if tc
                         else "measured FP32 FMA probe", "box_pairs": st["m2l_pairs"],
                         "flops_per_pair": 6 * m2l_p ** 4, "useful_only": "split products issue 3x these flops",
                         "frac_issued": (3.0 if tc else 1.0) * (m2l_flops / (m2l_ms / 1e3) / 1e12)
                         / (tf32_peak if tc else fma_peak) if m2l_ms and (tf32_peak if tc else fma_peak) else None,
                         "mean_launch_ms": m2l_ms},
        "peaks_measured": probes,
        "peaks_driver": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")},
        "peaks_driver_kind": peak_kind,
        "stage_ms_per_step": {k: v / max(st["stage_launches"].get("p2p", 4) // 4, 1)
                              for k, v in st["stage_ms"].items() if v > 0},
        "launch_shape": shape,
        "graph": st.get("graph"),
        "t_vs_over_t_phigrad": ratio,
        "batched_form_blobs64": batched,
        "filaments_ring": filaments,
        "m2l_rcr_vs_fused": rcr,
        "cpu_baseline": cb,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(2 * n * 16),
                "d2h_bytes_per_step": int(2 * n * 16), "steps": e2e_steps},
        "gpu_launches": st["kernel_launches"],
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def batched_form(torch, LHV, steps, warmup, rank=0, world=1, precision="tf32x3"):
    """Batched form: 64 independent Gaussian-blob systems (sizes log-uniform in
    [1e4, 5e5], about 1e7 elements), one RK4 step per timed step from the same state, three
    arms in the same precision: (a) one lhv_step_batched call for all systems, (b) the same
    with the whole step as one CUDA graph replay, (c) the single-system path called once per
    system.  Independent systems shard over ranks (a block each, no collective)."""
    systems = workloads.blob_systems(64, 4)
    mine = shard(64, rank, world)
    systems = [systems[k] for k in mine]
    x = np.concatenate([q[0] for q in systems])
    w = np.concatenate([q[1] for q in systems])
    off = [0] + [int(v) for v in np.cumsum([q[0].shape[0] for q in systems])]
    n = int(off[-1])
    spec = dict(p=12, leaf_max=64, a=0.01, eps=1e-6, dt=1e-3)
    side = torch.cuda.Stream()  # graph capture needs a stream other than the legacy default
    out = {"systems": len(systems), "n": n, **spec, "precision": precision}
    with torch.cuda.stream(side):
        x0 = torch.from_numpy(workloads.to_f4(x)).cuda()
        w0 = torch.from_numpy(workloads.to_f4(w)).cuda()
        x4, w4 = x0.clone(), w0.clone()

        def timed(fn):
            for _ in range(max(warmup, 3)):
                x4.copy_(x0)
                w4.copy_(w0)
                fn()
            side.synchronize()
            tot = 0.0
            for _ in range(steps):
                x4.copy_(x0)
                w4.copy_(w0)
                ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ea.record(side)
                fn()
                eb.record(side)
                eb.synchronize()
                tot += ea.elapsed_time(eb)
            return tot / steps

        def make():
            return LHV(p=spec["p"], leaf_max=spec["leaf_max"], core_a=spec["a"], eps=spec["eps"],
                       precision=precision, stream=side)

        cb = make()
        tuned = cb.autotune(x0, w0, offsets=off)  # launch shapes for the batch, outside the timed regions
        out["launch_shape"] = tuned
        out["batched_ms_per_step"] = timed(lambda: cb.step_batched(off, x4, w4, spec["dt"]))
        cg = make()
        cg.set_launch_shape(tuned["p2p_targets_per_thread"], tuned["m2l_pairs_per_chunk"], tuned["m2l_tensor_cores"],
                            p2p_sources_per_stage=tuned["p2p_sources_per_stage"])
        cg.set_graph(True)
        cg.reset_stats()
        out["batched_graph_ms_per_step"] = timed(lambda: cg.step_batched(off, x4, w4, spec["dt"]))
        out["graph"] = cg.stats()["graph"]
        cs = make()
        cs.set_launch_shape(tuned["p2p_targets_per_thread"], tuned["m2l_pairs_per_chunk"], tuned["m2l_tensor_cores"],
                            p2p_sources_per_stage=tuned["p2p_sources_per_stage"])

        def seq():
            for k in range(len(systems)):
                cs.step(x4[off[k]:off[k + 1]], w4[off[k]:off[k + 1]], spec["dt"])

        out["sequential_ms_per_step"] = timed(seq)
        out["leaf_level"] = cb.stats()["leaf_level"]
        for c in (cb, cg, cs):
            c.close()
    for k in ("batched", "batched_graph", "sequential"):
        out[k + "_evals_per_s"] = 4 * n * world / (out[k + "_ms_per_step"] / 1e3)
    out["speedup_batched_vs_sequential"] = out["sequential_ms_per_step"] / out["batched_ms_per_step"]
    out["speedup_graph_vs_sequential"] = out["sequential_ms_per_step"] / out["batched_graph_ms_per_step"]
    out["steps"] = steps
    return out


def run_learned_trajectory(args, torch, LHV, rank):
    """The learned form over the leapfrog pair's trajectory: per-step selection (sampled
    checks against FP64 direct sums every 10 steps), against uniform TF32x3 p = 16 (the
    smallest tensor-core p that reaches eps on this workload) over the same consecutive RK4
    steps from the initial state; L2 flushed before each step, CUDA events around each; the
    final states' eps_2(v), eps_2(s) at 1000 sampled elements against FP64 direct sums."""
    from paper_1201_5430_gb300 import selector
    name = SINGLE["leapfrog"]
    x, w, spec = workloads.make(name)
    n = x.shape[0]
    steps = args.trajectory_steps
    x0 = torch.from_numpy(workloads.to_f4(x)).cuda()
    w0 = torch.from_numpy(workloads.to_f4(w)).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    W, b, _ = selector.load()
    idx = torch.from_numpy(np.random.default_rng(0).choice(n, 1000, replace=False).astype(np.int32)).cuda()
    il = idx.long()
    arms, finals = {}, {}
    for key in ("uniform_tf32x3_p16", "learned_tf32x3"):
        learned = key.startswith("learned")
        c = LHV(p=spec["p"] if learned else 16, leaf_max=spec["leaf_max"], core_a=spec["a"], eps=spec["eps"],
                precision="tf32x3")
        if learned:
            c.set_selector(W, b, eps=EPS, check_every=10, check_samples=1000)
        x4, w4 = x0.clone(), w0.clone()
        for _ in range(3):
            c.step(x4, w4, spec["dt"])
        x4.copy_(x0)
        w4.copy_(w0)
        torch.cuda.synchronize()
        c.set_timing(True)
        c.reset_stats()
        times, schedules = [], {}
        with Clocks(0) as clk:
            for _ in range(steps):
                flush.zero_()
                ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ea.record(stream)
                c.step(x4, w4, spec["dt"])
                eb.record(stream)
                eb.synchronize()
                times.append(ea.elapsed_time(eb))
                if learned:
                    k = ",".join(str(v) for v in c.stats()["level_p"])
                    schedules[k] = schedules.get(k, 0) + 1
        st = c.stats()
        v, s_ = c.evaluate_velocity_stretching(x4, w4)
        ref = LHV(p=4, leaf_max=spec["leaf_max"], core_a=spec["a"])
        vr, sr = ref.direct_sampled(x4, w4, idx)
        ref.close()
        rec = {"ms_per_step": float(np.mean(times)), "ms_total": float(np.sum(times)),
               "ms_per_step_first_last_10": [float(np.mean(times[:10])), float(np.mean(times[-10:]))],
               "final_err_v": float(torch.linalg.norm(v[il].double()[:, :3] - vr[:, :3])
                                    / torch.linalg.norm(vr[:, :3])),
               "final_err_s": float(torch.linalg.norm(s_[il].double()[:, :3] - sr[:, :3])
                                    / torch.linalg.norm(sr[:, :3])),
               "leaf_level_final": st["leaf_level"], "clocks": clk.summary()}
        if learned:
            rec["schedules"] = schedules
            rec["checks"] = st["selector"]["checks"]
            rec["fallbacks"] = st["selector"]["fallbacks"]
            rec["check_err_v_last"] = st["selector"]["err_v"]
        arms[key] = rec
        finals[key] = x4[:, :3].double().clone()
        c.close()
    x00 = x0[:, :3].double()
    drift = float(torch.linalg.norm(finals["learned_tf32x3"] - finals["uniform_tf32x3_p16"])
                  / torch.linalg.norm(finals["uniform_tf32x3_p16"] - x00))
    speed = arms["uniform_tf32x3_p16"]["ms_per_step"] / arms["learned_tf32x3"]["ms_per_step"]
    if rank == 0:
        print(json.dumps({"metric": METRIC + " (learned form over the trajectory)",
                          "value": 4 * n / (arms["learned_tf32x3"]["ms_per_step"] / 1e3), "unit": UNIT,
                          "n_gpus": 1, "steps": steps, "warmup": 3,
                          "ms_per_step": arms["learned_tf32x3"]["ms_per_step"], "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f32+tf32x3", "data": "synthetic",
                          "config": {"workload": name, "n": n, "dt": spec["dt"], "eps": EPS,
                                     "l2": "flushed before every step (256 MB write)"},
                          "speedup_learned_vs_uniform_p16": speed,
                          "final_positions_rel_diff_vs_displacement": drift, "arms": arms}), flush=True)


def run_blobs64(args, torch, LHV, local, world, rank, dist):
    """The batched form's own line (see batched_form)."""
    r = batched_form(torch, LHV, args.steps, args.warmup, rank, world, args.precision)
    ms = max_over_ranks(r["batched_graph_ms_per_step"], dist)
    tot_n = r["n"]
    if dist:
        tn = torch.tensor([float(tot_n)], dtype=torch.float64, device="cuda")
        dist.all_reduce(tn)
        tot_n = int(tn.item())
    if rank == 0:
        print(json.dumps({"metric": METRIC + " (batched form)", "value": 4 * tot_n / (ms / 1e3), "unit": UNIT,
                          "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
                          "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
                          "dtype": "f32" if args.precision == "fp32" else "f32+tf32x3", "data": "synthetic",
                          "config": {"workload": "blobs64", "n": tot_n, "form": "batched + CUDA graph"},
                          "arms": r}), flush=True)


def run_offset_rings(args, torch, LHV, local, world, rank, dist):
    """Mixed-precision form on the two colliding offset rings (2 x 2^20 elements, p = 16):
    evaluations of v and s per second, TF32x3 against plain FP32, each with its error
    against FP64 direct sums at 10,000 random targets (GPU direct-sum kernel)."""
    x, w, spec = workloads.make("offset_rings_2097152")
    n = x.shape[0]
    x0 = torch.from_numpy(workloads.to_f4(x)).cuda()
    w0 = torch.from_numpy(workloads.to_f4(w)).cuda()
    stream = torch.cuda.current_stream()
    idx = torch.from_numpy(np.random.default_rng(3).choice(n, 10000, replace=False).astype(np.int32)).cuda()
    ref = LHV(p=4, leaf_max=spec["leaf_max"], core_a=spec["a"])
    v0, s0 = ref.direct_sampled(x0, w0, idx)
    ref.close()
    out = {}
    for prec in ("fp32", "tf32x3"):
        c = LHV(p=spec["p"], leaf_max=spec["leaf_max"], core_a=spec["a"], eps=spec["eps"], precision=prec)
        c.autotune(x0, w0)
        v, s = c.evaluate_velocity_stretching(x0, w0)
        il = idx.long()
        ev = float(torch.linalg.norm(v[il].double()[:, :3] - v0[:, :3]) / torch.linalg.norm(v0[:, :3]))
        es = float(torch.linalg.norm(s[il].double()[:, :3] - s0[:, :3]) / torch.linalg.norm(s0[:, :3]))
        for _ in range(3):
            c.evaluate_velocity_stretching(x0, w0)
        torch.cuda.synchronize()
        c.set_timing(True)
        c.reset_stats()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(args.steps):
            c.evaluate_velocity_stretching(x0, w0)
        eb.record(stream)
        eb.synchronize()
        ms = max_over_ranks(ea.elapsed_time(eb), dist) / args.steps
        st = c.stats()
        out[prec] = {"ms_per_evaluation": ms, "evals_per_s": n * world / (ms / 1e3), "err_v": ev, "err_s": es,
                     "stage_ms_per_evaluation": {k: v / args.steps for k, v in st["stage_ms"].items() if v > 0},
                     "p2p_pairs": st["p2p_pairs"], "m2l_pairs": st["m2l_pairs"], "leaf_level": st["leaf_level"]}
        c.close()
    if rank == 0:
        print(json.dumps({"metric": METRIC + " (mixed-precision form)", "value": out["tf32x3"]["evals_per_s"],
                          "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": 3,
                          "ms_per_step": out["tf32x3"]["ms_per_evaluation"], "higher_is_better": True,
                          "scaling": "weak", "dtype": "f32+tf32x3", "data": "synthetic",
                          "config": {"workload": "offset_rings_2097152", "n": n, "p": spec["p"], "a": spec["a"],
                                     "step": "one evaluation of v and s",
                                     "error_sample": "10,000 random targets, FP64 direct sums"},
                          "arms": out,
                          "speedup_vs_plain_fp32": out["fp32"]["ms_per_evaluation"] / out["tf32x3"]["ms_per_evaluation"]}),
              flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scalar-ratio", action="store_true",
                    help="skip T(v, s) / T(phi, grad phi) against the scalar reference case")
    ap.add_argument("--no-filaments", action="store_true",
                    help="skip the vortex filament ring (segments, Sec. 5.3)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched form (64 blob systems: batched, CUDA graph, per system)")
    ap.add_argument("--workload", default="leapfrog",
                    choices=list(SINGLE) + ["blobs64", "offset_rings", "filaments", "leapfrog_learned"],
                    help="leapfrog (headline), ring_262144 (single ring), offset_rings (mixed precision on "
                         "two offset colliding rings of 2,097,152 elements), blobs64 (the batched form), "
                         "filaments (vortex filament ring), leapfrog_learned (the learned form over 100 steps)")
    ap.add_argument("--precision", default="tf32x3", choices=["tf32x3", "fp32"],
                    help="blobs64 only: tf32x3 (M2L on the tensor cores) or fp32")
    ap.add_argument("--trajectory-steps", type=int, default=100,
                    help="leapfrog_learned: consecutive RK4 steps of each arm")
    ap.add_argument("--no-rcr", action="store_true",
                    help="skip the M2L products by RCR translations against the fused tables (uniform cube)")
    ap.add_argument("--form", default="phi_chi", choices=["phi_chi", "rcr"],
                    help="--profile only: the far-field form of the profiled evaluations (rcr: p = 16, FP32)")
    ap.add_argument("--profile", action="store_true",
                    help="ncu target: one warm-up evaluation and one evaluation of the workload, nothing else")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1201_5430_gb300 import LHV
    if args.workload == "filaments":
        r = vfm_ring(torch, LHV)
        if rank == 0:
            print(json.dumps({"metric": METRIC + " (vortex filaments)", "value": r["evals_per_s"] * world,
                              "unit": UNIT, "n_gpus": world, "steps": 3, "warmup": 1,
                              "ms_per_step": r["ms_per_evaluation"], "higher_is_better": True, "scaling": "weak",
                              "dtype": "f32+tf32x3", "data": "synthetic",
                              "config": {"workload": "vfm_ring", "n": r["n"], "p": r["p"]}, "details": r}),
                  flush=True)
    elif args.workload == "leapfrog_learned":
        run_learned_trajectory(args, torch, LHV, rank)
    elif args.workload == "blobs64":
        run_blobs64(args, torch, LHV, local, world, rank, dist)
    elif args.workload == "offset_rings":
        run_offset_rings(args, torch, LHV, local, world, rank, dist)
    else:
        side = torch.cuda.Stream()  # a non-default stream: the graph arm captures on it
        with torch.cuda.stream(side):
            run_single(args, torch, LHV, local, world, rank, dist)


if __name__ == "__main__":
    main()
