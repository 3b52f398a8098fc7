"""Training of the learned form's selector network.

The data are error-versus-p curves that the method itself produces: for each
training system and each octree level l = 2..L, the FMM is run with p at level l
and p_ref = 20 at every other level, and E_l(p) = |v - v_ref| / |v_ref| (relative
L2 over all elements) is recorded against the run with p_ref everywhere.
The errors of different levels add about in quadrature, so for a target eps the
labels are the schedule (p_2 .. p_L) of least M2L cost with sum_l E_l(p_l)^2 <=
eps^2: cost_l(p) = (M2L pairs of level l) x (measured time per pair at p in the
context's arithmetic, where p a multiple of 4 runs on the tensor cores under
TF32x3), minimised level by level for a Lagrange multiplier found by bisection.
Each schedule is then run once and, if its measured error exceeds eps, the
target is tightened until it does not.  The leaf cap label of a system is the
fastest of 16, 32, 64, 128 at fixed p when the caps give different trees, else
64.  One feature row per (system, level, eps) comes from
``lhv_selector_features``; the network is trained by Adam through
``lhv_mlp_loss_grad`` / ``lhv_mlp_adam``.

Run ``python -m paper_1201_5430_gb300.selector`` on a GPU to regenerate
``selector_weights.npz`` (bfloat16 weights as uint16 bit patterns, FP32 biases).
"""
import json
import math
import os
import time

import numpy as np
import torch

from . import _lib as L
from .api import LHV, mlp_adam, mlp_loss_grad

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "selector_weights.npz")
P_VALUES = list(range(4, 21))
LEAF_CAPS = [16, 32, 64, 128]
EPS_GRID = [1e-3, 3e-4, 1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7]
P_REF = 20


def training_systems():
    """(name, x, w, a) of the training set: rings, ring pairs, cubes and blob
    clouds of several sizes, seeds disjoint from the benchmark workloads."""
    import workloads as W
    out = []
    for n, seed in ((32768, 11), (65536, 12), (131072, 13), (262144, 14)):
        x, w = W.ring(n, seed)
        out.append((f"ring{n}_s{seed}", x, w, W.RING_CORE_A))
    for kind, seed in (("leapfrog", 15), ("offset", 16)):
        x, w = W.ring_pair(65536, seed, kind)
        out.append((f"{kind}131072_s{seed}", x, w, W.RING_CORE_A))
    for n, seed in ((16384, 21), (65536, 22), (262144, 23)):
        x, w = W.cube(n, seed)
        out.append((f"cube{n}_s{seed}", x, w, 0.01))
    for k, (x, w) in enumerate(W.blob_systems(nsys=3, seed=31, n_lo=2e4, n_hi=1.5e5)):
        out.append((f"blobs{x.shape[0]}_{k}", x, w, 0.01))
    return out


def _f4(a):
    import workloads as W
    return torch.from_numpy(W.to_f4(a)).cuda()


def _timed_eval(ctx, x4, w4, reps=3):
    ctx.evaluate_velocity_stretching(x4, w4)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        ctx.evaluate_velocity_stretching(x4, w4)
    torch.cuda.synchronize()
    return (time.perf_counter() - t) / reps


def error_curves(ctx, x4, w4):
    """E[l][p] for the levels 2..L of the tree of x4 (context at p = P_REF)."""
    ctx.set_level_p(None)
    v_ref, _ = ctx.evaluate_velocity_stretching(x4, w4)
    v_ref = v_ref[:, :3].double().cpu().numpy()
    Lv = ctx.stats()["leaf_level"]
    nref = np.linalg.norm(v_ref)
    curves = {}
    for lev in range(2, Lv + 1):
        row = {}
        for p in P_VALUES:
            sched = [P_REF] * (Lv + 1)
            sched[lev] = p
            ctx.set_level_p(sched)
            v, _ = ctx.evaluate_velocity_stretching(x4, w4)
            row[p] = float(np.linalg.norm(v[:, :3].double().cpu().numpy() - v_ref) / nref)
        curves[lev] = row
    ctx.set_level_p(None)
    return Lv, curves


def pair_cost(ctx, x4, w4):
    """Measured M2L product time per box pair for every p (uniform runs of one system)."""
    ctx.set_timing(True)
    out = {}
    for p in P_VALUES:
        ctx.set_level_p([p] * 22)
        ctx.evaluate_velocity_stretching(x4, w4)
        ctx.reset_stats()
        for _ in range(3):
            ctx.evaluate_velocity_stretching(x4, w4)
        st = ctx.stats()
        out[p] = st["stage_ms"]["m2l_products"] / 3 / max(st["m2l_pairs"], 1)
    ctx.set_timing(False)
    ctx.set_level_p(None)
    return out


def optimal_schedule(curves, pairs, cost, eps):
    """Least-cost (p_2 .. p_L) with sum_l E_l(p_l)^2 <= eps^2 (Lagrangian, bisection on the multiplier)."""
    levels = sorted(curves)

    def pick(lam):
        sched, err2 = {}, 0.0
        for lev in levels:
            best = min(P_VALUES, key=lambda p: pairs[lev] * cost[p] + lam * curves[lev][p] ** 2)
            sched[lev] = best
            err2 += curves[lev][best] ** 2
        return sched, err2

    lo, hi = 0.0, 1.0
    while pick(hi)[1] > eps * eps and hi < 1e40:
        hi *= 10.0
    if pick(hi)[1] > eps * eps:
        return {lev: P_VALUES[-1] for lev in levels}
    for _ in range(80):
        mid = math.sqrt(lo * hi) if lo > 0 else hi / 1e6
        if pick(mid)[1] <= eps * eps:
            hi = mid
        else:
            lo = mid
    return pick(hi)[0]


def run_error(ctx, x4, w4, v_ref, sched, Lv):
    full = [P_REF] * (Lv + 1)
    for lev, p in sched.items():
        full[lev] = p
    ctx.set_level_p(full)
    v, _ = ctx.evaluate_velocity_stretching(x4, w4)
    ctx.set_level_p(None)
    return float(np.linalg.norm(v[:, :3].double().cpu().numpy() - v_ref) / np.linalg.norm(v_ref))


def generate(precisions=("fp32", "tf32x3"), log=print):
    """Feature rows X, labels yp (p - 4) and yl (leaf cap index, -1 if none), and a record."""
    import workloads as W
    rows, yps, yls, record = [], [], [], []
    systems = training_systems()
    ctxs = {}
    for prec in precisions:
        # time per M2L pair against p, on one ring of the training set
        xr, wr = W.ring(262144, 14)
        c0 = LHV(p=P_REF, leaf_max=64, core_a=W.RING_CORE_A, precision=prec)
        cost = pair_cost(c0, _f4(xr), _f4(wr))
        c0.close()
        log(f"{prec} M2L ns per pair: " + ", ".join(f"{p}:{cost[p] * 1e6:.1f}" for p in P_VALUES))
        for name, x, w, a in systems:
            key = (prec, a)
            if key not in ctxs:
                ctxs[key] = LHV(p=P_REF, leaf_max=64, core_a=a, precision=prec)
            ctx = ctxs[key]
            x4, w4 = _f4(x), _f4(w)
            t0 = time.time()
            Lv, curves = error_curves(ctx, x4, w4)
            ctx.set_level_p(None)
            v_ref, _ = ctx.evaluate_velocity_stretching(x4, w4)
            v_ref = v_ref[:, :3].double().cpu().numpy()
            nbox = ctx.stats()["nbox"]
            F0 = ctx.selector_features(x4, w4, eps=1e-6).cpu().numpy()
            pairs = {lev: float(F0[lev - 2, 7] * 189.0 * nbox[lev]) for lev in range(2, Lv + 1)}
            # leaf cap: the fastest at fixed p = 12 when the caps change the tree, else 64
            times, depths = [], []
            for cap in LEAF_CAPS:
                c2 = LHV(p=12, leaf_max=cap, core_a=a, precision=prec)
                times.append(_timed_eval(c2, x4, w4))
                depths.append(c2.stats()["leaf_level"])
                c2.close()
            leaf = int(np.argmin(times)) if len(set(depths)) > 1 else LEAF_CAPS.index(64)
            scheds = {}
            for eps in EPS_GRID:
                target = eps
                for _ in range(4):
                    sched = optimal_schedule(curves, pairs, cost, target)
                    err = run_error(ctx, x4, w4, v_ref, sched, Lv)
                    if err <= eps or all(p == P_VALUES[-1] for p in sched.values()):
                        break
                    target *= 0.9 * eps / err
                scheds[eps] = (sched, err)
                F = ctx.selector_features(x4, w4, eps=eps).cpu().numpy()
                for lev in range(2, Lv + 1):
                    rows.append(F[lev - 2])
                    yps.append(sched[lev] - 4)
                    yls.append(leaf if lev == Lv else -1)
            record.append({"system": name, "precision": prec, "n": int(x.shape[0]), "a": a, "L": Lv,
                           "curves": {str(k): v for k, v in curves.items()}, "pairs": pairs,
                           "leaf_times_s": times, "leaf_depths": depths, "leaf_label": LEAF_CAPS[leaf],
                           "schedules": {str(e): [[int(k), int(v)] for k, v in s.items()] + [err]
                                         for e, (s, err) in scheds.items()}})
            s6, e6 = scheds[1e-6]
            log(f"{prec} {name}: L={Lv} leaf={LEAF_CAPS[leaf]} schedule@1e-6={[s6[l] for l in sorted(s6)]} "
                f"err {e6:.2e} ({time.time() - t0:.1f} s)")
    for c in ctxs.values():
        c.close()
    return (np.array(rows, np.float32), np.array(yps, np.int32), np.array(yls, np.int32), record)


def _init(seed):
    """He-uniform weights, zero biases (FP32)."""
    rng = np.random.default_rng(seed)
    sizes = [(64, 12), (64, 64), (64, 64), (21, 64)]
    ws = [rng.uniform(-1, 1, (o, i)) * math.sqrt(6.0 / i) for o, i in sizes]
    return np.concatenate([w.ravel() for w in ws]).astype(np.float32), np.zeros(L.MLP_NB, np.float32)


def fit(X, yp, yl, steps=4000, lr=2e-3, seed=0, log=print):
    """Adam on the GPU kernels; returns (W bfloat16 tensor, b float32 tensor, final loss)."""
    w0, b0 = _init(seed)
    dev = torch.device("cuda")
    Xd = torch.from_numpy(X).to(dev)
    YP = torch.from_numpy(yp).to(dev)
    YL = torch.from_numpy(yl).to(dev)
    W32 = torch.from_numpy(w0).to(dev)
    B = torch.from_numpy(b0).to(dev)
    W = W32.to(torch.bfloat16)
    mW, vW, mb, vb = (torch.zeros_like(W32), torch.zeros_like(W32), torch.zeros_like(B), torch.zeros_like(B))
    loss = None
    for t in range(1, steps + 1):
        loss, gW, gb = mlp_loss_grad(Xd, YP, YL, W, B)
        mlp_adam(W32, W, gW, mW, vW, B, gb, mb, vb, t, lr)
        if t % 500 == 0:
            log(f"step {t}: loss {float(loss):.4f}")
    loss, _, _ = mlp_loss_grad(Xd, YP, YL, W, B)
    return W, B, float(loss)


def save(W, B, meta, path=WEIGHTS):
    bits = W.detach().cpu().contiguous().view(torch.int16).numpy().view(np.uint16)
    np.savez(path, W=bits, b=B.detach().cpu().numpy().astype(np.float32), meta=json.dumps(meta))


def load(path=WEIGHTS):
    """(W bfloat16 tensor, b float32 tensor, meta dict) of a saved network."""
    z = np.load(path)
    W = torch.from_numpy(z["W"].astype(np.uint16).view(np.int16).copy()).view(torch.bfloat16)
    return W, torch.from_numpy(z["b"].copy()), json.loads(str(z["meta"]))


def main():
    t0 = time.time()
    X, yp, yl, record = generate()
    W, B, loss = fit(X, yp, yl)
    from .api import mlp_forward
    Z = mlp_forward(torch.from_numpy(X).cuda(), W, B).cpu().numpy()
    acc_p = float(np.mean(np.argmax(Z[:, :17], axis=1) == yp))
    within1 = float(np.mean(np.abs(np.argmax(Z[:, :17], axis=1) - yp) <= 1))
    meta = {"rows": int(X.shape[0]), "loss": loss, "train_acc_p": acc_p, "train_within1_p": within1,
            "eps_grid": EPS_GRID, "p_ref": P_REF, "systems": record, "seconds": time.time() - t0}

    save(W, B, meta)
    print(json.dumps({k: v for k, v in meta.items() if k != "systems"}))


if __name__ == "__main__":
    main()
