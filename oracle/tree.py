"""Morton keys, uniform octree and the FMM lists, written out plainly.

Test infrastructure (see ``oracle/__init__``).

The paper fixes only that the FMM uses an octree with neighbour lists and the
standard 189-box M2L stencil at a depth l_max chosen for speed (Sec. 4 table;
Sec. 5). The construction below is the reading used throughout this repository:

* cube: origin x0 = per-axis minimum of the FP32 positions; side = the smallest
  r_q 2^k >= the largest per-axis extent (k an integer), r_q = r_K (below) rounded up
  to an 8-bit mantissa, so that the box side of one level lies in [r_K, 1.008 r_K);
  without a core (a = 0) the smallest power of two >= the extent; 1 if the extent is 0;
  in a batch of independent systems with a core, every system takes the largest of the
  systems' sides (``batch_side``; origins stay per system), so that the batch's one leaf
  level gives every system leaves of side r_q;
* keys: q = floor((x - x0) * 2^21 / side) in FP64, clamped to [0, 2^21 - 1];
  the key interleaves the 21 bits of (qx, qy, qz) with x in bit 0, y in bit 1,
  z in bit 2 of each triple; elements are stably sorted by key;
* leaf level L = min(L_leaf, L_K): L_leaf is the shallowest level at which no
  box holds more than ``leaf_max`` elements; L_K is the deepest level whose box
  side is >= r_K = x_K a, where 1 - K(x_K a; a) = eps/10 (Eq. vem1), so that
  every pair handled by the far field sees K = 1 within eps/10 (Eq. 2);
* colleagues: the boxes of the same level whose integer coordinates differ by at
  most one per axis (the box itself included);
* interaction list of a box at level >= 2: the children of its parent's
  colleagues that are not its colleagues (at most 189 boxes).
"""
import math

import numpy as np
from scipy.optimize import brentq
from scipy.special import erfc

__all__ = ["cube", "core_unit", "batch_side", "morton_keys", "leaf_level", "core_cutoff", "Tree", "build_tree"]

KEY_BITS = 21


def core_unit(rK):
    """r_K rounded up to an 8-bit mantissa (0 without a core)."""
    if not rK > 0.0:
        return 0.0
    mant, e = math.frexp(rK)                # rK = mant * 2^e, 0.5 <= mant < 1
    return math.ldexp(math.ceil(mant * 256.0) / 256.0, e)


def cube(x, unit=0.0, side=None):
    """Cube origin (FP32 minimum, as float64) and side: the smallest unit * 2^k >= the
    largest extent (k an integer), unit = 1 when 0 (a power of two); ``side`` given: that."""
    x = np.asarray(x, dtype=np.float32).reshape(-1, 3)
    lo = x.min(axis=0).astype(np.float64)
    if side is not None:
        return lo, float(side)
    hi = x.max(axis=0).astype(np.float64)
    extent = float((hi - lo).max())
    if extent <= 0.0:
        return lo, 1.0
    u = unit if unit > 0.0 else 1.0
    k = 0
    while math.ldexp(u, k) < extent:
        k += 1
    while math.ldexp(u, k - 1) >= extent:
        k -= 1
    return lo, math.ldexp(u, k)


def quantise(x, x0, side):
    x = np.asarray(x, dtype=np.float32).reshape(-1, 3).astype(np.float64)
    q = np.floor((x - x0) * (float(1 << KEY_BITS) / side))
    return np.clip(q, 0, (1 << KEY_BITS) - 1).astype(np.uint64)


def interleave(q):
    """Bit interleave of (qx, qy, qz), x in the lowest bit of each triple."""
    key = np.zeros(q.shape[0], dtype=np.uint64)
    for b in range(KEY_BITS):
        for axis in range(3):
            bit = (q[:, axis] >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(3 * b + axis)
    return key


def deinterleave(key):
    key = np.asarray(key, dtype=np.uint64)
    q = np.zeros(key.shape + (3,), dtype=np.int64)
    for b in range(KEY_BITS):
        for axis in range(3):
            q[..., axis] |= (((key >> np.uint64(3 * b + axis)) & np.uint64(1)).astype(np.int64) << b)
    return q


def morton_keys(x, unit=0.0, side=None):
    x0, side = cube(x, unit, side)
    return interleave(quantise(x, x0, side)), x0, side


def core_cutoff(a, eps):
    """r_K = x_K a with 1 - K(x_K a; a) = eps/10, where by Eq. vem1
    1 - K = erfc(x/sqrt 2) + sqrt(2/pi) x exp(-x^2/2) (x = r/a).  0 if a = 0."""
    if a <= 0:
        return 0.0
    target = eps / 10.0

    def g(xx):
        return erfc(xx / math.sqrt(2.0)) + math.sqrt(2.0 / math.pi) * xx * math.exp(-0.5 * xx * xx) - target

    return brentq(g, 0.0, 60.0, xtol=1e-14, rtol=1e-15, maxiter=500) * a


def leaf_level(keys_sorted, leaf_max, side, a, eps):
    """L = min(L_leaf, L_K), both as defined in the module docstring."""
    n = keys_sorted.shape[0]
    L_leaf = KEY_BITS
    for lev in range(KEY_BITS + 1):
        pref = keys_sorted >> np.uint64(3 * (KEY_BITS - lev))
        _, counts = np.unique(pref, return_counts=True)
        if n == 0 or counts.max() <= leaf_max:
            L_leaf = lev
            break
    rK = core_cutoff(a, eps)
    L_K = KEY_BITS
    if rK > 0:
        L_K = 0
        for lev in range(KEY_BITS + 1):
            if side / (1 << lev) >= rK:
                L_K = lev
    return min(L_leaf, L_K)


class Tree:
    """Sorted elements and, per level, boxes with their lists.

    levels[l] has: keys (prefix), coords (n, 3), begin/end (element ranges in
    sorted order), parent (index at level l-1), children (list of index lists),
    colleagues (list of index lists), il (list of index lists; empty for l < 2)."""

    def __init__(self, x, leaf_max, a, eps, L_override=None, side=None):
        x = np.asarray(x, dtype=np.float32).reshape(-1, 3)
        self.n = x.shape[0]
        keys, self.x0, self.side = morton_keys(x, core_unit(core_cutoff(a, eps)), side)
        self.perm = np.argsort(keys, kind="stable")
        self.keys = keys[self.perm]
        self.L = leaf_level(self.keys, leaf_max, self.side, a, eps) if L_override is None else int(L_override)
        self.levels = []
        for lev in range(self.L + 1):
            pref = self.keys >> np.uint64(3 * (KEY_BITS - lev))
            start = np.flatnonzero(np.r_[True, pref[1:] != pref[:-1]]) if self.n else np.zeros(0, np.int64)
            end = np.r_[start[1:], self.n].astype(np.int64)
            bkeys = pref[start]
            coords = deinterleave(bkeys)
            self.levels.append({"keys": bkeys, "coords": coords, "begin": start.astype(np.int64), "end": end})
        for lev in range(self.L + 1):
            d = self.levels[lev]
            lookup = {tuple(c): i for i, c in enumerate(d["coords"])}
            d["lookup"] = lookup
            nb = d["keys"].shape[0]
            d["colleagues"] = []
            for i in range(nb):
                cx, cy, cz = d["coords"][i]
                col = []
                for dx in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dz in (-1, 0, 1):
                            j = lookup.get((cx + dx, cy + dy, cz + dz))
                            if j is not None:
                                col.append(j)
                d["colleagues"].append(sorted(col))
            if lev == 0:
                d["parent"] = np.full(nb, -1, dtype=np.int64)
            else:
                up = self.levels[lev - 1]["lookup"]
                d["parent"] = np.array([up[tuple(c // 2)] for c in d["coords"]], dtype=np.int64)
        for lev in range(self.L + 1):
            d = self.levels[lev]
            nb = d["keys"].shape[0]
            d["children"] = [[] for _ in range(nb)]
            if lev < self.L:
                for j, par in enumerate(self.levels[lev + 1]["parent"]):
                    d["children"][par].append(j)
        for lev in range(self.L + 1):
            d = self.levels[lev]
            nb = d["keys"].shape[0]
            d["il"] = [[] for _ in range(nb)]
            if lev < 2:
                continue
            up = self.levels[lev - 1]
            for i in range(nb):
                mine = set(d["colleagues"][i])
                cand = []
                for pc in up["colleagues"][d["parent"][i]]:
                    for ch in up["children"][pc]:
                        if ch not in mine:
                            cand.append(ch)
                d["il"][i] = sorted(cand)

    def h(self, lev):
        return self.side / (1 << lev)

    def centre(self, lev, i):
        return self.x0 + (self.levels[lev]["coords"][i].astype(np.float64) + 0.5) * self.h(lev)


def build_tree(x, leaf_max=64, a=0.0, eps=1e-6, L_override=None, side=None):
    """``L_override`` forces the leaf level (tests use it to switch the L_K rule off);
    ``side`` the cube side (a system of a batch: ``batch_side``)."""
    return Tree(x, leaf_max, a, eps, L_override, side)


def batch_side(xs, a=0.0, eps=1e-6):
    """The cube side of every system of a batch (positions xs, one array per system): with
    a core the largest of the systems' own sides, else None (each keeps its own)."""
    rK = core_cutoff(a, eps)
    if not rK > 0.0 or len(xs) < 2:
        return None
    return max(cube(x, core_unit(rK))[1] for x in xs)
