"""Vortex filament elements (VFM, Sec. 5.3 and App. B), FP64.

Test infrastructure (see ``oracle/__init__``).

A filament is a polyline of nodes; segment k runs from node k to the next node (the first
one again for a closed filament) with constant circulation Gamma_k.  Its velocity at y is
the Biot-Savart line integral of Eq. dis1 in closed form, Eq. dis2,

  v_k(y) = Gamma_k / (4 pi) (r1 x r2) / (r1 r2 + r1 . r2) (1/r1 + 1/r2),  rj = y - x_k^(j),

and v_k(y) = 0 for y on the segment (applied by index: a node gets nothing from the two
segments it ends).  The receivers are the nodes (Sec. 5.3: the end points propagate with the
fluid, so stretching needs no extra term).

FMM ("O2f"): the octree of the nodes; segment k belongs to the leaf of node k.  Its
S-expansion is that of Eq. eve4 with (Gamma/8 pi) l in place of w and g~ of Eq. vf6, the
Gauss-Legendre quadrature of R_n^{-m} along the segment with N_q = [(p-1)/2] + 1 points
(Eq. vf7), exact for every n < p; i.e. N_q point vortices of strength Gamma l w_j / (8 pi) at
x_c + l xi_j / 2 (x_c the segment's centre, Eq. vf2), expanded about the leaf centre.
Translations as in O2.  L2P gives v at the nodes (Eq. evf3); the near field is Eq. dis2 over
the segments of the colleague leaves.  Valid while segments are short against the leaf
side (their quadrature points then stay close to their leaf).
"""
import math

import numpy as np
from numpy.polynomial.legendre import leggauss

from .expansions import l2p, p2m_method2
from .fmm import _Ops
from .operators import convert_R, convert_S, empty
from .tree import build_tree

__all__ = ["segments_of", "segment_velocity", "direct_filaments", "n_quad", "p2m_segment", "fmm_filaments"]


def segments_of(n_nodes, offsets, closed):
    """(start, end) node indices of every segment: filament f owns nodes
    offsets[f] .. offsets[f+1]-1; a closed filament also joins its last node to its first."""
    start, end = [], []
    for f in range(len(offsets) - 1):
        a, b = int(offsets[f]), int(offsets[f + 1])
        for k in range(a, b - 1):
            start.append(k)
            end.append(k + 1)
        if closed[f] and b - a >= 2:
            start.append(b - 1)
            end.append(a)
    return np.asarray(start, dtype=np.int64), np.asarray(end, dtype=np.int64)


def segment_velocity(y, x1, x2, gamma):
    """Eq. dis2 at points y (M, 3) from segments x1 -> x2 (K, 3) with circulations gamma (K,):
    returns (M, K, 3).  Points on a segment's line (r1 x r2 = 0) get 0."""
    r1 = np.asarray(y, np.float64)[:, None, :] - np.asarray(x1, np.float64)[None, :, :]
    r2 = np.asarray(y, np.float64)[:, None, :] - np.asarray(x2, np.float64)[None, :, :]
    a = np.linalg.norm(r1, axis=-1)
    b = np.linalg.norm(r2, axis=-1)
    c = np.cross(r1, r2)
    den = a * b + (r1 * r2).sum(axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.asarray(gamma, np.float64)[None, :] / (4.0 * math.pi) * (1.0 / a + 1.0 / b) / den
    f = np.where(np.isfinite(f) & ((c * c).sum(axis=-1) > 0), f, 0.0)
    return f[..., None] * c


def direct_filaments(x, gamma, offsets, closed, targets=None):
    """O1f: v at the nodes `targets` (all when None): the sum of Eq. dis2 over every segment
    that does not end at the node."""
    x = np.asarray(x, dtype=np.float32).reshape(-1, 3).astype(np.float64)
    s0, s1 = segments_of(x.shape[0], offsets, closed)
    g = np.asarray(gamma, dtype=np.float32).astype(np.float64)[s0]
    idx = np.arange(x.shape[0]) if targets is None else np.asarray(targets)
    v = np.zeros((idx.shape[0], 3))
    for k0 in range(0, idx.shape[0], 256):
        t = idx[k0:k0 + 256]
        vv = segment_velocity(x[t], x[s0], x[s1], g)
        own = (t[:, None] == s0[None, :]) | (t[:, None] == s1[None, :])
        v[k0:k0 + 256] = np.where(own[..., None], 0.0, vv).sum(axis=1)
    return v


def n_quad(p):
    """Eq. vf7."""
    return (p - 1) // 2 + 1


def p2m_segment(x1, x2, gamma, centre, p, nq=None):
    """S-expansion (phi, chi) of segments x1 -> x2 about `centre`: Eq. eve4 with
    (Gamma / 8 pi) l and the quadrature of Eq. vf6 (nq points, Eq. vf7 by default)."""
    x1 = np.asarray(x1, np.float64).reshape(-1, 3)
    x2 = np.asarray(x2, np.float64).reshape(-1, 3)
    if x1.shape[0] == 0:
        return empty(p), empty(p)
    xi, wq = leggauss(nq or n_quad(p))
    l = x2 - x1
    xc = 0.5 * (x1 + x2)
    pts = (xc[:, None, :] + 0.5 * l[:, None, :] * xi[None, :, None]).reshape(-1, 3)
    stren = (np.asarray(gamma, np.float64)[:, None, None] / (8.0 * math.pi) * l[:, None, :]
             * wq[None, :, None]).reshape(-1, 3)
    return p2m_method2(pts, stren, centre, p)


def fmm_filaments(x, gamma, offsets, closed, p, leaf_max=64, tree=None):
    """O2f: v at every node (input order)."""
    x32 = np.asarray(x, dtype=np.float32).reshape(-1, 3)
    xd = x32.astype(np.float64)
    gd = np.asarray(gamma, dtype=np.float32).astype(np.float64)
    if tree is None:
        tree = build_tree(x32, leaf_max, 0.0, 1e-6)
    n = xd.shape[0]
    s0, s1 = segments_of(n, offsets, closed)
    owner_rank = np.empty(n, dtype=np.int64)
    owner_rank[tree.perm] = np.arange(n)              # sorted position of each node
    L = tree.L
    ops = _Ops()
    mp = [None] * (L + 1)
    lc = [None] * (L + 1)
    v = np.zeros((n, 3))
    lv = tree.levels[L]
    leaf_of_node = np.searchsorted(lv["begin"], owner_rank, side="right") - 1
    seg_leaf = leaf_of_node[s0]                        # segment k sits in the leaf of its first node
    if L >= 2:
        mp[L] = [p2m_segment(xd[s0[seg_leaf == b]], xd[s1[seg_leaf == b]], gd[s0[seg_leaf == b]],
                             tree.centre(L, b), p) for b in range(lv["keys"].shape[0])]
        for lev in range(L - 1, 1, -1):
            d = tree.levels[lev]
            out = []
            for b in range(d["keys"].shape[0]):
                phi, chi = empty(p), empty(p)
                cb = tree.centre(lev, b)
                for ch in d["children"][b]:
                    t = cb - tree.centre(lev + 1, ch)
                    key = (lev, tuple(2 * d["coords"][b] - tree.levels[lev + 1]["coords"][ch]))
                    ph, cc = convert_S(ops.apply("SS", key, t, mp[lev + 1][ch][0], p),
                                       ops.apply("SS", key, t, mp[lev + 1][ch][1], p), t)
                    phi += ph
                    chi += cc
                out.append((phi, chi))
            mp[lev] = out
        for lev in range(2, L + 1):
            d = tree.levels[lev]
            out = []
            for b in range(d["keys"].shape[0]):
                phi, chi = empty(p), empty(p)
                cb = tree.centre(lev, b)
                if lev > 2:
                    par = d["parent"][b]
                    t = cb - tree.centre(lev - 1, par)
                    key = (lev, tuple(d["coords"][b] - 2 * tree.levels[lev - 1]["coords"][par]))
                    ph, cc = convert_R(ops.apply("RR", key, t, lc[lev - 1][par][0], p),
                                       ops.apply("RR", key, t, lc[lev - 1][par][1], p), t)
                    phi += ph
                    chi += cc
                for s in d["il"][b]:
                    t = cb - tree.centre(lev, s)
                    key = (lev, tuple(d["coords"][b] - d["coords"][s]))
                    ph, cc = convert_R(ops.apply("SR", key, t, mp[lev][s][0], p),
                                       ops.apply("SR", key, t, mp[lev][s][1], p), t)
                    phi += ph
                    chi += cc
                out.append((phi, chi))
            lc[lev] = out
        xs = xd[tree.perm]
        for b in range(lv["keys"].shape[0]):
            e0, e1 = lv["begin"][b], lv["end"][b]
            vv, _, _ = l2p(lc[L][b][0], lc[L][b][1], xs[e0:e1] - tree.centre(L, b), np.zeros((e1 - e0, 3)))
            v[tree.perm[e0:e1]] += vv
    # near field: the segments of the colleague leaves
    for b in range(lv["keys"].shape[0]):
        nodes = tree.perm[lv["begin"][b]:lv["end"][b]]
        segs = np.flatnonzero(np.isin(seg_leaf, lv["colleagues"][b]))
        if segs.size == 0 or nodes.size == 0:
            continue
        vv = segment_velocity(xd[nodes], xd[s0[segs]], xd[s1[segs]], gd[s0[segs]])
        own = (nodes[:, None] == s0[segs][None, :]) | (nodes[:, None] == s1[segs][None, :])
        v[nodes] += np.where(own[..., None], 0.0, vv).sum(axis=1)

    class R:
        pass
    r = R()
    r.v, r.tree, r.seg_leaf = v, tree, seg_leaf
    return r
