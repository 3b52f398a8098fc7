"""The plain FP64 Lamb-Helmholtz FMM ("O2"), following Sec. 4 stage by stage.

Test infrastructure (see ``oracle/__init__``).

Stages (the FMM-run rows of the table in Sec. 4):
  1. S-expansions at the leaves: Eq. eve4 about each leaf centre (Sec. 4.3.2).
  2. Upward pass: M2M by (S|S) (Eq. mr3), then the S conversion (Eq. drt11),
     with t = parent centre - child centre (Eq. bas1), summed over the children.
  3. Downward pass, level 2 .. L: M2L by (S|R) from every box of the
     interaction list, then the R conversion (Eq. drt10), t = target - source;
     plus, below level 2, L2L by (R|R) from the parent, then Eq. drt10,
     t = child - parent.
  4. Evaluation of the local expansions at the leaf elements: v (Eq. evf3),
     grad v and s (Eqs. evf4-evf6).
  5. Local summation over the colleague leaves (Eq. fmm1, sparse part) with the
     smoothed kernel of Eqs. 2 and vem1, j != i.
One translation is converted at a time, as the paper's scheme does.
Translations use dense complex matrices; no rotation-based factorisation.
"""
import numpy as np

from .direct import pair_terms
from .expansions import l2p, p2m_method2
from .operators import convert_R, convert_S, empty, flatten, resize, translation_matrix, unflatten
from .tree import build_tree

__all__ = ["fmm", "FMMResult"]


class FMMResult:
    pass


class _Ops:
    """Memoised dense translation matrices, keyed by (kind, level, integer offset, size)."""

    def __init__(self):
        self.cache = {}

    def apply(self, kind, key, t, c, p_out):
        """Translate c (c.shape[0] terms) and keep p_out terms.  The square map at
        max(p_in, p_out) restricted to n' < p_out, n < p_in is the rectangular map."""
        pm = max(c.shape[0], p_out)
        T = self.cache.get((kind, pm) + key)
        if T is None:
            T = translation_matrix(kind, t, pm)
            self.cache[(kind, pm) + key] = T
        return resize(unflatten(T @ flatten(resize(c, pm)), pm), p_out)


def fmm(x, w, p, leaf_max=64, a=0.0, eps=1e-6, tree=None, far=True, near=True, level_p=None):
    """v, grad v ([i, l, k] = d_l v_k) and s at every element, in input order.

    x, w: (N, 3) FP32 (or any float) arrays; they are widened to FP64.
    level_p: optional truncation number per level (entry l for level l; 0 or a
    missing entry means p).  The expansions of level l then carry level_p[l]
    terms; every translation result is truncated to its level's p before its
    conversion, as in the uniform case."""
    x32 = np.asarray(x, dtype=np.float32).reshape(-1, 3)
    x = x32.astype(np.float64)
    w = np.asarray(w, dtype=np.float32).reshape(-1, 3).astype(np.float64)
    if tree is None:
        tree = build_tree(x32, leaf_max, a, eps)
    n = x.shape[0]
    xs, ws = x[tree.perm], w[tree.perm]
    L = tree.L
    ops = _Ops()
    pl = [int(level_p[l]) if level_p is not None and l < len(level_p) and level_p[l] > 0 else int(p)
          for l in range(L + 1)]
    res = FMMResult()
    res.level_p = pl
    res.tree = tree
    res.multipole = [None] * (L + 1)
    res.local = [None] * (L + 1)

    v_far = np.zeros((n, 3))
    u_far = np.zeros((n, 3, 3))
    if far and L >= 2:
        # 1. S-expansions at the leaves (Eq. eve4)
        lv = tree.levels[L]
        nb = lv["keys"].shape[0]
        res.multipole[L] = [p2m_method2(xs[lv["begin"][b]:lv["end"][b]], ws[lv["begin"][b]:lv["end"][b]],
                                        tree.centre(L, b), pl[L]) for b in range(nb)]
        # 2. upward pass: M2M + S conversion
        for lev in range(L - 1, 1, -1):
            d = tree.levels[lev]
            out = []
            for b in range(d["keys"].shape[0]):
                phi, chi = empty(pl[lev]), empty(pl[lev])
                cb = tree.centre(lev, b)
                for ch in d["children"][b]:
                    t = cb - tree.centre(lev + 1, ch)
                    key = (lev, tuple(2 * d["coords"][b] - tree.levels[lev + 1]["coords"][ch]))
                    mp, mc = res.multipole[lev + 1][ch]
                    ph = ops.apply("SS", key, t, mp, pl[lev])
                    cc = ops.apply("SS", key, t, mc, pl[lev])
                    ph, cc = convert_S(ph, cc, t)
                    phi += ph
                    chi += cc
                out.append((phi, chi))
            res.multipole[lev] = out
        # 3. downward pass: M2L + R conversion, L2L + R conversion
        for lev in range(2, L + 1):
            d = tree.levels[lev]
            out = []
            for b in range(d["keys"].shape[0]):
                phi, chi = empty(pl[lev]), empty(pl[lev])
                cb = tree.centre(lev, b)
                if lev > 2:
                    par = d["parent"][b]
                    t = cb - tree.centre(lev - 1, par)
                    key = (lev, tuple(d["coords"][b] - 2 * tree.levels[lev - 1]["coords"][par]))
                    lp, lc = res.local[lev - 1][par]
                    ph = ops.apply("RR", key, t, lp, pl[lev])
                    cc = ops.apply("RR", key, t, lc, pl[lev])
                    ph, cc = convert_R(ph, cc, t)
                    phi += ph
                    chi += cc
                for s in d["il"][b]:
                    t = cb - tree.centre(lev, s)
                    key = (lev, tuple(d["coords"][b] - d["coords"][s]))
                    mp, mc = res.multipole[lev][s]
                    ph = ops.apply("SR", key, t, mp, pl[lev])
                    cc = ops.apply("SR", key, t, mc, pl[lev])
                    ph, cc = convert_R(ph, cc, t)
                    phi += ph
                    chi += cc
                out.append((phi, chi))
            res.local[lev] = out
        # 4. evaluation of the local expansions at the leaf elements
        lv = tree.levels[L]
        for b in range(lv["keys"].shape[0]):
            s0, s1 = lv["begin"][b], lv["end"][b]
            phi, chi = res.local[L][b]
            vv, uu, _ = l2p(phi, chi, xs[s0:s1] - tree.centre(L, b), ws[s0:s1])
            v_far[s0:s1] = vv
            u_far[s0:s1] = uu

    v_near = np.zeros((n, 3))
    u_near = np.zeros((n, 3, 3))
    if near and n > 0:
        # 5. local summation over the colleague leaves, j != i
        lv = tree.levels[L]
        for b in range(lv["keys"].shape[0]):
            t0, t1 = lv["begin"][b], lv["end"][b]
            src = np.concatenate([np.arange(lv["begin"][c], lv["end"][c]) for c in lv["colleagues"][b]])
            tgt = np.arange(t0, t1)
            d = xs[tgt][:, None, :] - xs[src][None, :, :]
            same = tgt[:, None] == src[None, :]
            d = np.where(same[..., None], 1.0, d)
            vv, uu = pair_terms(d, np.broadcast_to(ws[src][None], d.shape), a)
            v_near[t0:t1] = np.where(same[..., None], 0.0, vv).sum(axis=1)
            u_near[t0:t1] = np.where(same[..., None, None], 0.0, uu).sum(axis=1)

    v_s = v_far + v_near
    u_s = u_far + u_near
    s_s = np.einsum("il,ilk->ik", ws, u_s)
    inv = np.empty_like(tree.perm)
    inv[tree.perm] = np.arange(n)
    res.v, res.grad, res.s = v_s[inv], u_s[inv], s_s[inv]
    res.v_far, res.v_near = v_far[inv], v_near[inv]
    res.s_far = np.einsum("il,ilk->ik", ws, u_far)[inv]
    res.s_near = np.einsum("il,ilk->ik", ws, u_near)[inv]
    return res
