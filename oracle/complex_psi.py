"""One complex FMM for Psi = phi + i chi (Sec. 4.2, Eq. chf1), FP64.

Test infrastructure (see ``oracle/__init__``).

Sec. 4.2 proposes to carry the two real harmonic potentials of Eq. 4 as one complex
harmonic function Psi = phi + i chi, so that each translation is one complex
translation of Psi instead of two real ones, "with the only difference in the
conversion operators".  Coefficient-wise Psi_n^m = phi_n^m + i chi_n^m (both real
functions: c_n^{-m} = (-1)^m conj(c_n^m)), so the translation maps of Eq. mr3 act on
Psi directly (they are complex-linear), and the real potentials come back from Psi by

  phi_n^m = (Psi_n^m + (-1)^m conj(Psi_n^{-m})) / 2,
  chi_n^m = (Psi_n^m - (-1)^m conj(Psi_n^{-m})) / (2 i),

which the conversions of Eqs. drt10 / drt11 need (they couple phi and chi).  The
stages are those of ``fmm`` (O2): P2M (Eq. eve4) gives phi and chi, combined into Psi;
M2M by (S|S) on Psi, then the S conversion; M2L by (S|R) and L2L by (R|R) on Psi, then
the R conversion; L2P of phi and chi split from Psi (Eqs. evf3, evf6); the near field
as in O1.  Same tree and lists.
"""
import numpy as np

from .direct import pair_terms
from .expansions import l2p, p2m_method2
from .operators import convert_R, convert_S, empty, flatten, resize, translation_matrix, unflatten
from .tree import build_tree

__all__ = ["psi_of", "split_psi", "fmm_psi"]


def psi_of(phi, chi):
    """Eq. chf1, coefficient-wise."""
    return phi + 1j * chi


def split_psi(psi):
    """(phi, chi) of Psi = phi + i chi for real harmonic phi, chi (full-m arrays)."""
    p = psi.shape[-2]
    m = np.arange(-(p - 1), p)
    sign = np.where(m % 2 == 0, 1.0, -1.0)
    mirror = np.conj(psi[..., ::-1]) * sign        # (-1)^m conj(Psi_n^{-m}) at (n, m)
    return 0.5 * (psi + mirror), (psi - mirror) / 2j


def _translate(cache, kind, key, t, c, p):
    T = cache.get((kind, p) + key)
    if T is None:
        T = translation_matrix(kind, t, p)
        cache[(kind, p) + key] = T
    return unflatten(T @ flatten(resize(c, p)), p)


def fmm_psi(x, w, p, leaf_max=64, a=0.0, eps=1e-6, tree=None):
    """v, grad v and s at every element (input order) by one complex FMM of Psi."""
    x32 = np.asarray(x, dtype=np.float32).reshape(-1, 3)
    xd = x32.astype(np.float64)
    wd = np.asarray(w, dtype=np.float32).reshape(-1, 3).astype(np.float64)
    if tree is None:
        tree = build_tree(x32, leaf_max, a, eps)
    n = xd.shape[0]
    xs, ws = xd[tree.perm], wd[tree.perm]
    L = tree.L
    cache = {}
    mp = [None] * (L + 1)
    lc = [None] * (L + 1)
    v = np.zeros((n, 3))
    u = np.zeros((n, 3, 3))
    if L >= 2:
        lv = tree.levels[L]
        mp[L] = [psi_of(*p2m_method2(xs[lv["begin"][b]:lv["end"][b]], ws[lv["begin"][b]:lv["end"][b]],
                                     tree.centre(L, b), p)) for b in range(lv["keys"].shape[0])]
        for lev in range(L - 1, 1, -1):   # M2M: one complex (S|S) translation, then Eq. drt11
            d = tree.levels[lev]
            out = []
            for b in range(d["keys"].shape[0]):
                acc = empty(p)
                cb = tree.centre(lev, b)
                for ch in d["children"][b]:
                    t = cb - tree.centre(lev + 1, ch)
                    key = (lev, tuple(2 * d["coords"][b] - tree.levels[lev + 1]["coords"][ch]))
                    ph, cc = convert_S(*split_psi(_translate(cache, "SS", key, t, mp[lev + 1][ch], p)), t)
                    acc += psi_of(ph, cc)
                out.append(acc)
            mp[lev] = out
        for lev in range(2, L + 1):       # L2L and M2L on Psi, then Eq. drt10
            d = tree.levels[lev]
            out = []
            for b in range(d["keys"].shape[0]):
                acc = empty(p)
                cb = tree.centre(lev, b)
                if lev > 2:
                    par = d["parent"][b]
                    t = cb - tree.centre(lev - 1, par)
                    key = (lev, tuple(d["coords"][b] - 2 * tree.levels[lev - 1]["coords"][par]))
                    acc += psi_of(*convert_R(*split_psi(_translate(cache, "RR", key, t, lc[lev - 1][par], p)), t))
                for s in d["il"][b]:
                    t = cb - tree.centre(lev, s)
                    key = (lev, tuple(d["coords"][b] - d["coords"][s]))
                    acc += psi_of(*convert_R(*split_psi(_translate(cache, "SR", key, t, mp[lev][s], p)), t))
                out.append(acc)
            lc[lev] = out
        for b in range(lv["keys"].shape[0]):
            s0, s1 = lv["begin"][b], lv["end"][b]
            ph, cc = split_psi(lc[L][b])
            vv, uu, _ = l2p(ph, cc, xs[s0:s1] - tree.centre(L, b), ws[s0:s1])
            v[s0:s1] += vv
            u[s0:s1] += uu
    lv = tree.levels[L]
    for b in range(lv["keys"].shape[0]):
        t0, t1 = lv["begin"][b], lv["end"][b]
        src = np.concatenate([np.arange(lv["begin"][c], lv["end"][c]) for c in lv["colleagues"][b]])
        tgt = np.arange(t0, t1)
        dd = xs[tgt][:, None, :] - xs[src][None, :, :]
        same = tgt[:, None] == src[None, :]
        dd = np.where(same[..., None], 1.0, dd)
        vv, uu = pair_terms(dd, np.broadcast_to(ws[src][None], dd.shape), a)
        v[t0:t1] += np.where(same[..., None], 0.0, vv).sum(axis=1)
        u[t0:t1] += np.where(same[..., None, None], 0.0, uu).sum(axis=1)
    s_ = np.einsum("il,ilk->ik", ws, u)
    inv = np.empty_like(tree.perm)
    inv[tree.perm] = np.arange(n)

    class R:
        pass
    r = R()
    r.tree, r.v, r.grad, r.s = tree, v[inv], u[inv], s_[inv]
    r.multipole, r.local = mp, lc
    return r
