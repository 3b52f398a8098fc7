"""The paper's reference case, the scalar harmonic FMM for phi and grad phi, FP64.

Test infrastructure (see ``oracle/__init__``).

Sec. 5.2 times the Lamb-Helmholtz FMM against "a reference case for the scalar
Laplace equation, where the potential or both potential and its gradient should
be computed" (Tables 1-2; the ratio of run times, mean 1.405, is the paper's
central cost claim, Sec. 4.1 Eqs. fmm2-fmm3).  Sources are monopoles of strength
q_j (Sec. 2: a monopole distribution gives the scalar potential):

  phi(x_i)      = sum_{j != i} q_j / |x_i - x_j|                (excluded by index)
  grad phi(x_i) = -sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3

Written with no 1/(4 pi), like Eq. 1.  The singular kernel has no value at r = 0:
distinct elements at the same point contribute nothing to each other.  The FMM ("O2s") takes the stages of the
Sec. 4 table for one potential: S-expansions of the leaves by Eq. rsbf5
(|r - r0|^{-1} = sum R_n^{-m}(-r0) S_n^m(r)), M2M by (S|S), M2L by (S|R), L2L by
(R|R) (Eq. mr3), with no conversion (there is no chi), then the local expansions
evaluated for phi and for its gradient (D_t of Eq. dt3 with t = i_x, i_y, i_z),
plus the direct sum over the colleague leaves.  Same octree and lists as the
vortex FMM (``tree``), dense complex translations.
"""
import numpy as np

from .basis import R_table
from .expansions import eval_R
from .operators import apply_Dt, empty, flatten, resize, translation_matrix, unflatten
from .tree import build_tree

__all__ = ["direct_scalar", "p2m_scalar", "l2p_scalar", "fmm_scalar"]


def direct_scalar(x, q, targets=None):
    """O1s: phi and grad phi at the elements `targets` (all when None) from every
    element j != target (excluded by index), FP64."""
    x = np.asarray(x, dtype=np.float32).reshape(-1, 3).astype(np.float64)
    q = np.asarray(q, dtype=np.float32).reshape(-1).astype(np.float64)
    idx = np.arange(x.shape[0]) if targets is None else np.asarray(targets)
    phi = np.zeros(idx.shape[0])
    grad = np.zeros((idx.shape[0], 3))
    for k0 in range(0, idx.shape[0], 256):
        t = idx[k0:k0 + 256]
        d = x[t][:, None, :] - x[None, :, :]
        r = np.sqrt((d * d).sum(axis=-1))
        same = t[:, None] == np.arange(x.shape[0])[None, :]
        skip = same | (r == 0.0)
        inv = np.where(skip, 0.0, 1.0 / np.where(skip, 1.0, r))
        phi[k0:k0 + 256] = (q[None, :] * inv).sum(axis=1)
        grad[k0:k0 + 256] = -((q[None, :] * inv ** 3)[..., None] * d).sum(axis=1)
    return phi, grad


def p2m_scalar(x, q, centre, p):
    """S-expansion of the monopoles q at x about `centre` (Eq. rsbf5):
    phi_n^m = sum_l q_l R_n^{-m}(-(x_l - centre)), n < p."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    if x.shape[0] == 0:
        return empty(p)
    R = R_table(p - 1, -(x - np.asarray(centre, dtype=np.float64)))   # [l, n, mu + p - 1] = R_n^mu(-r_l)
    g = R[..., ::-1]                                                   # [l, n, m + p - 1] = R_n^{-m}(-r_l)
    return (q[:, None, None] * g).sum(axis=0)


def l2p_scalar(c, r):
    """phi = sum c_n^m R_n^m(r) and grad phi, whose component k has the
    coefficients D_{i_k} c (Eq. dt3, R basis), at points r (N, 3) relative to the
    expansion centre."""
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    units = np.eye(3)
    phi = eval_R(c, r).real
    grad = np.stack([eval_R(apply_Dt(c, units[k], "R"), r).real for k in range(3)], axis=-1)
    return phi, grad


def _translate(cache, kind, key, t, c, p_out):
    pm = max(c.shape[0], p_out)
    T = cache.get((kind, pm) + key)
    if T is None:
        T = translation_matrix(kind, t, pm)
        cache[(kind, pm) + key] = T
    return resize(unflatten(T @ flatten(resize(c, pm)), pm), p_out)


class ScalarResult:
    pass


def fmm_scalar(x, q, p, leaf_max=64, tree=None, far=True, near=True, L_override=None):
    """O2s: phi and grad phi at every element (input order) by the scalar FMM over
    the octree of x (singular kernel: the leaf level is set by leaf_max alone,
    or by L_override)."""
    x32 = np.asarray(x, dtype=np.float32).reshape(-1, 3)
    xd = x32.astype(np.float64)
    qd = np.asarray(q, dtype=np.float32).reshape(-1).astype(np.float64)
    if tree is None:
        tree = build_tree(x32, leaf_max, 0.0, 1e-6, L_override=L_override)
    n = xd.shape[0]
    xs, qs = xd[tree.perm], qd[tree.perm]
    L = tree.L
    cache = {}
    res = ScalarResult()
    res.tree = tree
    res.multipole = [None] * (L + 1)
    res.local = [None] * (L + 1)
    phi_far = np.zeros(n)
    grad_far = np.zeros((n, 3))
    if far and L >= 2:
        lv = tree.levels[L]
        res.multipole[L] = [p2m_scalar(xs[lv["begin"][b]:lv["end"][b]], qs[lv["begin"][b]:lv["end"][b]],
                                       tree.centre(L, b), p) for b in range(lv["keys"].shape[0])]
        for lev in range(L - 1, 1, -1):          # upward pass: M2M
            d = tree.levels[lev]
            out = []
            for b in range(d["keys"].shape[0]):
                acc = empty(p)
                cb = tree.centre(lev, b)
                for ch in d["children"][b]:
                    t = cb - tree.centre(lev + 1, ch)
                    key = (lev, tuple(2 * d["coords"][b] - tree.levels[lev + 1]["coords"][ch]))
                    acc += _translate(cache, "SS", key, t, res.multipole[lev + 1][ch], p)
                out.append(acc)
            res.multipole[lev] = out
        for lev in range(2, L + 1):              # downward pass: L2L, M2L
            d = tree.levels[lev]
            out = []
            for b in range(d["keys"].shape[0]):
                acc = empty(p)
                cb = tree.centre(lev, b)
                if lev > 2:
                    par = d["parent"][b]
                    t = cb - tree.centre(lev - 1, par)
                    key = (lev, tuple(d["coords"][b] - 2 * tree.levels[lev - 1]["coords"][par]))
                    acc += _translate(cache, "RR", key, t, res.local[lev - 1][par], p)
                for s in d["il"][b]:
                    t = cb - tree.centre(lev, s)
                    key = (lev, tuple(d["coords"][b] - d["coords"][s]))
                    acc += _translate(cache, "SR", key, t, res.multipole[lev][s], p)
                out.append(acc)
            res.local[lev] = out
        lv = tree.levels[L]
        for b in range(lv["keys"].shape[0]):
            s0, s1 = lv["begin"][b], lv["end"][b]
            ph, gr = l2p_scalar(res.local[L][b], xs[s0:s1] - tree.centre(L, b))
            phi_far[s0:s1] = ph
            grad_far[s0:s1] = gr
    phi_near = np.zeros(n)
    grad_near = np.zeros((n, 3))
    if near and n > 0:
        lv = tree.levels[L]
        for b in range(lv["keys"].shape[0]):
            t0, t1 = lv["begin"][b], lv["end"][b]
            src = np.concatenate([np.arange(lv["begin"][c], lv["end"][c]) for c in lv["colleagues"][b]])
            tgt = np.arange(t0, t1)
            d = xs[tgt][:, None, :] - xs[src][None, :, :]
            r = np.sqrt((d * d).sum(axis=-1))
            skip = (tgt[:, None] == src[None, :]) | (r == 0.0)
            inv = np.where(skip, 0.0, 1.0 / np.where(skip, 1.0, r))
            phi_near[t0:t1] = (qs[src][None, :] * inv).sum(axis=1)
            grad_near[t0:t1] = -((qs[src][None, :] * inv ** 3)[..., None] * d).sum(axis=1)
    inv_perm = np.empty_like(tree.perm)
    inv_perm[tree.perm] = np.arange(n)
    res.phi = (phi_far + phi_near)[inv_perm]
    res.grad = (grad_far + grad_near)[inv_perm]
    res.phi_far, res.grad_far = phi_far[inv_perm], grad_far[inv_perm]
    res.phi_near, res.grad_near = phi_near[inv_perm], grad_near[inv_perm]
    return res
