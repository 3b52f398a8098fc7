"""Rotation - coaxial translation - back rotation (RCR) with coaxial conversion (Sec. 4.4,
Eq. rcr1, Fig. FigTscheme), FP64.

Test infrastructure (see ``oracle/__init__``).

A translation by t is carried out in the frame whose z axis is t: with Q a rotation taking
i_z to t/|t| (so that r = Q r'), the coefficients of each potential are rotated degree by
degree (f(c + Q r') = sum c'_n^m F_n^m(r'), which mixes only the 2n + 1 orders of degree n),
translated along z by |t| (the coaxial maps of Eq. mr3, which do not mix orders), converted by
the coaxial forms of the conversion operators (Eq. rcr1: t = |t| i_z in Eqs. drt10, drt11),
and rotated back with Q^T.  Rotations keep the Lamb-Helmholtz form (Eq. 4 is covariant under
rotations), so phi and chi are rotated as two scalar functions and the conversion acts in the
rotated frame.  The rotation of degree n is found from its definition: the 2n + 1 harmonics
evaluated at sample points r' on the unit sphere and at Q r', and the least-squares solution
(numpy.linalg.lstsq) of  F_n^m(Q r') = sum_m' X_{m'm} F_n^m'(r').
"""
import math

import numpy as np

from .basis import R_table, S_table
from .direct import pair_terms
from .expansions import l2p, p2m_method2
from .operators import empty, flatten, translation_matrix, unflatten
from .tree import build_tree

__all__ = ["frame_of", "rotation_blocks", "rotate", "coax_convert_R", "coax_convert_S",
           "translate_convert_rcr", "fmm_rcr"]


def _sphere_points(k):
    """k points spread over the unit sphere (the Fibonacci lattice)."""
    i = np.arange(k) + 0.5
    z = 1.0 - 2.0 * i / k
    rho = np.sqrt(1.0 - z * z)
    ph = math.pi * (1.0 + math.sqrt(5.0)) * i
    return np.stack([rho * np.cos(ph), rho * np.sin(ph), z], axis=1)


def frame_of(t):
    """A rotation Q (3 x 3) with Q i_z = t / |t|."""
    t = np.asarray(t, np.float64)
    z = t / np.linalg.norm(t)
    a = np.array([1.0, 0.0, 0.0]) if abs(z[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    x = a - (a @ z) * z
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=1)


def rotation_blocks(p, Q, basis):
    """X_n ((2n+1) x (2n+1), n < p): F_n^m(Q r') = sum_m' X_n[m', m] F_n^m'(r')."""
    pts = _sphere_points(6 * p + 12)
    tab = R_table if basis == "R" else S_table
    A = tab(p - 1, pts)                     # [k, n, m + p - 1]
    B = tab(p - 1, pts @ np.asarray(Q, np.float64).T)
    out = []
    for n in range(p):
        cols = slice(p - 1 - n, p + n)
        X, *_ = np.linalg.lstsq(A[:, n, cols], B[:, n, cols], rcond=None)
        out.append(X)
    return out


def rotate(c, blocks):
    """Coefficients of f(c + Q r') in r' from those of f(c + r) (blocks of rotation_blocks)."""
    p = c.shape[-2]
    out = empty(p)
    for n in range(p):
        cols = slice(p - 1 - n, p + n)
        out[n, cols] = blocks[n] @ c[n, cols]
    return out


def _nm(p):
    n = np.arange(p)[:, None] * np.ones((1, 2 * p - 1))
    m = np.arange(-(p - 1), p)[None, :] * np.ones((p, 1))
    return n, m


def _shift_n(c, dn):
    """Array whose (n, m) entry is c_{n+dn}^m (zero outside)."""
    out = np.zeros_like(c)
    p = c.shape[0]
    if dn > 0:
        out[:p - dn] = c[dn:]
    else:
        out[-dn:] = c[:p + dn]
    return out


def coax_convert_R(phi, chi, t):
    """Eq. rcr1, R conversion for t = t i_z:
    phi~ = phi^ + i t (m/n) chi^ (phi~_0^0 = phi^_0^0),  chi~ = chi^ - t/(n+1) chi^_{n+1}."""
    n, m = _nm(phi.shape[0])
    ratio = np.where(n > 0, m / np.maximum(n, 1), 0.0)
    valid = np.abs(m) <= n  # chi_{n+1}^m exists for |m| = n + 1, chi~_n^m does not
    return phi + 1j * t * ratio * chi, (chi - t / (n + 1) * _shift_n(chi, 1)) * valid


def coax_convert_S(phi, chi, t):
    """Eq. rcr1, S conversion for t = t i_z:
    phi~ = phi^ - i t m/(n+1) chi^,  chi~ = chi^ + (t/n) chi^_{n-1} (chi~_0^0 = chi^_0^0)."""
    n, m = _nm(phi.shape[0])
    inv_n = np.where(n > 0, 1.0 / np.maximum(n, 1), 0.0)
    valid = np.abs(m) <= n
    return phi - 1j * t * m / (n + 1) * chi, (chi + t * inv_n * _shift_n(chi, -1)) * valid


def translate_convert_rcr(kind, phi, chi, t, cache=None, key=None):
    """One translation of the pair (phi, chi) by t (kind "SS", "SR" or "RR") with its
    conversion, by RCR: rotate, coaxial translation by |t| along z, Eq. rcr1, rotate back."""
    p = phi.shape[0]
    d = float(np.linalg.norm(t))
    basis_in = "R" if kind == "RR" else "S"
    basis_out = "S" if kind == "SS" else "R"
    cache = {} if cache is None else cache
    ck = (kind, p) + (key if key is not None else tuple(np.round(np.asarray(t, np.float64), 14)))
    if ck not in cache:
        Q = frame_of(t)
        cache[ck] = (rotation_blocks(p, Q, basis_in), rotation_blocks(p, Q.T, basis_out),
                     translation_matrix(kind, (0.0, 0.0, d), p))
    fwd, back, T = cache[ck]
    ph = unflatten(T @ flatten(rotate(phi, fwd)), p)
    cc = unflatten(T @ flatten(rotate(chi, fwd)), p)
    ph, cc = (coax_convert_S if kind == "SS" else coax_convert_R)(ph, cc, d)
    return rotate(ph, back), rotate(cc, back)


def fmm_rcr(x, w, p, leaf_max=64, a=0.0, eps=1e-6, tree=None):
    """The two-potential FMM of ``fmm`` (O2) with every translation and conversion by RCR."""
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
    lv = tree.levels[L]
    if L >= 2:
        mp[L] = [p2m_method2(xs[lv["begin"][b]:lv["end"][b]], ws[lv["begin"][b]:lv["end"][b]], tree.centre(L, b), p)
                 for b in range(lv["keys"].shape[0])]
        for lev in range(L - 1, 1, -1):
            d = tree.levels[lev]
            out = []
            for b in range(d["keys"].shape[0]):
                phi, chi = empty(p), empty(p)
                cb = tree.centre(lev, b)
                for ch in d["children"][b]:
                    t = cb - tree.centre(lev + 1, ch)
                    k = (lev, tuple(2 * d["coords"][b] - tree.levels[lev + 1]["coords"][ch]))
                    ph, cc = translate_convert_rcr("SS", *mp[lev + 1][ch], t, cache, k)
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
                    k = (lev, tuple(d["coords"][b] - 2 * tree.levels[lev - 1]["coords"][par]))
                    ph, cc = translate_convert_rcr("RR", *lc[lev - 1][par], t, cache, k)
                    phi += ph
                    chi += cc
                for s in d["il"][b]:
                    t = cb - tree.centre(lev, s)
                    k = (lev, tuple(d["coords"][b] - d["coords"][s]))
                    ph, cc = translate_convert_rcr("SR", *mp[lev][s], t, cache, k)
                    phi += ph
                    chi += cc
                out.append((phi, chi))
            lc[lev] = out
        for b in range(lv["keys"].shape[0]):
            s0, s1 = lv["begin"][b], lv["end"][b]
            vv, uu, _ = l2p(lc[L][b][0], lc[L][b][1], xs[s0:s1] - tree.centre(L, b), ws[s0:s1])
            v[s0:s1] += vv
            u[s0:s1] += uu
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

    class Res:
        pass
    r = Res()
    r.tree, r.v, r.grad, r.s = tree, v[inv], u[inv], s_[inv]
    return r
