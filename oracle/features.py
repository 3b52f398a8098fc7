"""The selector network's input: 12 features of each octree level l = 2 .. L
(test infrastructure).  Written from their definitions over the oracle's tree:

  0  l / 10                          6  log2(a / h_l) / 10, at least -3 (-3 when a = 0)
  1  (L - l) / 10                    7  mean interaction-list size of the level / 189
  2  log2(boxes at l) / 20           8  mean colleague count of the level / 27
  3  log2(boxes(l) / boxes(l-1)) / 3 9  log10(sum_b |sum_{j in b} w_j| / sum_j |w_j|) / 3, at least -3
  4  log2(n / boxes at l) / 20       10 log2(n) / 24
  5  -log10(eps) / 10                11 0 for FP32, 0.5 for TF32x3 arithmetic

Interaction list and colleagues as in Sec. 5 (the 189-box stencil): colleagues
are the occupied boxes of the 3x3x3 block around a box, the interaction list the
children of the parent's colleagues that are not colleagues.
"""
import math

import numpy as np

__all__ = ["level_features"]


def level_features(tree, w, eps, a, prec=0.0):
    """(L - 1, 12) FP64 rows for the levels 2..L of ``tree`` (oracle.tree.Tree);
    w: (n, 3) strengths in the caller's order."""
    w = np.asarray(w, dtype=np.float64).reshape(-1, 3)
    ws = w[tree.perm]
    L, n = tree.L, tree.n
    total = np.linalg.norm(ws, axis=1).sum()
    rows = []
    for lev in range(2, L + 1):
        d = tree.levels[lev]
        nb = d["keys"].shape[0]
        nbp = tree.levels[lev - 1]["keys"].shape[0]
        moments = sum(np.linalg.norm(ws[d["begin"][b]:d["end"][b]].sum(axis=0)) for b in range(nb))
        il = np.mean([len(v) for v in d["il"]])
        col = np.mean([len(v) for v in d["colleagues"]])
        h = tree.side / 2 ** lev
        rows.append([
            lev / 10.0,
            (L - lev) / 10.0,
            math.log2(nb) / 20.0,
            math.log2(nb / nbp) / 3.0,
            math.log2(n / nb) / 20.0,
            -math.log10(eps) / 10.0,
            max(-3.0, math.log2(a / h) / 10.0) if a > 0 else -3.0,
            il / 189.0,
            col / 27.0,
            max(-3.0, math.log10(moments / total) / 3.0) if moments > 0 and total > 0 else -3.0,
            math.log2(n) / 24.0,
            prec,
        ])
    return np.array(rows, dtype=np.float64).reshape(-1, 12)
