"""The selector network of the learned form, in FP64 (test infrastructure).

The paper uses one truncation number for the whole octree (Sec. 5 lists
"variable truncation number" among the optimisations it left out).  The learned
form picks one per level: a multilayer perceptron maps 12 features of an octree
level to scores of the truncation numbers p = 4 .. 20 and of the leaf caps
16, 32, 64, 128.  This module is the plain definition the GPU kernels are
checked against; nothing in it is tuned.

Network (weights W_k of shape (out, in), biases b_k):
    h1 = relu(W1 x + b1)      12 -> 64
    h2 = relu(W2 h1 + b2)     64 -> 64
    h3 = relu(W3 h2 + b3)     64 -> 64
    z  = W4 h3 + b4           64 -> 21   (z[0:17]: p = 4 .. 20, z[17:21]: leaf caps)
The weights enter as their bfloat16 values (``bf16_round``), the arithmetic is FP64.

Loss of a batch (rows r with labels yp[r] in 0..16 or -1, yl[r] in 0..3 or -1):
    mean over rows with yp >= 0 of  -log softmax(z[r, 0:17])[yp]
  + mean over rows with yl >= 0 of  -log softmax(z[r, 17:21])[yl]
Backward pass: the chain rule through the same layers (gradients with respect to
the weights as continuous variables, evaluated at their bfloat16 values).
"""
import numpy as np

__all__ = ["SIZES", "N_P", "N_LEAF", "P_VALUES", "LEAF_CAPS", "bf16_round", "init", "unpack", "forward",
           "loss_and_grad", "adam"]

SIZES = [(64, 12), (64, 64), (64, 64), (21, 64)]
N_P = 17
N_LEAF = 4
P_VALUES = list(range(4, 21))
LEAF_CAPS = [16, 32, 64, 128]


def bf16_round(a):
    """Nearest bfloat16 value of each FP32 number (ties to even), as float64.

    A bfloat16 keeps the top 16 bits of an FP32 word: add 0x7fff plus the lowest
    kept bit, then clear the low 16 bits."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64).reshape(f.shape)


def n_weights():
    return sum(o * i for o, i in SIZES)


def n_biases():
    return sum(o for o, _ in SIZES)


def init(seed=0):
    """He-uniform weights and zero biases, FP32 (flat vectors in the layout of unpack)."""
    rng = np.random.default_rng(seed)
    ws = [rng.uniform(-1, 1, (o, i)) * np.sqrt(6.0 / i) for o, i in SIZES]
    return (np.concatenate([w.ravel() for w in ws]).astype(np.float32),
            np.zeros(n_biases(), dtype=np.float32))


def unpack(wflat, bflat):
    """Flat vectors -> lists of (out, in) weight matrices and bias vectors.
    Layout: W1, W2, W3, W4 row-major one after the other; b1, b2, b3, b4 likewise."""
    ws, bs, i, j = [], [], 0, 0
    for o, n in SIZES:
        ws.append(np.asarray(wflat[i:i + o * n], dtype=np.float64).reshape(o, n))
        bs.append(np.asarray(bflat[j:j + o], dtype=np.float64))
        i += o * n
        j += o
    return ws, bs


def forward(x, wflat, bflat, rnd=bf16_round):
    """Logits z (rows, 21) of the feature rows x (rows, 12); weights rounded to bfloat16."""
    ws, bs = unpack(rnd(wflat), bflat)
    h = np.asarray(x, dtype=np.float64)
    for k in range(3):
        h = np.maximum(ws[k] @ h.T + bs[k][:, None], 0.0).T
    return (ws[3] @ h.T + bs[3][:, None]).T


def _softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss_and_grad(x, yp, yl, wflat, bflat, rnd=bf16_round):
    """Loss of the batch and its gradient (flat, same layout as wflat / bflat).
    rnd: the rounding applied to the weights (identity for a finite-difference check)."""
    ws, bs = unpack(rnd(wflat), bflat)
    x = np.asarray(x, dtype=np.float64)
    acts = [x]
    pre = []
    h = x
    for k in range(3):
        a = h @ ws[k].T + bs[k]
        pre.append(a)
        h = np.maximum(a, 0.0)
        acts.append(h)
    z = h @ ws[3].T + bs[3]
    yp = np.asarray(yp)
    yl = np.asarray(yl)
    dz = np.zeros_like(z)
    loss = 0.0
    mp, ml = yp >= 0, yl >= 0
    if mp.any():
        sp = _softmax(z[mp, :N_P])
        loss -= np.log(sp[np.arange(sp.shape[0]), yp[mp]]).mean()
        g = sp.copy()
        g[np.arange(g.shape[0]), yp[mp]] -= 1.0
        dz[np.where(mp)[0], :N_P] = g / mp.sum()
    if ml.any():
        sl = _softmax(z[ml, N_P:])
        loss -= np.log(sl[np.arange(sl.shape[0]), yl[ml]]).mean()
        g = sl.copy()
        g[np.arange(g.shape[0]), yl[ml]] -= 1.0
        dz[np.where(ml)[0], N_P:] = g / ml.sum()
    gws, gbs = [None] * 4, [None] * 4
    d = dz
    for k in range(3, -1, -1):
        gws[k] = d.T @ acts[k]
        gbs[k] = d.sum(axis=0)
        if k > 0:
            d = (d @ ws[k]) * (pre[k - 1] > 0)
    return loss, np.concatenate([g.ravel() for g in gws]), np.concatenate(gbs)


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) in place; t counts from 1."""
    m[:] = b1 * m + (1 - b1) * g
    v[:] = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    theta[:] = theta - lr * mh / (np.sqrt(vh) + eps)
