"""Helpers of the GPU parity tests: device transfer and the coefficient layout of
lhv_export (scaled real -> the oracle's complex, unscaled, full-m arrays)."""
import math

import numpy as np

import workloads


def dev(a3, dtype):
    import torch
    t = torch.from_numpy(workloads.to_f4(a3, np.float32 if dtype == "fp32" else np.float64))
    return t.cuda()


def host3(t):
    return t[:, :3].double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def nu(n, m):
    m = abs(m)
    return math.sqrt(math.factorial(n - m) * math.factorial(n + m))


def to_complex(vec, p, h, basis):
    """One box's exported (2, p*p) scaled real vector -> (phi, chi) complex (p, 2p-1).

    Layout (include/lhv.h): Re c_n^0 at n*n; Re, Im c_n^m at n*n + 2m - 1, n*n + 2m.
    S: phi = stored h^(n+1)/nu, chi = stored h^n/nu.  R: phi = stored nu/h^n, chi = stored nu/h^(n+1)."""
    P = p * p
    vec = np.asarray(vec, dtype=np.float64).reshape(2, P)
    out = []
    for pot in range(2):
        c = np.zeros((p, 2 * p - 1), dtype=np.complex128)
        for n in range(p):
            for m in range(0, n + 1):
                if m == 0:
                    val = vec[pot, n * n] + 0j
                else:
                    val = vec[pot, n * n + 2 * m - 1] + 1j * vec[pot, n * n + 2 * m]
                if basis == "S":
                    val *= h ** (n + 1 - pot) / nu(n, m)
                else:
                    val *= nu(n, m) / h ** (n + pot)
                c[n, m + p - 1] = val
                c[n, -m + p - 1] = (-1) ** m * np.conj(val)
        out.append(c)
    return out
