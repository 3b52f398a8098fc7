"""Thin Python binding over the C ABI: torch tensors in, raw pointers to liblhv.so.

Every step of the computation runs in the library's CUDA kernels; this module
only checks tensor shapes/dtypes and passes pointers, sizes and the current
CUDA stream."""
import ctypes

import torch

from . import _lib as L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class LHV:
    """One library context (operator tables, tree and work buffers) on one stream."""

    def __init__(self, p, leaf_max=64, core_a=0.0, eps=1e-6, precision="fp32", terms="all",
                 max_level=0, stream=None, device=None):
        self.lib = L.load()
        if precision not in ("fp32", "fp64", "tf32x3"):
            raise ValueError("precision must be fp32, fp64 or tf32x3")
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        cfg = L.Config(p=int(p), leaf_max=int(leaf_max), core_a=float(core_a), eps=float(eps),
                       precision={"fp32": L.LHV_FP32, "fp64": L.LHV_FP64, "tf32x3": L.LHV_TF32X3}[precision],
                       terms={"near": 1, "far": 2, "all": 3}[terms], max_level=int(max_level))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.lhv_create(ctypes.byref(cfg), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise L.LHVError(st, "lhv_create: " + self.lib.lhv_status_string(st).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lhv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.lhv_last_error(self.h).decode() or self.lib.lhv_status_string(st).decode()
            raise L.LHVError(st, f"{what}: {msg}")

    def _elems(self, t):
        if t.device.type != "cuda" or t.dtype != self.dtype or t.dim() != 2 or t.shape[1] != 4 or not t.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA {self.dtype} tensor of shape [n, 4]")
        return t

    def build_tree(self, x4):
        self._elems(x4)
        self._check(self.lib.lhv_build_tree(self.h, x4.shape[0], _ptr(x4)), "lhv_build_tree")

    def evaluate_velocity_stretching(self, x4, w4, v4=None, s4=None):
        self._elems(x4)
        self._elems(w4)
        n = x4.shape[0]
        v4 = torch.empty_like(x4) if v4 is None else self._elems(v4)
        s4 = torch.empty_like(x4) if s4 is None else self._elems(s4)
        fn = self.lib.lhv_evaluate_velocity_stretching_f64 if self.precision == "fp64" else \
            self.lib.lhv_evaluate_velocity_stretching
        self._check(fn(self.h, n, _ptr(x4), _ptr(w4), _ptr(v4), _ptr(s4)), "evaluate_velocity_stretching")
        return v4, s4

    def evaluate_potential_gradient(self, x4, q, pg4=None):
        """The scalar reference case (lhv_evaluate_potential_gradient): monopoles q (CUDA [n],
        the context's dtype) at x4; returns pg4 [n, 4] = (grad phi, phi)."""
        self._elems(x4)
        if q.device.type != "cuda" or q.dtype != self.dtype or q.dim() != 1 or q.shape[0] != x4.shape[0] \
                or not q.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA {self.dtype} vector of {x4.shape[0]} charges")
        pg4 = torch.empty_like(x4) if pg4 is None else self._elems(pg4)
        fn = self.lib.lhv_evaluate_potential_gradient_f64 if self.precision == "fp64" else \
            self.lib.lhv_evaluate_potential_gradient
        self._check(fn(self.h, x4.shape[0], _ptr(x4), _ptr(q), _ptr(pg4)), "evaluate_potential_gradient")
        return pg4

    def evaluate_filaments(self, offsets, closed, x4, gamma, v4=None):
        """Vortex filaments (lhv_evaluate_filaments): filament f owns the nodes
        offsets[f]:offsets[f+1] of x4, closed[f] joins its last node to its first; gamma
        (CUDA [n], the context's dtype) is the circulation of the segment starting at each
        node.  Returns v at the nodes, [n, 4]."""
        self._elems(x4)
        if gamma.device.type != "cuda" or gamma.dtype != self.dtype or gamma.dim() != 1 or \
                gamma.shape[0] != x4.shape[0] or not gamma.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA {self.dtype} vector of {x4.shape[0]} circulations")
        off = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
        cl = (ctypes.c_int32 * len(closed))(*[1 if c else 0 for c in closed])
        v4 = torch.empty_like(x4) if v4 is None else self._elems(v4)
        fn = self.lib.lhv_evaluate_filaments_f64 if self.precision == "fp64" else self.lib.lhv_evaluate_filaments
        self._check(fn(self.h, len(offsets) - 1, off, cl, _ptr(x4), _ptr(gamma), _ptr(v4)), "evaluate_filaments")
        return v4

    def evaluate_batched(self, offsets, x4, w4, v4=None, s4=None):
        """Independent systems: system k owns rows offsets[k]:offsets[k+1]."""
        self._elems(x4)
        self._elems(w4)
        off = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
        v4 = torch.empty_like(x4) if v4 is None else self._elems(v4)
        s4 = torch.empty_like(x4) if s4 is None else self._elems(s4)
        self._check(self.lib.lhv_evaluate_batched(self.h, len(offsets) - 1, off, _ptr(x4), _ptr(w4), _ptr(v4),
                                                  _ptr(s4)), "evaluate_batched")
        return v4, s4

    def step_batched(self, offsets, x4, w4, dt):
        self._elems(x4)
        self._elems(w4)
        off = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
        self._check(self.lib.lhv_step_batched(self.h, len(offsets) - 1, off, _ptr(x4), _ptr(w4), float(dt)),
                    "step_batched")

    def step(self, x4, w4, dt):
        self._elems(x4)
        self._elems(w4)
        fn = self.lib.lhv_step_f64 if self.precision == "fp64" else self.lib.lhv_step
        self._check(fn(self.h, x4.shape[0], _ptr(x4), _ptr(w4), float(dt)), "step")

    def step_host(self, x4_host, w4_host, dt):
        """x4_host, w4_host: contiguous CPU float32 [n, 4] tensors (pinned or pageable)."""
        for t in (x4_host, w4_host):
            if t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous() or t.shape[1] != 4:
                raise ValueError("expected contiguous CPU float32 [n, 4] tensors")
        self._check(self.lib.lhv_step_host(self.h, x4_host.shape[0], _ptr(x4_host), _ptr(w4_host), float(dt)),
                    "step_host")

    def set_timing(self, on=True):
        self._check(self.lib.lhv_set_timing(self.h, 1 if on else 0), "set_timing")

    def reset_stats(self):
        self._check(self.lib.lhv_reset_stats(self.h), "reset_stats")

    def stats(self):
        s = L.Stats()
        self._check(self.lib.lhv_get_stats(self.h, ctypes.byref(s)), "get_stats")
        return {
            "leaf_level": s.leaf_level, "nbox": list(s.nbox)[: s.leaf_level + 1], "n": s.n,
            "p2p_pairs": s.p2p_pairs, "m2l_pairs": s.m2l_pairs,
            "stage_ms": dict(zip(L.STAGES, list(s.stage_ms))),
            "stage_launches": dict(zip(L.STAGES, list(s.stage_launches))),
            "kernel_launches": s.kernel_launches,
            "level_p": list(s.level_p)[: s.leaf_level + 1],
            "launch_shape": {"p2p_targets_per_thread": s.tuned_p2p_targets_per_thread,
                             "p2p_sources_per_stage": s.tuned_p2p_sources_per_stage,
                             "m2l_pairs_per_chunk": s.tuned_m2l_pairs_per_chunk,
                             "m2l_tensor_cores": s.tuned_m2l_tensor_cores, "tune_ms": list(s.tune_ms)},
            "selector": {"leaf_max": s.selector_leaf_max, "selections": s.selector_selections,
                         "checks": s.selector_checks, "fallbacks": s.selector_fallbacks,
                         "err_v": s.selector_err_v, "err_s": s.selector_err_s},
            "graph": {"captures": s.graph_captures, "replays": s.graph_replays, "fallbacks": s.graph_fallbacks,
                      "kernels": s.graph_kernels},
        }

    def autotune(self, x4, w4, offsets=None):
        """lhv_autotune (or lhv_autotune_batched with host offsets): keeps the fastest launch shapes."""
        self._elems(x4)
        self._elems(w4)
        v4, s4 = torch.empty_like(x4), torch.empty_like(x4)
        if offsets is None:
            self._check(self.lib.lhv_autotune(self.h, x4.shape[0], _ptr(x4), _ptr(w4), _ptr(v4), _ptr(s4)), "autotune")
        else:
            off = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
            self._check(self.lib.lhv_autotune_batched(self.h, len(offsets) - 1, off, _ptr(x4), _ptr(w4), _ptr(v4),
                                                      _ptr(s4)), "autotune_batched")
        return self.stats()["launch_shape"]

    def set_launch_shape(self, p2p_targets_per_thread=1, m2l_pairs_per_chunk=0, m2l_tensor_cores=1,
                         p2p_sources_per_stage=128):
        self._check(self.lib.lhv_set_launch_shape(self.h, int(p2p_targets_per_thread), int(p2p_sources_per_stage),
                                                  int(m2l_pairs_per_chunk), int(m2l_tensor_cores)),
                    "set_launch_shape")

    def set_selector(self, W=None, b=None, eps=1e-6, check_every=1, check_samples=1000):
        """Switch the learned form on with network weights W (bfloat16 [LHV_MLP_NW]) and
        biases b (float32 [LHV_MLP_NB]), host or device tensors; W = None switches it off."""
        if W is None:
            self._check(self.lib.lhv_set_selector(self.h, None, None, float(eps), 0, 1), "set_selector")
            return
        Wh = W.detach().to("cpu", torch.bfloat16).contiguous()
        bh = b.detach().to("cpu", torch.float32).contiguous()
        if Wh.numel() != L.MLP_NW or bh.numel() != L.MLP_NB:
            raise ValueError("selector weights have the wrong size")
        self._check(self.lib.lhv_set_selector(self.h, _ptr(Wh), _ptr(bh), float(eps), int(check_every),
                                              int(check_samples)), "set_selector")

    def selector_features(self, x4, w4, eps=1e-6):
        """Feature rows (CUDA float32 [L-1, 12]) of the levels 2..L of the tree of x4."""
        self._elems(x4)
        self._elems(w4)
        rows = ctypes.c_int(0)
        self._check(self.lib.lhv_selector_features(self.h, x4.shape[0], _ptr(x4), _ptr(w4), float(eps), None, 0,
                                                   ctypes.byref(rows)), "selector_features")
        X = torch.empty((max(rows.value, 1), L.MLP_IN), dtype=torch.float32, device=self.device)
        self._check(self.lib.lhv_selector_features(self.h, x4.shape[0], _ptr(x4), _ptr(w4), float(eps), _ptr(X),
                                                   X.shape[0], ctypes.byref(rows)), "selector_features")
        return X[: rows.value]

    def direct_sampled(self, x4, w4, idx):
        """FP64 direct sums (lhv_direct_sampled) at the elements idx (CUDA int32 [m]):
        returns (v, s) as CUDA float64 [m, 4] tensors."""
        self._elems(x4)
        self._elems(w4)
        if not (idx.is_cuda and idx.dtype == torch.int32 and idx.dim() == 1 and idx.is_contiguous()):
            raise ValueError("idx must be a contiguous CUDA int32 vector")
        m = idx.shape[0]
        v = torch.empty((m, 4), dtype=torch.float64, device=self.device)
        s = torch.empty((m, 4), dtype=torch.float64, device=self.device)
        fn = self.lib.lhv_direct_sampled_f64 if self.precision == "fp64" else self.lib.lhv_direct_sampled
        self._check(fn(self.h, x4.shape[0], _ptr(x4), _ptr(w4), m, _ptr(idx), _ptr(v), _ptr(s)), "direct_sampled")
        return v, s

    def set_graph(self, enable=True):
        """lhv_set_graph: each RK4 step (step / step_batched / step_host) as one CUDA graph
        replay; the context must use a stream other than the legacy default stream."""
        self._check(self.lib.lhv_set_graph(self.h, 1 if enable else 0), "set_graph")

    def set_form(self, form="phi_chi"):
        """Far-field representation (lhv_set_form): "phi_chi" (two real potentials, the default),
        "psi" (one complex function Psi = phi + i chi, Eq. chf1) or "rcr" (the two potentials
        with M2L by rotation - coaxial translation - back rotation, Sec. 4.4, Eq. rcr1)."""
        code = {"phi_chi": L.LHV_FORM_PHI_CHI, "psi": L.LHV_FORM_PSI, "rcr": L.LHV_FORM_RCR}[form]
        self._check(self.lib.lhv_set_form(self.h, code), "set_form")

    def set_level_p(self, p_per_level=None):
        """Truncation number per octree level (lhv_set_level_p); None restores config p."""
        vals = [int(v) for v in (p_per_level or [])]
        arr = (ctypes.c_int * max(len(vals), 1))(*vals)
        self._check(self.lib.lhv_set_level_p(self.h, arr, len(vals)), "set_level_p")

    def export(self, what, level=0):
        """Copy an internal array (see lhv_export) into a new CUDA tensor."""
        code = L.EXPORT[what]
        nbytes = ctypes.c_int64(0)
        self._check(self.lib.lhv_export(self.h, code, int(level), None, 0, ctypes.byref(nbytes)), f"export {what}")
        buf = torch.empty(max(int(nbytes.value), 1), dtype=torch.uint8, device=self.device)
        self._check(self.lib.lhv_export(self.h, code, int(level), _ptr(buf), buf.numel(), ctypes.byref(nbytes)),
                    f"export {what}")
        buf = buf[: int(nbytes.value)]
        if what == "keys":
            return buf.view(torch.int64)
        if what in ("perm", "box_range", "colleagues"):
            return buf.view(torch.int32)
        if what == "box_keys":
            return buf.view(torch.int64)
        if what == "cube":
            return buf.view(torch.float64)
        return buf.view(self.dtype)


def morton_sort_noalloc(x4, keys, perm, w4=None):
    """lhv_morton_sort_noalloc: sorted Morton keys and permutation of one system
    without any device allocation, written into the caller's CUDA tensors
    ``keys`` (int64 [n]) and ``perm`` (int32 [n]); x4 (and w4) float32 [n][4].
    Runs on the current CUDA stream and returns when it has finished.  Calls
    that overlap in time on one device race on the library's fixed scratch."""
    lib = L.load()
    n = x4.shape[0]
    for t, dt, shape in ((x4, torch.float32, (n, 4)), (keys, torch.int64, (n,)), (perm, torch.int32, (n,))):
        if not (t.is_cuda and t.dtype == dt and tuple(t.shape) == shape and t.is_contiguous()):
            raise ValueError(f"expected a contiguous CUDA {dt} tensor of shape {shape}")
    if w4 is not None and not (w4.is_cuda and w4.dtype == torch.float32 and w4.shape == x4.shape
                               and w4.is_contiguous()):
        raise ValueError("w4 must match x4")
    with torch.cuda.device(x4.device):
        stream = ctypes.c_void_p(torch.cuda.current_stream(x4.device).cuda_stream)
        st = lib.lhv_morton_sort_noalloc(n, _ptr(x4), _ptr(w4) if w4 is not None else None, _ptr(keys),
                                         _ptr(perm), stream)
    if st != 0:
        raise L.LHVError(st, "morton_sort_noalloc: " + lib.lhv_status_string(st).decode())


# ---- selector network (lhv_mlp_*): stateless calls on caller tensors ------------

def _stream(t):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _need(t, dtype, numel=None):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and (numel is None or t.numel() == numel)):
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor" + (f" of {numel} values" if numel else ""))


def mlp_forward(X, W, b):
    """Logits [rows, 21] of feature rows X (float32 [rows, 12]); W: bfloat16 [LHV_MLP_NW], b: float32."""
    lib = L.load()
    _need(X, torch.float32)
    _need(W, torch.bfloat16, L.MLP_NW)
    _need(b, torch.float32, L.MLP_NB)
    rows = X.shape[0]
    Z = torch.empty((rows, L.MLP_OUT), dtype=torch.float32, device=X.device)
    with torch.cuda.device(X.device):
        st = lib.lhv_mlp_forward(rows, _ptr(X), _ptr(W), _ptr(b), _ptr(Z), _stream(X))
    if st:
        raise L.LHVError(st, "mlp_forward")
    return Z


def mlp_loss_grad(X, yp, yl, W, b):
    """(loss, gW, gb) of lhv_mlp_loss_grad; yp, yl int32 [rows] (-1 = no label)."""
    lib = L.load()
    _need(X, torch.float32)
    _need(yp, torch.int32, X.shape[0])
    _need(yl, torch.int32, X.shape[0])
    _need(W, torch.bfloat16, L.MLP_NW)
    _need(b, torch.float32, L.MLP_NB)
    dev = X.device
    gW = torch.empty(L.MLP_NW, dtype=torch.float32, device=dev)
    gb = torch.empty(L.MLP_NB, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    work = torch.empty(2, dtype=torch.int32, device=dev)
    with torch.cuda.device(dev):
        st = lib.lhv_mlp_loss_grad(X.shape[0], _ptr(X), _ptr(yp), _ptr(yl), _ptr(W), _ptr(b), _ptr(gW), _ptr(gb),
                                   _ptr(loss), _ptr(work), _stream(X))
    if st:
        raise L.LHVError(st, "mlp_loss_grad")
    return loss, gW, gb


def mlp_adam(W32, W, gW, mW, vW, b, gb, mb, vb, t, lr):
    """One lhv_mlp_adam step in place (all CUDA tensors; W bfloat16, the rest float32)."""
    lib = L.load()
    for x in (W32, gW, mW, vW):
        _need(x, torch.float32, L.MLP_NW)
    for x in (b, gb, mb, vb):
        _need(x, torch.float32, L.MLP_NB)
    _need(W, torch.bfloat16, L.MLP_NW)
    with torch.cuda.device(W32.device):
        st = lib.lhv_mlp_adam(_ptr(W32), _ptr(W), _ptr(gW), _ptr(mW), _ptr(vW), _ptr(b), _ptr(gb), _ptr(mb),
                              _ptr(vb), int(t), float(lr), _stream(W32))
    if st:
        raise L.LHVError(st, "mlp_adam")
