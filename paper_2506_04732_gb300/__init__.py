"""GB300 (sm_103a) hot path of T^2S^2 (arXiv 2506.04732): thin Python binding.

Every function here marshals arguments and calls the C ABI declared in
``include/t2s2.h`` (``libt2s2.so``, built in-tree by ``build.py``); all
arithmetic of the path runs in that library's CUDA kernels.  PyTorch only
provides device / pinned-host memory and the current CUDA stream.  There is
no CPU fallback: if the library is missing, ``load()`` raises.

Names follow the C entry points: ``t2s2_build_operator``, ``t2s2_apply``,
``t2s2_round``, ``t2s2_solve``, ``t2s2_cn_step`` and helpers.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

__all__ = ["load", "T2S2Error", "Operator", "TT", "SolveInfo", "FP64", "FP32_REFINE",
           "TF32_REFINE", "BF16_REFINE", "RANK_KICK", "t2s2_build_operator", "t2s2_apply", "t2s2_round",
           "t2s2_norm", "t2s2_diff_norm", "t2s2_norm_noalloc", "t2s2_residual", "t2s2_solve", "t2s2_solve_batched", "t2s2_cn_step", "t2s2_be_step",
           "t2s2_device_count", "t2s2_strerror", "t2s2_gemm", "WarmStartNet", "t2s2_apply_batched",
           "t2s2_autotune_report", "t2s2_kernel_launches", "t2s2_trace",
           "t2s2_trace_read", "t2s2_trace_overhead", "t2s2_fastmath", "t2s2_tt_fibre", "TRACE_FAMILIES", "lib_path", "t2s2_dim_matrices", "DIM_SPACE",
           "t2s2_build_spacetime_operator", "t2s2_spacetime_rhs", "t2s2_build_operator_var", "t2s2_dirichlet_rhs", "t2s2_solve_dirichlet",
           "DIM_SPACE_PLAIN", "DIM_TIME"]

FP64, FP32_REFINE, TF32_REFINE, BF16_REFINE = 0, 1, 2, 3
DIM_SPACE, DIM_SPACE_PLAIN, DIM_TIME = 0, 1, 2
# enrichment rank of the solver (T2S2_RANK_KICK; the T2S2_KICK environment
# variable overrides it): a solution can carry ranks up to rmax + RANK_KICK
RANK_KICK = int(os.environ.get("T2S2_KICK", "8")) if 1 <= int(os.environ.get("T2S2_KICK", "8")) <= 16 else 8
_DEVICE, _HOST = 0, 1
MAX_D = 16

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "libt2s2.so")
_lib = None


class T2S2Error(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {t2s2_strerror(status)} (status {status})")


class _Problem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.POINTER(ctypes.c_int)),
                ("beta", ctypes.POINTER(ctypes.c_double)), ("eps", ctypes.c_double),
                ("plain_sc", ctypes.c_int)]


_COEF_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_void_p)


class _ProblemVar(ctypes.Structure):
    _fields_ = [("base", _Problem), ("beta_fn", _COEF_FN), ("rho_fn", _COEF_FN), ("rho0", ctypes.c_double),
                ("ctx", ctypes.c_void_p), ("prod_fn", _COEF_FN)]


class _TT(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("m", ctypes.POINTER(ctypes.c_int)),
                ("r", ctypes.POINTER(ctypes.c_int)),
                ("cores", ctypes.POINTER(ctypes.c_void_p)),
                ("cap", ctypes.POINTER(ctypes.c_size_t)), ("loc", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("residual", ctypes.c_double), ("sweeps", ctypes.c_int),
                ("max_rank", ctypes.c_int), ("refinements", ctypes.c_int),
                ("local_iters", ctypes.c_longlong)]


@dataclass
class SolveInfo:
    status: int
    residual: float
    sweeps: int
    max_rank: int
    refinements: int
    local_iters: int


_SIGS = {
    "t2s2_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "t2s2_device_count": (ctypes.c_int, []),
    "t2s2_build_operator": (ctypes.c_int, [ctypes.POINTER(_Problem), ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "t2s2_build_operator_var": (ctypes.c_int, [ctypes.POINTER(_ProblemVar), ctypes.c_void_p,
                                               ctypes.POINTER(ctypes.c_void_p)]),
    "t2s2_build_spacetime_operator": (ctypes.c_int, [ctypes.POINTER(_Problem), ctypes.c_int, ctypes.c_double,
                                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "t2s2_spacetime_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.POINTER(_TT),
                                          ctypes.POINTER(_TT), ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "t2s2_dirichlet_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.POINTER(_TT), ctypes.c_double,
                                          ctypes.c_double, ctypes.POINTER(_TT), ctypes.c_double, ctypes.c_int,
                                          ctypes.c_void_p]),
    "t2s2_solve_dirichlet": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.POINTER(_TT),
                                            ctypes.POINTER(_TT), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.POINTER(_Info)]),
    "t2s2_op_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "t2s2_dim_matrices": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
                          + [ctypes.c_void_p] * 6),
    "t2s2_op_nodes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "t2s2_op_matrices": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "t2s2_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.POINTER(_TT),
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "t2s2_round": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.c_double,
                                  ctypes.c_int, ctypes.c_void_p]),
    "t2s2_norm": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT),
                                 ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "t2s2_norm_noalloc": (ctypes.c_int, [ctypes.POINTER(_TT), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_void_p]),
    "t2s2_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.POINTER(_TT),
                                     ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "t2s2_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.POINTER(_TT),
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(_Info)]),
    "t2s2_solve_batched": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_TT),
                                          ctypes.POINTER(_TT), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_Info), ctypes.POINTER(ctypes.c_int)]),
    "t2s2_cn_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(_Info)]),
    "t2s2_be_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(_Info)]),
    "t2s2_gemm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_long, ctypes.c_long,
                                 ctypes.c_void_p, ctypes.c_long, ctypes.c_long, ctypes.c_double,
                                 ctypes.c_void_p, ctypes.c_long, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_void_p]),
    "t2s2_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "t2s2_mlp_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "t2s2_mlp_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_int)]),
    "t2s2_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "t2s2_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "t2s2_mlp_pack_target": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_TT),
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "t2s2_mlp_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_void_p]),
    "t2s2_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                           ctypes.c_void_p]),
    "t2s2_mlp_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.c_void_p]),
    "t2s2_mlp_init_output": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.c_float,
                                            ctypes.c_void_p]),
    "t2s2_mlp_calibrate_scale": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_void_p]),
    "t2s2_mlp_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_float), ctypes.c_void_p]),
    "t2s2_apply_batched": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_TT), ctypes.POINTER(_TT),
                                          ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_void_p]),
    "t2s2_autotune_report": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int]),
    "t2s2_diff_norm": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.POINTER(_TT),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "t2s2_tt_fibre": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_TT), ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "t2s2_fastmath": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long,
                                     ctypes.c_void_p]),
    "t2s2_kernel_launches": (ctypes.c_longlong, []),
    "t2s2_trace": (ctypes.c_int, [ctypes.c_int]),
    "t2s2_trace_overhead": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "t2s2_trace_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
}

# Kernel families of t2s2_trace_read, in the library's order.
TRACE_FAMILIES = ["gemm", "apply", "local_solve", "small_factor", "elementwise", "apply_tc", "gemm_tc",
                  "mlp", "cholqr", "sylvester", "dots"]


def load():
    """Load libt2s2.so (built in-tree).  Raises if it is missing: no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(lib_path):
        raise RuntimeError(f"{lib_path} is missing; run __graft_entry__.build() first")
    lib = ctypes.CDLL(lib_path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def t2s2_strerror(status: int) -> str:
    try:
        return load().t2s2_strerror(int(status)).decode()
    except Exception:  # library not loadable: still give a message
        return f"status {status}"


def t2s2_device_count() -> int:
    return int(load().t2s2_device_count())


def t2s2_gemm(op: Operator, A, B, C, tA=False, tB=False, alpha=1.0, beta=0.0, prec=FP64, stream=None):
    """C = alpha op(A) op(B) + beta C (t2s2_gemm) on float64 CUDA tensors.

    2-D operands, or 3-D with a leading batch dimension; the last dimension
    of each must be contiguous.  Returns C.
    """
    def lay(t):
        if t.dtype != torch.float64 or (t.numel() > 0 and t.stride(-1) != 1):
            raise ValueError("float64 tensors with a contiguous last dimension expected")
        if t.numel() == 0:  # empty: strides carry no layout
            rows, cols = t.shape[-2], t.shape[-1]
            return rows, cols, cols, 0, (t.shape[0] if t.dim() == 3 else 1)
        if t.dim() == 2:
            return t.shape[0], t.shape[1], t.stride(0), 0, 1
        return t.shape[1], t.shape[2], t.stride(1), t.stride(0), t.shape[0]
    import torch
    ra, ca, lda, sA, ba = lay(A)
    rb, cb, ldb, sB, bb = lay(B)
    rc, cc, ldc, sC, bc = lay(C)
    M, K = (ca, ra) if tA else (ra, ca)
    K2, N = (cb, rb) if tB else (rb, cb)
    if K2 != K or (rc, cc) != (M, N):
        raise ValueError("shape mismatch")
    batch = max(ba, bb, bc)
    _check(load().t2s2_gemm(op.handle, M, N, K, int(tA), int(tB), float(alpha), A.data_ptr(), lda, sA,
                            B.data_ptr(), ldb, sB, float(beta), C.data_ptr(), ldc, sC, batch, int(prec),
                            _stream_handle(stream)), "t2s2_gemm")
    return C


class WarmStartNet:
    """The learned warm start (t2s2_mlp_*): p -> TT cores of an initial guess.

    ``m`` are the interior mode sizes, ``r`` the output rank and ``ru`` the
    largest target rank.  Training data live on the device: ``P`` a float32
    (N, in_dim) tensor, targets packed by :meth:`pack_targets`.
    """

    def __init__(self, in_dim, hidden, m, r, ru, seed=0):
        import torch
        h = ctypes.c_void_p()
        m_arr = (ctypes.c_int * len(m))(*[int(v) for v in m])
        _check(load().t2s2_mlp_create(int(in_dim), int(hidden), len(m), m_arr, int(r), int(ru),
                                      int(seed), ctypes.byref(h)), "t2s2_mlp_create")
        self._h = h
        self.in_dim, self.hidden, self.m, self.r, self.ru = in_dim, hidden, list(m), r, ru
        self.d, self.mmax = len(m), max(m)
        n, od = ctypes.c_longlong(), ctypes.c_int()
        _check(load().t2s2_mlp_info(h, ctypes.byref(n), ctypes.byref(od)), "t2s2_mlp_info")
        self.nparams, self.out_dim = n.value, od.value
        self._torch = torch

    def close(self):
        if self._h:
            load().t2s2_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        t = self._torch.empty(self.nparams, dtype=self._torch.float32, device="cuda")
        _check(load().t2s2_mlp_get_params(self._h, t.data_ptr(), None, _stream_handle(None)),
               "t2s2_mlp_get_params")
        return t

    def grads(self):
        t = self._torch.empty(self.nparams, dtype=self._torch.float32, device="cuda")
        _check(load().t2s2_mlp_get_params(self._h, None, t.data_ptr(), _stream_handle(None)),
               "t2s2_mlp_get_params")
        return t

    def set_params(self, flat):
        t = flat.to(device="cuda", dtype=self._torch.float32).contiguous()
        _check(load().t2s2_mlp_set_params(self._h, t.data_ptr(), _stream_handle(None)), "t2s2_mlp_set_params")

    def pack_targets(self, op: "Operator", tts):
        """Device arrays (targets, uu) for a list of device TTs."""
        n = len(tts)
        per = self.d * self.ru * self.mmax * self.ru
        targets = self._torch.zeros(n * per, dtype=self._torch.float32, device="cuda")
        uu = self._torch.zeros(n, dtype=self._torch.float32, device="cuda")
        for i, u in enumerate(tts):
            s = u._struct()
            _check(load().t2s2_mlp_pack_target(self._h, op.handle, ctypes.byref(s),
                                               targets.data_ptr() + 4 * i * per, uu.data_ptr() + 4 * i,
                                               _stream_handle(None)), "t2s2_mlp_pack_target")
        return targets, uu

    def pack_target_into(self, op: "Operator", u: "TT", targets, uu, i):
        """Pack one device TT into slot i of the arrays of pack_targets."""
        per = self.d * self.ru * self.mmax * self.ru
        if targets.numel() < (i + 1) * per or uu.numel() < i + 1:
            raise ValueError("slot outside the target arrays")
        s = u._struct()
        _check(load().t2s2_mlp_pack_target(self._h, op.handle, ctypes.byref(s),
                                           targets.data_ptr() + 4 * i * per, uu.data_ptr() + 4 * i,
                                           _stream_handle(None)), "t2s2_mlp_pack_target")

    def _batch_ptrs(self, P, targets, uu, lo, hi):
        per = self.d * self.ru * self.mmax * self.ru
        n = P.shape[0]
        if P.dim() != 2 or P.shape[1] != self.in_dim or P.dtype != self._torch.float32 or not P.is_contiguous():
            raise ValueError(f"P must be a contiguous float32 (N, {self.in_dim}) tensor")
        if not (0 <= lo < hi <= n) or targets.numel() < n * per or uu.numel() < n:
            raise ValueError("minibatch outside the training set")
        return (P.data_ptr() + 4 * lo * self.in_dim, targets.data_ptr() + 4 * lo * per, uu.data_ptr() + 4 * lo)

    def loss_grad(self, P, targets, uu, lo=0, hi=None):
        hi = P.shape[0] if hi is None else hi
        pp, tp, up = self._batch_ptrs(P, targets, uu, lo, hi)
        loss = ctypes.c_float()
        _check(load().t2s2_mlp_loss_grad(self._h, pp, hi - lo, tp, up, ctypes.byref(loss), _stream_handle(None)),
               "t2s2_mlp_loss_grad")
        return loss.value

    def init_output_bias(self, op: "Operator", u: "TT", weight_scale=0.1):
        """Start the network's output at a representative target u
        (t2s2_mlp_init_output): the output bias takes the cores of u rounded to
        the network's rank, the output weights are scaled by weight_scale."""
        if u.d != self.d or u.m != self.m:
            raise ValueError("u does not live on the network's grid")
        s = u._struct()
        _check(load().t2s2_mlp_init_output(self._h, op.handle, ctypes.byref(s), float(weight_scale),
                                           _stream_handle(None)), "t2s2_mlp_init_output")

    def calibrate_scale(self, P, targets, uu, lo=0, hi=None):
        """Shift the log-scale bias so that X(p) starts at the targets' size."""
        hi = P.shape[0] if hi is None else hi
        pp, tp, up = self._batch_ptrs(P, targets, uu, lo, hi)
        shift = ctypes.c_float()
        _check(load().t2s2_mlp_calibrate_scale(self._h, pp, hi - lo, tp, up, ctypes.byref(shift),
                                               _stream_handle(None)), "t2s2_mlp_calibrate_scale")
        return shift.value

    def train_step(self, P, targets, uu, lr, lo=0, hi=None):
        hi = P.shape[0] if hi is None else hi
        pp, tp, up = self._batch_ptrs(P, targets, uu, lo, hi)
        loss = ctypes.c_float()
        _check(load().t2s2_mlp_train_step(self._h, pp, hi - lo, tp, up, float(lr), ctypes.byref(loss),
                                          _stream_handle(None)), "t2s2_mlp_train_step")
        return loss.value

    def train(self, P, targets, uu, batch, steps, lr, use_graph=True):
        """`steps` Adam steps cycling through the resident set; returns the last loss."""
        self._batch_ptrs(P, targets, uu, 0, int(batch))  # shape checks
        loss = ctypes.c_float()
        _check(load().t2s2_mlp_train(self._h, P.data_ptr(), int(P.shape[0]), targets.data_ptr(), uu.data_ptr(),
                                     int(batch), int(steps), float(lr), int(bool(use_graph)), ctypes.byref(loss),
                                     _stream_handle(None)), "t2s2_mlp_train")
        return loss.value

    def predict(self, p, x: "TT"):
        """Write the network's guess for parameter vector p (in_dim floats) into x."""
        v = self._torch.as_tensor(np.asarray(p, dtype=np.float32)).contiguous()
        if v.numel() != self.in_dim:
            raise ValueError(f"expected {self.in_dim} parameters, got {v.numel()}")
        s = x._struct()
        _check(load().t2s2_mlp_predict(self._h, v.data_ptr(), ctypes.byref(s), _stream_handle(None)),
               "t2s2_mlp_predict")
        x._sync_ranks()
        return x


def t2s2_fastmath(x):
    """(rsqrt, rcp) of a float64 CUDA tensor by the library's Newton-refined
    FP64 routines (t2s2_fastmath)."""
    import torch
    x = x.to(device="cuda", dtype=torch.float64).contiguous()
    rs, rc = torch.empty_like(x), torch.empty_like(x)
    _check(load().t2s2_fastmath(x.data_ptr(), rs.data_ptr(), rc.data_ptr(), x.numel(), _stream_handle(None)),
           "t2s2_fastmath")
    return rs, rc


def t2s2_kernel_launches() -> int:
    """Kernels this library has launched in this process."""
    return int(load().t2s2_kernel_launches())


def t2s2_trace(enable: bool):
    """Clear the per-family counters; turn CUDA-event timing on or off."""
    _check(load().t2s2_trace(1 if enable else 0), "t2s2_trace")


def t2s2_trace_overhead(n=200, stream=None) -> float:
    """Event-bracketed time (ms) of an empty library-style launch."""
    out = ctypes.c_double()
    _check(load().t2s2_trace_overhead(int(n), _stream_handle(stream), ctypes.byref(out)), "t2s2_trace_overhead")
    return out.value


def t2s2_trace_read(family) -> dict:
    """Launches, event ms, algorithmic FLOPs and bytes of one kernel family."""
    idx = TRACE_FAMILIES.index(family) if isinstance(family, str) else int(family)
    n = ctypes.c_longlong(0)
    ms, fl, by = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(load().t2s2_trace_read(idx, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                  ctypes.byref(by)), "t2s2_trace_read")
    return {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}


def t2s2_dim_matrices(n: int, eps: float, beta: float, kind: int = DIM_SPACE):
    """One dimension's 1D collocation matrices, computed on the host (no
    device): returns dict x (n), eta (m), Rt, Lt (m x m), Rb, Lb (m x nb) with
    m = n-2, nb = 2 for the space kinds and m = n-1, nb = 1 for DIM_TIME."""
    time = kind == DIM_TIME
    m, nb = (n - 1, 1) if time else (n - 2, 2)
    out = {"x": np.zeros(n), "eta": np.zeros(max(m, 0)), "Rt": np.zeros((max(m, 0), max(m, 0))),
           "Lt": np.zeros((max(m, 0), max(m, 0))), "Rb": np.zeros((max(m, 0), nb)),
           "Lb": np.zeros((max(m, 0), nb))}
    _check(load().t2s2_dim_matrices(int(n), float(eps), float(beta), int(kind),
                                    *[out[k].ctypes.data for k in ("x", "eta", "Rt", "Lt", "Rb", "Lb")]),
           "t2s2_dim_matrices")
    return out


def _check(status: int, what: str, ok=(0,)):
    if status not in ok:
        raise T2S2Error(status, what)
    return status


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Operator:
    """Handle on the library's operator (t2s2_build_operator / t2s2_op_destroy)."""

    def __init__(self, handle, d, n, beta, eps, plain_sc, m=None):
        self._h = handle
        self.d, self.n, self.beta, self.eps, self.plain_sc = d, tuple(n), tuple(beta), eps, plain_sc
        self.m = tuple(v - 2 for v in self.n) if m is None else tuple(int(v) for v in m)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("operator destroyed")
        return self._h

    def nodes(self, k):
        x = np.zeros(self.n[k])
        eta = np.zeros(self.m[k])
        _check(load().t2s2_op_nodes(self.handle, k, x.ctypes.data, eta.ctypes.data), "t2s2_op_nodes")
        return x, eta

    def matrices(self, k):
        m = self.m[k]
        Rt = np.zeros((m, m))
        Lt = np.zeros((m, m))
        _check(load().t2s2_op_matrices(self.handle, k, Rt.ctypes.data, Lt.ctypes.data),
               "t2s2_op_matrices")
        return Rt, Lt

    def destroy(self):
        if self._h is not None:
            load().t2s2_op_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def t2s2_build_operator(d, n, beta, eps, plain_sc=False, stream=None) -> Operator:
    lib = load()
    n = [int(v) for v in (n if np.ndim(n) else [n] * d)]
    beta = [float(v) for v in beta]
    na = (ctypes.c_int * d)(*n)
    ba = (ctypes.c_double * d)(*beta)
    prob = _Problem(d, na, ba, float(eps), int(bool(plain_sc)))
    h = ctypes.c_void_p()
    _check(lib.t2s2_build_operator(ctypes.byref(prob), _stream_handle(stream), ctypes.byref(h)),
           "t2s2_build_operator")
    return Operator(h, d, n, beta, float(eps), bool(plain_sc))


def t2s2_build_operator_var(d, n, beta_ref, eps, beta_fns=None, rho_fns=None, rho0=0.0, plain_sc=False,
                            stream=None, prod_fns=None) -> Operator:
    """Operator with variable coefficients: beta_fns[k](x) (vectorised over
    numpy arrays or scalar; None: the constant beta_ref[k]) and the reaction
    rho0 + sum_k rho_fns[k](x_k) + prod_k prod_fns[k](x_k).  beta_ref[k] picks
    dimension k's superconsistent points."""
    lib = load()
    n = [int(v) for v in (n if np.ndim(n) else [n] * d)]
    beta_ref = [float(v) for v in beta_ref]
    na = (ctypes.c_int * d)(*n)
    ba = (ctypes.c_double * d)(*beta_ref)

    def wrap(fns, default):
        if fns is None:
            return _COEF_FN()
        def f(k, x, _ctx):
            g = fns[k]
            return float(default(k) if g is None else g(np.float64(x)))
        return _COEF_FN(f)

    bfn = wrap(beta_fns, lambda k: beta_ref[k])
    rfn = wrap(rho_fns, lambda k: 0.0)
    pfn = wrap(prod_fns, lambda k: 1.0)
    prob = _ProblemVar(_Problem(d, na, ba, float(eps), int(bool(plain_sc))), bfn, rfn, float(rho0), None, pfn)
    h = ctypes.c_void_p()
    _check(lib.t2s2_build_operator_var(ctypes.byref(prob), _stream_handle(stream), ctypes.byref(h)),
           "t2s2_build_operator_var")
    return Operator(h, d, n, beta_ref, float(eps), bool(plain_sc))


def t2s2_build_spacetime_operator(d, n, beta, eps, n_t, t_len, plain_sc=False, stream=None) -> Operator:
    """Operator of the unified space-time form: time (n_t nodes, n_t - 1
    unknowns, interval length t_len) as dimension 0, then the d spatial
    dimensions of t2s2_build_operator."""
    lib = load()
    n = [int(v) for v in (n if np.ndim(n) else [n] * d)]
    beta = [float(v) for v in beta]
    na = (ctypes.c_int * d)(*n)
    ba = (ctypes.c_double * d)(*beta)
    prob = _Problem(d, na, ba, float(eps), int(bool(plain_sc)))
    h = ctypes.c_void_p()
    _check(lib.t2s2_build_spacetime_operator(ctypes.byref(prob), int(n_t), float(t_len), _stream_handle(stream),
                                             ctypes.byref(h)), "t2s2_build_spacetime_operator")
    return Operator(h, d + 1, [int(n_t)] + n, [2.0 / float(t_len)] + beta, float(eps), bool(plain_sc),
                    m=[int(n_t) - 1] + [v - 2 for v in n])


def t2s2_spacetime_rhs(op: Operator, b: "TT", u0: "TT", out: "TT", tol: float, rmax: int, stream=None):
    """out = round(b - L0 (x) M_x u0 - R0 (x) A_x u0): the space-time right-hand
    side with the initial condition u0 lifted (op from
    t2s2_build_spacetime_operator)."""
    sb, su, so = b._struct(), u0._struct(), out._struct()
    _check(load().t2s2_spacetime_rhs(op.handle, ctypes.byref(sb), ctypes.byref(su), ctypes.byref(so),
                                     float(tol), int(rmax), _stream_handle(stream)), "t2s2_spacetime_rhs")
    out._sync_ranks()
    return out


class TT:
    """A tensor train whose cores live in torch tensors (device or pinned host).

    Core k holds r[k] * m[k] * r[k+1] doubles ([r_k][m_k][r_{k+1}] row-major)
    inside a buffer of capacity ``cap[k]``.
    """

    def __init__(self, m, r, buffers, loc):
        self.d = len(m)
        self.m = [int(v) for v in m]
        self.r = [int(v) for v in r]
        self.buffers = buffers
        self.loc = loc

    @classmethod
    def empty(cls, m, rcap, device="cuda", ranks=None):
        import torch
        d = len(m)
        bufs = []
        for k in range(d):
            a = 1 if k == 0 else rcap
            b = 1 if k == d - 1 else rcap
            if device == "cpu":
                bufs.append(torch.zeros(a * m[k] * b, dtype=torch.float64).pin_memory())
            else:
                bufs.append(torch.zeros(a * m[k] * b, dtype=torch.float64, device=device))
        r = ranks if ranks is not None else [1] * (d + 1)
        return cls(m, r, bufs, _HOST if device == "cpu" else _DEVICE)

    @classmethod
    def from_cores(cls, cores, rcap=None, device="cuda"):
        import torch
        m = [c.shape[1] for c in cores]
        r = [cores[0].shape[0]] + [c.shape[2] for c in cores]
        rcap = max(r) if rcap is None else max(rcap, max(r))
        t = cls.empty(m, rcap, device=device, ranks=r)
        for k, c in enumerate(cores):
            flat = torch.from_numpy(np.ascontiguousarray(c, dtype=np.float64).ravel())
            t.buffers[k][: flat.numel()].copy_(flat)
        return t

    def cores(self):
        out = []
        for k in range(self.d):
            n = self.r[k] * self.m[k] * self.r[k + 1]
            out.append(self.buffers[k][:n].detach().cpu().numpy().reshape(self.r[k], self.m[k],
                                                                            self.r[k + 1]).copy())
        return out

    def _struct(self):
        d = self.d
        self._m_arr = (ctypes.c_int * d)(*self.m)
        self._r_arr = (ctypes.c_int * (d + 1))(*self.r)
        self._p_arr = (ctypes.c_void_p * d)(*[b.data_ptr() for b in self.buffers])
        self._c_arr = (ctypes.c_size_t * d)(*[b.numel() for b in self.buffers])
        self._s = _TT(d, self._m_arr, self._r_arr, self._p_arr, self._c_arr, self.loc)
        return self._s

    def _sync_ranks(self):
        self.r = [int(self._r_arr[k]) for k in range(self.d + 1)]


def t2s2_apply(op: Operator, x: TT, y: TT, c_mass=0.0, c_op=1.0, prec=FP64, stream=None):
    sx, sy = x._struct(), y._struct()
    _check(load().t2s2_apply(op.handle, ctypes.byref(sx), ctypes.byref(sy), float(c_mass),
                             float(c_op), int(prec), _stream_handle(stream)), "t2s2_apply")
    y._sync_ranks()
    return y


def t2s2_apply_batched(ops, xs, ys, c_mass=0.0, c_op=1.0, prec=FP64, stream=None):
    """Grouped apply over many instances in one persistent launch."""
    n = len(ops)
    if not (len(xs) == len(ys) == n):
        raise ValueError("ops, xs and ys must have the same length")
    h = (ctypes.c_void_p * n)(*[o.handle for o in ops])
    sx = (_TT * n)(*[x._struct() for x in xs])
    sy = (_TT * n)(*[y._struct() for y in ys])
    _check(load().t2s2_apply_batched(h, sx, sy, n, float(c_mass), float(c_op), int(prec),
                                     _stream_handle(stream)), "t2s2_apply_batched")
    for y, s in zip(ys, sy):
        y.r = [int(s.r[k]) for k in range(y.d + 1)]
    return ys


def t2s2_autotune_report() -> str:
    """The grouped apply's tuned launch shapes, one line per shape class."""
    n = load().t2s2_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    load().t2s2_autotune_report(buf, n + 1)
    return buf.value.decode()


def t2s2_round(op: Operator, x: TT, tol, rmax=0, stream=None):
    sx = x._struct()
    _check(load().t2s2_round(op.handle, ctypes.byref(sx), float(tol), int(rmax),
                             _stream_handle(stream)), "t2s2_round")
    x._sync_ranks()
    return x


def t2s2_tt_fibre(op: Operator, x: TT, mode: int, idx, stream=None) -> np.ndarray:
    """x along `mode` with the other indices fixed at idx (d entries)."""
    ia = (ctypes.c_int * x.d)(*[int(v) for v in idx])
    out = np.zeros(x.m[mode] if 0 <= mode < x.d else 1)
    _check(load().t2s2_tt_fibre(op.handle, ctypes.byref(x._struct()), int(mode), ia, out.ctypes.data,
                                _stream_handle(stream)), "t2s2_tt_fibre")
    return out


def t2s2_norm(op: Operator, x: TT, stream=None) -> float:
    out = ctypes.c_double()
    _check(load().t2s2_norm(op.handle, ctypes.byref(x._struct()), ctypes.byref(out),
                            _stream_handle(stream)), "t2s2_norm")
    return out.value


def t2s2_diff_norm(op: Operator, x: TT, y: TT, stream=None) -> float:
    """||x - y||_F through the TT difference (accurate for nearly equal x, y)."""
    out = ctypes.c_double()
    _check(load().t2s2_diff_norm(op.handle, ctypes.byref(x._struct()), ctypes.byref(y._struct()),
                                 ctypes.byref(out), _stream_handle(stream)), "t2s2_diff_norm")
    return out.value


def t2s2_norm_noalloc(x: TT, stream=None) -> float:
    """||x||_F without any device allocation (static scratch; see t2s2.h)."""
    out = ctypes.c_double()
    _check(load().t2s2_norm_noalloc(ctypes.byref(x._struct()), ctypes.byref(out),
                                    _stream_handle(stream)), "t2s2_norm_noalloc")
    return out.value


def t2s2_residual(op: Operator, b: TT, x: TT, c_mass=0.0, c_op=1.0, stream=None) -> float:
    out = ctypes.c_double()
    sb, sx = b._struct(), x._struct()
    _check(load().t2s2_residual(op.handle, ctypes.byref(sb), ctypes.byref(sx), float(c_mass),
                                float(c_op), ctypes.byref(out), _stream_handle(stream)),
           "t2s2_residual")
    return out.value


def _info(status, info):
    return SolveInfo(status, info.residual, info.sweeps, info.max_rank, info.refinements,
                     info.local_iters)


def t2s2_solve(op: Operator, b: TT, x: TT, tol, rmax, max_sweeps=50, prec=FP64, c_mass=0.0,
               c_op=1.0, stream=None, allow_noconv=False) -> SolveInfo:
    info = _Info()
    sb, sx = b._struct(), x._struct()
    st = load().t2s2_solve(op.handle, ctypes.byref(sb), ctypes.byref(sx), float(c_mass),
                           float(c_op), float(tol), int(rmax), int(max_sweeps), int(prec),
                           _stream_handle(stream), ctypes.byref(info))
    _check(st, "t2s2_solve", ok=(0, 4) if allow_noconv else (0,))
    x._sync_ranks()
    return _info(st, info)


def t2s2_solve_batched(ops, bs, xs, tol, rmax, max_sweeps=50, prec=FP64, workers=8,
                       allow_noconv=False):
    """Solve len(ops) independent steady problems concurrently; returns SolveInfo per instance."""
    n = len(ops)
    harr = (ctypes.c_void_p * n)(*[o.handle.value if hasattr(o.handle, "value") else o.handle for o in ops])
    barr = (_TT * n)(*[b._struct() for b in bs])
    xarr = (_TT * n)(*[x._struct() for x in xs])
    infos = (_Info * n)()
    sts = (ctypes.c_int * n)()
    st = load().t2s2_solve_batched(harr, barr, xarr, n, float(tol), int(rmax), int(max_sweeps), int(prec),
                                   int(workers), infos, sts)
    _check(st, "t2s2_solve_batched", ok=(0, 4) if allow_noconv else (0,))
    for i, x in enumerate(xs):
        x.r = [int(xarr[i].r[k]) for k in range(x.d + 1)]
    return [_info(sts[i], infos[i]) for i in range(n)]


def t2s2_dirichlet_rhs(op: Operator, b: TT, g: TT, out: TT, tol, rmax=0, c_mass=0.0, c_op=1.0, stream=None):
    """out = round(b - (c_mass M_full + c_op A_full) g): the source of the
    zero-data correction for Dirichlet data g (a TT on the full GLL grid)."""
    sb, sg, so = b._struct(), g._struct(), out._struct()
    _check(load().t2s2_dirichlet_rhs(op.handle, ctypes.byref(sb), ctypes.byref(sg), float(c_mass), float(c_op),
                                     ctypes.byref(so), float(tol), int(rmax), _stream_handle(stream)),
           "t2s2_dirichlet_rhs")
    out._sync_ranks()
    return out


def t2s2_solve_dirichlet(op: Operator, b: TT, g, x: TT, tol, rmax, max_sweeps=50, prec=FP64, c_mass=0.0,
                         c_op=1.0, stream=None, allow_noconv=False) -> SolveInfo:
    """Solve with Dirichlet data g (a full-grid TT, or None for zero data);
    x: initial guess in, interior values of u out."""
    info = _Info()
    sb, sx = b._struct(), x._struct()
    gp = ctypes.byref(g._struct()) if g is not None else None
    st = load().t2s2_solve_dirichlet(op.handle, ctypes.byref(sb), gp, ctypes.byref(sx), float(c_mass),
                                     float(c_op), float(tol), int(rmax), int(max_sweeps), int(prec),
                                     _stream_handle(stream), ctypes.byref(info))
    _check(st, "t2s2_solve_dirichlet", ok=(0, 4) if allow_noconv else (0,))
    x._sync_ranks()
    return _info(st, info)


def t2s2_cn_step(op: Operator, u: TT, dt, tol, rmax, prec=FP64, stream=None) -> SolveInfo:
    info = _Info()
    su = u._struct()
    st = load().t2s2_cn_step(op.handle, ctypes.byref(su), float(dt), float(tol), int(rmax),
                             int(prec), _stream_handle(stream), ctypes.byref(info))
    _check(st, "t2s2_cn_step")
    u._sync_ranks()
    return _info(st, info)


def t2s2_be_step(op: Operator, u: TT, dt, tol, rmax, prec=FP64, stream=None) -> SolveInfo:
    info = _Info()
    su = u._struct()
    st = load().t2s2_be_step(op.handle, ctypes.byref(su), float(dt), float(tol), int(rmax),
                             int(prec), _stream_handle(stream), ctypes.byref(info))
    _check(st, "t2s2_be_step")
    u._sync_ranks()
    return _info(st, info)
