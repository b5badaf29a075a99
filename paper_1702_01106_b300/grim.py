"""Thin ctypes binding of libgrim.so (include/grim.h), argument marshalling only.

Every step of the path runs in the library's CUDA kernels; PyTorch provides
device memory and streams.  The library is loaded on first use and a missing
library is an error: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrim.so")

GRIM_FP64, GRIM_MIXED = 0, 1

_lib = None

# Names every build of libgrim.so exports (the declarations of include/grim.h).
EXPORTS = (
    "grim_init", "grim_step", "grim_step_host", "grim_stage", "grim_residual", "grim_get_stats",
    "grim_reset_stats", "grim_last_error", "grim_strerror", "grim_destroy", "grim_peak_flops",
    "grim_profile", "grim_kernel_times", "grim_step_static", "grim_step_static_stats", "grim_math_selftest",
    "grim_mlp_create", "grim_mlp_destroy", "grim_mlp_param_count", "grim_mlp_get_params", "grim_mlp_set_params",
    "grim_mlp_fit_norm", "grim_mlp_train", "grim_mlp_gradient", "grim_mlp_sample", "grim_set_guess",
    "grim_gemm_nt_bf16",
    "grim_get_tuning", "grim_set_tuning", "grim_autotune", "grim_use_graphs",
    "grim_batch_init", "grim_batch_destroy", "grim_batch_context", "grim_batch_step", "grim_batch_use_graphs",
    "grim_batch_get_stats", "grim_batch_reset_stats", "grim_batch_last_error",
)
STATIC_MAX_ZONES = 65536
KERNEL_CLASSES = ("explicit", "newton64", "newton32", "residual", "faces", "zone_const", "mlp")


class GrimGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
                ("x_start", ctypes.c_double * 3), ("x_end", ctypes.c_double * 3),
                ("bc", (ctypes.c_int * 2) * 3)]


class GrimMetric(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("spin", ctypes.c_double), ("h", ctypes.c_double)]


class GrimPhysics(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("tau_R", ctypes.c_double), ("phi", ctypes.c_double),
                ("psi", ctypes.c_double), ("conduction", ctypes.c_int), ("viscosity", ctypes.c_int),
                ("higher_order", ctypes.c_int), ("recon", ctypes.c_int), ("theta", ctypes.c_double),
                ("floors", ctypes.c_int), ("riemann", ctypes.c_int)]


class GrimSolver(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("eps_fd", ctypes.c_double),
                ("eps_fd32", ctypes.c_double), ("k_max", ctypes.c_int), ("ls_max", ctypes.c_int),
                ("fd32_central", ctypes.c_int)]


class GrimTuning(ctypes.Structure):
    _fields_ = [("newton_bs", ctypes.c_int), ("newton_kcut", ctypes.c_int), ("faces_bs", ctypes.c_int),
                ("zone_bs", ctypes.c_int), ("newton_rounds", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GrimStats(ctypes.Structure):
    _fields_ = [("zones", ctypes.c_ulonglong), ("failed", ctypes.c_ulonglong), ("iters", ctypes.c_ulonglong),
                ("evals64", ctypes.c_ulonglong), ("evals32", ctypes.c_ulonglong), ("lu64", ctypes.c_ulonglong),
                ("lu32", ctypes.c_ulonglong), ("hist", ctypes.c_ulonglong * 32), ("max_res", ctypes.c_double),
                ("launches", ctypes.c_ulonglong), ("fallbacks", ctypes.c_ulonglong),
                ("rescued", ctypes.c_ulonglong), ("mlp_stalls", ctypes.c_ulonglong)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "hist"}
        d["hist"] = list(self.hist)
        return d


def load():
    """Load libgrim.so; raises if it is missing (build it with build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgrim.so not found at {LIB_PATH}: build it first "
                           "(python -m paper_1702_01106_b300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    lib.grim_init.argtypes = [ctypes.POINTER(GrimGrid), ctypes.POINTER(GrimMetric), ctypes.POINTER(GrimPhysics),
                              ctypes.POINTER(GrimSolver), vp, ctypes.POINTER(vp)]
    lib.grim_step.argtypes = [vp, vp, vp, dp]
    lib.grim_step_host.argtypes = [vp, vp, vp, dp]
    lib.grim_stage.argtypes = [vp, vp, vp, dp, vp, vp, vp, vp]
    lib.grim_residual.argtypes = [vp, vp, vp, dp, vp, i, vp]
    lib.grim_get_stats.argtypes = [vp, ctypes.POINTER(GrimStats)]
    lib.grim_reset_stats.argtypes = [vp]
    lib.grim_last_error.argtypes = [vp]
    lib.grim_last_error.restype = ctypes.c_char_p
    lib.grim_strerror.argtypes = [i]
    lib.grim_strerror.restype = ctypes.c_char_p
    lib.grim_destroy.argtypes = [vp]
    lib.grim_destroy.restype = None
    lib.grim_peak_flops.argtypes = [ctypes.POINTER(dp), ctypes.POINTER(dp)]
    lib.grim_step_static.argtypes = [ctypes.POINTER(GrimGrid), ctypes.POINTER(GrimMetric),
                                     ctypes.POINTER(GrimPhysics), ctypes.POINTER(GrimSolver), vp, vp, vp, dp]
    lib.grim_step_static_stats.argtypes = [vp, ctypes.POINTER(GrimStats)]
    lib.grim_profile.argtypes = [vp, i]
    lib.grim_math_selftest.argtypes = [i, ctypes.POINTER(dp)]
    ll, ull, fp = ctypes.c_longlong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_float)
    lib.grim_mlp_create.argtypes = [ull, ctypes.POINTER(vp)]
    lib.grim_mlp_destroy.argtypes = [vp]
    lib.grim_mlp_destroy.restype = None
    lib.grim_mlp_get_params.argtypes = [vp, vp, vp]
    lib.grim_mlp_set_params.argtypes = [vp, vp, vp]
    lib.grim_mlp_fit_norm.argtypes = [vp, vp, vp, ll]
    lib.grim_mlp_train.argtypes = [vp, vp, vp, ll, i, i, dp, ull, ctypes.POINTER(dp)]
    lib.grim_mlp_gradient.argtypes = [vp, vp, vp, ll, vp, ctypes.POINTER(dp)]
    lib.grim_mlp_sample.argtypes = [vp, vp, vp, vp, vp]
    lib.grim_gemm_nt_bf16.argtypes = [i, i, i, vp, i, vp, i, vp, i, i]
    lib.grim_set_guess.argtypes = [vp, vp, dp]
    lib.grim_kernel_times.argtypes = [vp, ctypes.POINTER(dp), ctypes.POINTER(ctypes.c_ulonglong)]
    lib.grim_get_tuning.argtypes = [vp, ctypes.POINTER(GrimTuning)]
    lib.grim_set_tuning.argtypes = [vp, ctypes.POINTER(GrimTuning)]
    lib.grim_autotune.argtypes = [vp, vp, dp, ctypes.c_char_p, ctypes.POINTER(GrimTuning), ctypes.POINTER(dp)]
    lib.grim_use_graphs.argtypes = [vp, i]
    lib.grim_batch_init.argtypes = [i, ctypes.POINTER(GrimGrid), ctypes.POINTER(GrimMetric),
                                    ctypes.POINTER(GrimPhysics), ctypes.POINTER(GrimSolver), vp, ctypes.POINTER(vp)]
    lib.grim_batch_destroy.argtypes = [vp]
    lib.grim_batch_destroy.restype = None
    lib.grim_batch_context.argtypes = [vp, i, ctypes.POINTER(vp)]
    lib.grim_batch_step.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(dp)]
    lib.grim_batch_use_graphs.argtypes = [vp, i]
    lib.grim_batch_get_stats.argtypes = [vp, ctypes.POINTER(GrimStats)]
    lib.grim_batch_reset_stats.argtypes = [vp]
    lib.grim_batch_last_error.argtypes = [vp]
    lib.grim_batch_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _f64(t):
    import torch
    if t is not None and t.dtype != torch.float64:
        raise ValueError("expected float64")
    return _ptr(t)


EPS_FD32 = 2.0 ** -7      # float32 Jacobian step (measured optimum with centred differences)
FD32_CENTRAL = 1


def _config(prob, precision, eps_fd32, fd32_central=FD32_CENTRAL):
    g = GrimGrid(prob.dim, prob.n[0], prob.n[1], prob.n[2],
                 (ctypes.c_double * 3)(*prob.x_start), (ctypes.c_double * 3)(*prob.x_end),
                 ((ctypes.c_int * 2) * 3)(*[(ctypes.c_int * 2)(*b) for b in prob.bc]))
    m = GrimMetric(prob.metric, prob.spin, prob.h_mks)
    ph = GrimPhysics(prob.gamma, prob.tau_R, prob.phi, prob.psi, int(prob.conduction), int(prob.viscosity),
                     int(prob.higher_order), prob.recon, prob.theta, int(prob.floors), int(prob.riemann))
    sv = GrimSolver(precision, prob.tol, prob.eps_fd, eps_fd32, prob.k_max, prob.ls_max, int(fd32_central))
    return g, m, ph, sv


def step_static(prob, P_in, P_out, dt: float, precision: int = GRIM_FP64, stream=None,
                eps_fd32: float = EPS_FD32, fd32_central: int = FD32_CENTRAL) -> int:
    """grim_step_static: one step with the library's static scratch (no device
    allocation), for callers that cannot call cudaMalloc.  Returns the C code."""
    import torch
    lib = load()
    g, m, ph, sv = _config(prob, precision, eps_fd32, fd32_central)
    if stream is None:
        stream = torch.cuda.current_stream()
    return lib.grim_step_static(ctypes.byref(g), ctypes.byref(m), ctypes.byref(ph), ctypes.byref(sv),
                                ctypes.c_void_p(stream.cuda_stream), _f64(P_in), _f64(P_out), dt)


def step_static_stats(stream=None) -> dict:
    """grim_step_static_stats: the counters of the last grim_step_static call
    on the current device (waits for the stream)."""
    import torch
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream()
    s = GrimStats()
    rc = lib.grim_step_static_stats(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(s))
    if rc != 0:
        raise RuntimeError(f"grim_step_static_stats: {lib.grim_strerror(rc).decode()}")
    return s.as_dict()


class Grim:
    """One context of the library (grim_init ... grim_destroy)."""

    def __init__(self, prob, precision: int = GRIM_FP64, stream=None, eps_fd32: float = EPS_FD32,
                 fd32_central: int = FD32_CENTRAL):
        import torch
        self.lib = load()
        self.prob = prob
        g, m, ph, sv = _config(prob, precision, eps_fd32, fd32_central)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.grim_init(ctypes.byref(g), ctypes.byref(m), ctypes.byref(ph), ctypes.byref(sv),
                                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"grim_init failed: {self.lib.grim_strerror(rc).decode()}")
        self.h = h

    def _check(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} failed ({self.lib.grim_strerror(rc).decode()}): "
                               f"{self.lib.grim_last_error(self.h).decode()}")

    def step(self, P_in, P_out, dt: float):
        self._check(self.lib.grim_step(self.h, _f64(P_in), _f64(P_out), dt), "grim_step")

    def step_host(self, P_in_host, P_out_host, dt: float):
        """grim_step on host tensors (pinned for asynchronous copies)."""
        self._check(self.lib.grim_step_host(self.h, ctypes.c_void_p(P_in_host.data_ptr()),
                                            ctypes.c_void_p(P_out_host.data_ptr()), dt), "grim_step_host")

    def stage(self, P_n, P_E, dts: float, P_out, guess=None, iters=None, status=None):
        self._check(self.lib.grim_stage(self.h, _f64(P_n), _f64(P_E), dts, _f64(guess), _f64(P_out),
                                        _ptr(iters), _ptr(status)), "grim_stage")

    def residual(self, P_n, P_E, dts: float, P_k, R_out, scaled: bool = True):
        self._check(self.lib.grim_residual(self.h, _f64(P_n), _f64(P_E), dts, _f64(P_k), int(scaled),
                                           _f64(R_out)), "grim_residual")

    def stats(self) -> dict:
        s = GrimStats()
        self._check(self.lib.grim_get_stats(self.h, ctypes.byref(s)), "grim_get_stats")
        return s.as_dict()

    def profile(self, enable: bool = True):
        self._check(self.lib.grim_profile(self.h, int(enable)), "grim_profile")

    def kernel_times(self) -> dict:
        """{class: (total ms, launches)} since the last read (synchronises)."""
        ms = (ctypes.c_double * 8)()
        n = (ctypes.c_ulonglong * 8)()
        self._check(self.lib.grim_kernel_times(self.h, ms, n), "grim_kernel_times")
        return {KERNEL_CLASSES[k]: (ms[k], n[k]) for k in range(len(KERNEL_CLASSES)) if n[k]}

    def set_guess(self, mlp, accept: float = 1e-7):
        """Start Newton from the MLP's prediction (None: from P_n)."""
        self._check(self.lib.grim_set_guess(self.h, mlp.h if mlp is not None else None, accept), "grim_set_guess")
        self._mlp = mlp

    def mlp_sample(self, P_n, P_conv, X, Y=None):
        """Features (and targets) of the last explicit stage into float32 X [N, 32], Y [N, 16]."""
        self._check(self.lib.grim_mlp_sample(self.h, _f64(P_n), _f64(P_conv) if P_conv is not None else None,
                                             _ptr(X), _ptr(Y)), "grim_mlp_sample")

    def reset_stats(self):
        self._check(self.lib.grim_reset_stats(self.h), "grim_reset_stats")

    def tuning(self) -> dict:
        t = GrimTuning()
        self._check(self.lib.grim_get_tuning(self.h, ctypes.byref(t)), "grim_get_tuning")
        return t.as_dict()

    def set_tuning(self, **kw):
        """Change fields of the launch shape (newton_bs, newton_kcut, faces_bs, zone_bs, newton_rounds)."""
        t = GrimTuning(**{**self.tuning(), **kw})
        self._check(self.lib.grim_set_tuning(self.h, ctypes.byref(t)), "grim_set_tuning")

    def autotune(self, P, dt: float, cache_path=None):
        """grim_autotune: (tuning dict, step ms)."""
        t, ms = GrimTuning(), ctypes.c_double()
        path = cache_path.encode() if cache_path else None
        self._check(self.lib.grim_autotune(self.h, _f64(P), dt, path, ctypes.byref(t), ctypes.byref(ms)),
                    "grim_autotune")
        return t.as_dict(), ms.value

    def use_graphs(self, enable: bool = True):
        self._check(self.lib.grim_use_graphs(self.h, int(enable)), "grim_use_graphs")

    def close(self):
        if getattr(self, "h", None):
            self.lib.grim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent boxes stepped together (grim_batch_*): probs share
    metric, physics and solver settings; grids may differ."""

    def __init__(self, probs, precision: int = GRIM_FP64, stream=None, eps_fd32: float = EPS_FD32,
                 fd32_central: int = FD32_CENTRAL):
        import torch
        self.lib = load()
        cfgs = [_config(p, precision, eps_fd32, fd32_central) for p in probs]
        grids = (GrimGrid * len(probs))(*[c[0] for c in cfgs])
        _, m, ph, sv = cfgs[0]
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.n = len(probs)
        h = ctypes.c_void_p()
        rc = self.lib.grim_batch_init(self.n, grids, ctypes.byref(m), ctypes.byref(ph), ctypes.byref(sv),
                                      ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"grim_batch_init failed: {self.lib.grim_strerror(rc).decode()}")
        self.h = h
        self._keep = []

    def _check(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} failed ({self.lib.grim_strerror(rc).decode()}): "
                               f"{self.lib.grim_batch_last_error(self.h).decode()}")

    def step(self, P_in, P_out, dts):
        vp = ctypes.c_void_p
        pin = (vp * self.n)(*[_f64(t) for t in P_in])
        pout = (vp * self.n)(*[_f64(t) for t in P_out])
        d = (ctypes.c_double * self.n)(*dts)
        self._check(self.lib.grim_batch_step(self.h, pin, pout, d), "grim_batch_step")

    def use_graphs(self, enable: bool = True):
        self._check(self.lib.grim_batch_use_graphs(self.h, int(enable)), "grim_batch_use_graphs")

    def set_guess(self, mlp, accept: float = 1e-3):
        for i in range(self.n):
            c = ctypes.c_void_p()
            self._check(self.lib.grim_batch_context(self.h, i, ctypes.byref(c)), "grim_batch_context")
            rc = self.lib.grim_set_guess(c, mlp.h if mlp is not None else None, accept)
            if rc != 0:
                raise RuntimeError("grim_set_guess failed")
        self._mlp = mlp

    def stats(self) -> dict:
        s = GrimStats()
        self._check(self.lib.grim_batch_get_stats(self.h, ctypes.byref(s)), "grim_batch_get_stats")
        return s.as_dict()

    def reset_stats(self):
        self._check(self.lib.grim_batch_reset_stats(self.h), "grim_batch_reset_stats")

    def close(self):
        if getattr(self, "h", None):
            self.lib.grim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def peak_flops():
    """(fp64, fp32) FMA throughput of the current device in TFLOP/s."""
    lib = load()
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = lib.grim_peak_flops(ctypes.byref(a), ctypes.byref(b))
    if rc != 0:
        raise RuntimeError(f"grim_peak_flops failed: {lib.grim_strerror(rc).decode()}")
    return a.value, b.value


def math_selftest(n: int = 1 << 20) -> float:
    """Largest relative difference of the kernels' float64 reciprocal from IEEE division."""
    lib = load()
    out = ctypes.c_double()
    rc = lib.grim_math_selftest(n, ctypes.byref(out))
    if rc != 0:
        raise RuntimeError(f"grim_math_selftest failed: {lib.grim_strerror(rc).decode()}")
    return out.value


def gemm_nt_bf16(A, B, splits: int = 0, out=None):
    """C = A B^T on the tensor cores (grim_gemm_nt_bf16): A [M][K] and B [N][K]
    bfloat16 CUDA tensors with unit column stride, C float32 [M][N]."""
    import torch
    lib = load()
    for t in (A, B):
        if not t.is_cuda or t.dtype != torch.bfloat16 or t.dim() != 2 or t.stride(1) != 1:
            raise ValueError("expected 2-D bfloat16 CUDA matrices with unit column stride")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A and B differ in K")
    C = torch.empty((M, N), dtype=torch.float32, device=A.device) if out is None else out
    rc = lib.grim_gemm_nt_bf16(M, N, K, ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                               B.stride(0), ctypes.c_void_p(C.data_ptr()), C.stride(0), splits)
    if rc != 0:
        raise RuntimeError(f"grim_gemm_nt_bf16 failed: {lib.grim_strerror(rc).decode()}")
    return C


class MLP:
    """Learned initial guess (grim_mlp_*): training and parameters on the device."""

    def __init__(self, seed: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.grim_mlp_create(seed, ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"grim_mlp_create failed: {self.lib.grim_strerror(rc).decode()}")
        self.h = h
        self.nparam = int(self.lib.grim_mlp_param_count())

    def _check(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} failed: {self.lib.grim_strerror(rc).decode()}")

    def get_params(self):
        p = np.empty(self.nparam, dtype=np.float32)
        n = np.empty(96, dtype=np.float32)
        self._check(self.lib.grim_mlp_get_params(self.h, p.ctypes.data_as(ctypes.c_void_p),
                                                 n.ctypes.data_as(ctypes.c_void_p)), "grim_mlp_get_params")
        return p, n

    def set_params(self, params=None, norm=None):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        n = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        self._check(self.lib.grim_mlp_set_params(self.h, p.ctypes.data_as(ctypes.c_void_p) if p is not None else None,
                                                 n.ctypes.data_as(ctypes.c_void_p) if n is not None else None),
                    "grim_mlp_set_params")

    def fit_norm(self, X, Y):
        self._check(self.lib.grim_mlp_fit_norm(self.h, _ptr(X), _ptr(Y), X.shape[0]), "grim_mlp_fit_norm")

    def train(self, X, Y, steps: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0) -> float:
        loss = ctypes.c_double()
        self._check(self.lib.grim_mlp_train(self.h, _ptr(X), _ptr(Y), X.shape[0], batch, steps, lr, seed,
                                            ctypes.byref(loss)), "grim_mlp_train")
        return loss.value

    def gradient(self, X, Y):
        g = np.empty(self.nparam, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self.lib.grim_mlp_gradient(self.h, _ptr(X), _ptr(Y), X.shape[0],
                                               g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss)),
                    "grim_mlp_gradient")
        return g, loss.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.grim_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
