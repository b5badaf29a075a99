"""ctypes front end of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

The oracle is a plain restatement of the paper's scheme (grim_oracle.cpp).
Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
it; the product library never imports it.

Parameter vectors passed to the C++ side:
  ip = [dim, n1, n2, n3, bc1lo, bc1hi, bc2lo, bc2hi, bc3lo, bc3hi, metric,
        recon, conduction, viscosity, higher_order, k_max, ls_max, floors, riemann,
        nthreads]
  dp = [x0_1, x0_2, x0_3, dx1, dx2, dx3, gamma, phi, psi, tau_R, theta, tol,
        eps_fd, spin, h_mks]
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

I_COUNT = 20
D_COUNT = 15
ST_MAXIT, ST_LSSTALL, ST_SINGULAR, ST_NONFINITE, ST_INADMISSIBLE = 1, 2, 4, 8, 16


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def params(prob, threads: int = 0):
    ip = np.array([prob.dim, prob.n[0], prob.n[1], prob.n[2],
                   prob.bc[0][0], prob.bc[0][1], prob.bc[1][0], prob.bc[1][1],
                   prob.bc[2][0], prob.bc[2][1], prob.metric, prob.recon,
                   int(prob.conduction), int(prob.viscosity), int(prob.higher_order),
                   prob.k_max, prob.ls_max, int(prob.floors), prob.riemann, threads], dtype=np.int32)
    dx = prob.dx
    dp = np.array([prob.x_start[0], prob.x_start[1], prob.x_start[2], dx[0], dx[1], dx[2],
                   prob.gamma, prob.phi, prob.psi, prob.tau_R, prob.theta, prob.tol,
                   prob.eps_fd, prob.spin, prob.h_mks], dtype=np.float64)
    assert ip.size == I_COUNT and dp.size == D_COUNT
    return ip, dp


def _c(P):
    return np.ascontiguousarray(P, dtype=np.float64)


def stage(prob, Pn, PE, dts, guess=None, threads: int = 0):
    """One stage solve; returns (P_out, iters, status, residual_evals)."""
    ip, dp = params(prob, threads)
    Pn, PE = _c(Pn), _c(PE)
    out = np.empty_like(Pn)
    it = np.zeros(prob.zones, dtype=np.int32)
    st = np.zeros(prob.zones, dtype=np.int32)
    ev = ctypes.c_longlong(0)
    g = _c(guess) if guess is not None else None
    lib().oracle_stage(_iptr(ip), _dptr(dp), _dptr(Pn), _dptr(PE), ctypes.c_double(dts),
                       _dptr(g) if g is not None else None, _dptr(out), _iptr(it), _iptr(st),
                       ctypes.byref(ev))
    return out, it, st, ev.value


def step(prob, Pn, dt, threads: int = 0):
    """One full step (half + full stage); returns (P_out, iters, status, evals)."""
    ip, dp = params(prob, threads)
    Pn = _c(Pn)
    out = np.empty_like(Pn)
    it = np.zeros(prob.zones, dtype=np.int32)
    st = np.zeros(prob.zones, dtype=np.int32)
    ev = ctypes.c_longlong(0)
    lib().oracle_step(_iptr(ip), _dptr(dp), _dptr(Pn), ctypes.c_double(dt), _dptr(out), _iptr(it),
                      _iptr(st), ctypes.byref(ev))
    return out, it, st, ev.value


def residual(prob, Pn, PE, dts, Pk, scaled: bool = True, threads: int = 0):
    ip, dp = params(prob, threads)
    Pn, PE, Pk = _c(Pn), _c(PE), _c(Pk)
    out = np.empty_like(Pn)
    lib().oracle_residual(_iptr(ip), _dptr(dp), _dptr(Pn), _dptr(PE), ctypes.c_double(dts), _dptr(Pk),
                          ctypes.c_int(1 if scaled else 0), _dptr(out))
    return out


def fluxes(prob, PE, threads: int = 0):
    """Face fluxes after flux-CT on the low face of every zone: [dim, 10, n3, n2, n1]."""
    ip, dp = params(prob, threads)
    PE = _c(PE)
    out = np.empty((prob.dim, 10) + PE.shape[1:])
    lib().oracle_fluxes(_iptr(ip), _dptr(dp), _dptr(PE), _dptr(out))
    return out


def geometry(prob, X):
    """Metric quantities at the point X (3 coordinates): dict with gcov, gcon
    [4,4], sqrtg, alpha, Gam [4,4,4] ([l][mu][nu]) and tauR."""
    ip, dp = params(prob)
    X = np.ascontiguousarray(X, dtype=np.float64)
    gcov = np.empty((4, 4)); gcon = np.empty((4, 4)); Gam = np.empty((4, 4, 4))
    sg, al, tr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().oracle_geometry(_iptr(ip), _dptr(dp), _dptr(X), _dptr(gcov), _dptr(gcon), ctypes.byref(sg),
                          ctypes.byref(al), _dptr(Gam), ctypes.byref(tr))
    return {"gcov": gcov, "gcon": gcon, "sqrtg": sg.value, "alpha": al.value, "Gam": Gam, "tauR": tr.value}


def floors(prob, X, P):
    """The post-stage floors applied to one primitive vector at X (copy)."""
    ip, dp = params(prob)
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.array(P, dtype=np.float64, copy=True)
    lib().oracle_floors(_iptr(ip), _dptr(dp), _dptr(X), _dptr(out))
    return out


def point(prob, P):
    """U, F^1, F^2, F^3 and the (cmin, cmax) wave speeds per direction at one state."""
    ip, dp = params(prob)
    P = _c(P)
    U = np.empty(10); F = np.empty((3, 10)); c = np.empty(6)
    lib().oracle_point(_iptr(ip), _dptr(dp), _dptr(P), _dptr(U), _dptr(F[0]), _dptr(F[1]), _dptr(F[2]),
                       _dptr(c))
    return U, F, c.reshape(3, 2)


def linearize(prob, P0):
    """Complex-step linearisation about a uniform state: (MU, A[3], SP, SD[4])."""
    ip, dp = params(prob)
    P0 = _c(P0)
    MU = np.empty((10, 10)); A = np.empty((3, 10, 10)); SP = np.empty((10, 10)); SD = np.empty((4, 10, 10))
    lib().oracle_linearize(_iptr(ip), _dptr(dp), _dptr(P0), _dptr(MU), _dptr(A), _dptr(SP), _dptr(SD))
    return MU, A, SP, SD


ZC_SIZE = 80


def zone_residual(prob, zc, P):
    ip, dp = params(prob)
    r = np.empty(10)
    lib().oracle_zone_residual(_iptr(ip), _dptr(dp), _dptr(_c(zc)), _dptr(_c(P)), _dptr(r))
    return r


def zone_jacobian(prob, zc, P, method="fd"):
    ip, dp = params(prob)
    J = np.empty((10, 10))
    fn = lib().oracle_zone_jacobian_fd if method == "fd" else lib().oracle_zone_jacobian_cs
    fn(_iptr(ip), _dptr(dp), _dptr(_c(zc)), _dptr(_c(P)), _dptr(J))
    return J


def zone_newton(prob, zc, P0):
    ip, dp = params(prob)
    P = _c(P0).copy()
    out = np.zeros(3, dtype=np.int32)
    lib().oracle_zone_newton(_iptr(ip), _dptr(dp), _dptr(_c(zc)), _dptr(P), _iptr(out))
    return P, int(out[0]), int(out[1]), int(out[2])


def lu_solve(J, b):
    x = np.empty(10)
    rc = lib().oracle_lu_solve(_dptr(_c(J)), _dptr(_c(b)), _dptr(x))
    return x, rc


def flop_counts(prob, zc, P):
    """(residual, 10x10 LU solve, Newton bookkeeping, 7x7 LU solve of the
    non-magnetic block) algorithmic flops."""
    ip, dp = params(prob)
    out = np.zeros(4, dtype=np.int64)
    lib().oracle_flop_counts(_iptr(ip), _dptr(dp), _dptr(_c(zc)), _dptr(_c(P)),
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return out


def max_threads():
    return int(lib().oracle_max_threads())


def recon(prob, line7):
    """(left-face, right-face) values of the middle zone of a 7-zone line."""
    ip, dp = params(prob)
    out = np.empty(2)
    lib().oracle_recon(_iptr(ip), _dptr(dp), _dptr(_c(line7)), _dptr(out))
    return out


def stage_masked(prob, Pn, PE, dts, mask, guess=None, threads: int = 0):
    """One stage solved only where mask != 0; returns (P_out, iters, status, evals)
    with P_out = P_n elsewhere."""
    ip, dp = params(prob, threads)
    Pn, PE = _c(Pn), _c(PE)
    out = Pn.copy()
    it = np.zeros(prob.zones, dtype=np.int32)
    st = np.zeros(prob.zones, dtype=np.int32)
    ev = ctypes.c_longlong(0)
    m = np.ascontiguousarray(np.asarray(mask).reshape(-1).astype(np.int8))
    g = _c(guess) if guess is not None else None
    lib().oracle_stage_masked(_iptr(ip), _dptr(dp), _dptr(Pn), _dptr(PE), ctypes.c_double(dts),
                              _dptr(g) if g is not None else None, m.ctypes.data_as(ctypes.c_char_p),
                              _dptr(out), _iptr(it), _iptr(st), ctypes.byref(ev))
    return out, it, st, ev.value


def step_sampled(prob, Pn, dt, zones, threads: int = 0):
    """One full step at the listed flat zone indices only: (P [10, nz], iters, status, evals)."""
    ip, dp = params(prob, threads)
    Pn = _c(Pn)
    z = np.ascontiguousarray(np.asarray(zones, dtype=np.int64))
    nz = z.size
    out = np.empty((10, nz))
    it = np.zeros(nz, dtype=np.int32)
    st = np.zeros(nz, dtype=np.int32)
    ev = ctypes.c_longlong(0)
    lib().oracle_step_sampled(_iptr(ip), _dptr(dp), _dptr(Pn), ctypes.c_double(dt),
                              z.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), ctypes.c_int(nz),
                              _dptr(out), _iptr(it), _iptr(st), ctypes.byref(ev))
    return out, it, st, ev.value


def explicit_flops(prob, line8, Pn1):
    """(per-face, per-zone remainder) algorithmic flops of the explicit part."""
    ip, dp = params(prob)
    out = np.zeros(2, dtype=np.int64)
    lib().oracle_explicit_flops(_iptr(ip), _dptr(dp), _dptr(_c(line8)), _dptr(_c(Pn1)),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return out
