"""Viscous Bondi inflow (Section 8.2, "Bondi Inflow"): the steady pressure
anisotropy carried by the Michel flow when it does not act back on the flow.

The paper checks the scheme against reference profiles from one-dimensional
ODEs along the steady inflow, integrated with the anisotropy's feedback on
the flow turned off.  Here the feedback is made negligible instead of being
switched off: the physical anisotropy is dP = dP~ (nu rho Theta / tau_R)^(1/2)
with nu = psi c_s^2 tau_R, and the rescaled target dP~_0 scales as psi^(1/2),
so dP scales as psi; at psi = 1e-6 its stress is ~1e-6 of the gas pressure,
below the truncation error of the flow itself, and dP~ / psi^(1/2) is the
feedback-free profile.

Written from the model's equations (Section 4), apart from the oracle and the
CUDA path.  For a steady radial flow (Boyer-Lindquist or Kerr-Schild
coordinates share r and u^r; dP~ is a scalar) the rescaled evolution
equation nabla_mu(dP~ u^mu) = -(dP~ - dP~_0)/tau_R + h (dP~/2) nabla_mu u^mu
(h = 1 with the higher-order term, 0 without) becomes
    u^r d dP~/dr = -(dP~ - dP~_0)/tau_R - (1 - h/2) dP~ nabla_mu u^mu,
with nabla_mu u^mu = r^-2 d(r^2 u^r)/dr and, from Eq. dP0def,
    dP~_0 = 3 (bhat^mu bhat^nu nabla_mu u_nu - nabla_mu u^mu / 3)
            (rho nu tau_R / Theta)^(1/2).
The field is radial, so bhat is the unit vector of the (t, r) plane
orthogonal to u.  The shear bhat bhat nabla u is evaluated in
Boyer-Lindquist coordinates with the Schwarzschild connection written out,
and checked against the same scalar in Kerr-Schild coordinates with the
connection from sympy.  The flow enters at r = 40 through a copy boundary,
so the reference starts there with zero gradient (the ODE's fixed point)
and is integrated inwards (eighth-order Dormand-Prince, rtol 1e-11).
"""
from __future__ import annotations

import functools
import math

import numpy as np

from tests.bondi import bondi_problem, michel_constants, michel_rho

GAMMA = 4.0 / 3.0
RC = 8.0
PSI = 1e-6            # feedback of dP on the flow ~ psi: negligible
TAU0 = 1.0            # tau_R = TAU0 r^(3/2), the general-metric path's relaxation time
B_C = 1e-2            # radial field B^1 = B_C / r^3 in MKS: sqrt(-g) B^1 independent of r
R_OUT = 40.0         # far enough out that the copy boundary's disturbance misses 3 < r < 12 by t = 30


def viscous_bondi_problem(n1, higher_order=True, tol=1e-12):
    """The Michel flow's grid (Schwarzschild in MKS coordinates, an
    equatorial band, 2.5 <= r <= 40) with viscosity on, conduction off."""
    return bondi_problem(n1, r_out=R_OUT, tol=tol).with_(viscosity=True, conduction=False, higher_order=higher_order,
                                            psi=PSI, phi=0.0, tau_R=TAU0)


@functools.lru_cache(maxsize=None)
def _flow_cached(r):
    K, C1, _ = michel_constants(GAMMA, RC)
    rho = michel_rho(r, GAMMA, RC)
    h = 1e-5 * r
    drho = (michel_rho(r + h, GAMMA, RC) - michel_rho(r - h, GAMMA, RC)) / (2.0 * h)
    ur = C1 / (rho * r * r)
    dur = -ur * (2.0 / r + drho / rho)
    u = K * rho ** GAMMA / (GAMMA - 1.0)
    return rho, u, ur, dur


def flow(r):
    """rho, u (internal energy), u^r and du^r/dr of the Michel flow at r
    (the transonic branch is smooth through r_c, so a centred difference of
    the density, step 1e-5 r, gives its slope to ~1e-10)."""
    return _flow_cached(float(r))


def shear_bl(r):
    """(bhat^mu bhat^nu nabla_mu u_nu, nabla_mu u^mu) in Boyer-Lindquist
    coordinates, A = 1 - 2/r, with the Schwarzschild connection
    Gamma^r_tt = A/r^2, Gamma^t_tr = 1/(r^2 A), Gamma^r_rr = -1/(r^2 A)."""
    _, _, ur, dur = flow(r)
    A = 1.0 - 2.0 / r
    dA = 2.0 / (r * r)
    s = math.sqrt(A + ur * ur)
    u_t, u_r = -s, ur / A                     # covariant components
    bt, br = ur / A, s                        # unit, orthogonal to u, in the (t, r) plane
    d_ut = -(dA + 2.0 * ur * dur) / (2.0 * s)
    d_ur = dur / A - ur * dA / (A * A)
    g_rtt, g_ttr, g_rrr = A / (r * r), 1.0 / (r * r * A), -1.0 / (r * r * A)
    S = bt * bt * (-g_rtt * u_r) + bt * br * (d_ut - 2.0 * g_ttr * u_t) + br * br * (d_ur - g_rrr * u_r)
    divu = 2.0 * ur / r + dur
    return S, divu


@functools.lru_cache(maxsize=None)
def _ks_connection():
    """Kerr-Schild metric (a = 0) on the equator and its connection
    Gamma^l_{mu nu} for mu, nu in (t, r), as numpy functions of r."""
    import sympy as sp
    r, th = sp.symbols("r theta", positive=True)
    t, ph = sp.symbols("t phi")
    X = [t, r, th, ph]
    g = sp.zeros(4)
    g[0, 0] = -(1 - 2 / r)
    g[0, 1] = g[1, 0] = 2 / r
    g[1, 1] = 1 + 2 / r
    g[2, 2] = r ** 2
    g[3, 3] = r ** 2 * sp.sin(th) ** 2
    gi = g.inv()
    G = [[[sp.simplify(sum(gi[l, k] * (sp.diff(g[k, n], X[m]) + sp.diff(g[k, m], X[n]) - sp.diff(g[m, n], X[k]))
                           for k in range(4)) / 2).subs(th, sp.pi / 2) for n in range(2)] for m in range(2)]
         for l in range(2)]
    return sp.lambdify(r, g.subs(th, sp.pi / 2), "numpy"), sp.lambdify(r, G, "numpy")


def shear_ks(r):
    """The same scalar bhat bhat nabla u in Kerr-Schild coordinates:
    u^t_KS = u^t_BL + (2r/(r^2 - 2r)) u^r, u_nu from the metric, d_r u_nu by
    a centred difference, the connection from sympy."""
    gfun, Gfun = _ks_connection()

    def frame(x):
        _, _, ur, _ = flow(x)
        A = 1.0 - 2.0 / x
        ut = math.sqrt(A + ur * ur) / A + 2.0 * x / (x * x - 2.0 * x) * ur
        gm = np.array(gfun(x), dtype=float)[:2, :2]
        ucon = np.array([ut, ur])
        return gm, ucon, gm @ ucon

    gm, ucon, ucov = frame(r)
    h = 1e-5 * r
    d_ucov = (frame(r + h)[2] - frame(r - h)[2]) / (2.0 * h)
    v = np.array([-ucov[1] / ucov[0], 1.0])
    bh = v / math.sqrt(v @ gm @ v)
    G = np.array(Gfun(r), dtype=float)        # G[l][m][n] = Gamma^l_{mn}, l, m, n in (t, r)
    S = 0.0
    for m in range(2):
        for n in range(2):
            nab = (d_ucov[n] if m == 1 else 0.0) - sum(G[l][m][n] * ucov[l] for l in range(2))
            S += bh[m] * bh[n] * nab
    return S


def target(r):
    """dP~_0 of the steady flow at r (Eq. dP0def, rescaled), and the
    coefficients tau_R and nabla_mu u^mu there."""
    rho, u, _, _ = flow(r)
    S, divu = shear_bl(r)
    pg = (GAMMA - 1.0) * u
    theta = pg / rho
    cs2 = GAMMA * pg / (rho + GAMMA * u)
    tau = TAU0 * r ** 1.5
    nu = PSI * cs2 * tau
    return 3.0 * (S - divu / 3.0) * math.sqrt(rho * nu * tau / theta), tau, divu


@functools.lru_cache(maxsize=None)
def reference(higher_order=True, r_in=2.5):
    """Dense solution dP~(r) of the steady relaxation ODE from r = 40 inwards."""
    from scipy.integrate import solve_ivp
    c = 1.0 - (0.5 if higher_order else 0.0)

    def rhs(x, y):
        y0, tau, divu = target(x)
        _, _, ur, _ = flow(x)
        return [(-(y[0] - y0) / tau - c * y[0] * divu) / ur]

    y0, tau, divu = target(R_OUT)
    start = y0 / (1.0 + tau * c * divu)       # zero gradient at the outer edge
    sol = solve_ivp(rhs, (R_OUT, r_in), [start], method="DOP853", rtol=1e-11, atol=1e-16, dense_output=True)
    assert sol.status == 0
    return sol


def viscous_bondi_state(prob, higher_order=True):
    """The Michel flow of tests/bondi.py with the radial field B^1 = B_C/r^3
    and dP~ from the reference profile."""
    from tests.bondi import bondi_state
    from paper_1702_01106_b300 import inputs
    P = bondi_state(prob, RC)
    x1, _, _ = inputs.zone_centers(prob)
    r = np.exp(x1[0, 0])
    P[5] = B_C / r ** 3
    P[9] = reference(higher_order).sol(r)[0]
    return P, r
