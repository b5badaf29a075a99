"""Hydrostatic conducting atmosphere (Section 8.2), in thermal equilibrium
and with a radial heat flux: a static gas around a Schwarzschild black hole (M = 1) with a
radial field, 200 <= r <= 300, held up by its pressure with no heat flux.
Written here from the equilibrium conditions of that section; nothing comes
from the oracle or the CUDA path.

A static fluid moves along the Killing vector d_t, so its four-acceleration
is a_mu = d_mu ln alpha_t with alpha_t = (-g_tt)^(1/2) = (1 - 2/r)^(1/2) (the
same in Schwarzschild and Kerr-Schild coordinates).  Then
  - momentum balance:  dP/dr = -(rho + u + P) d ln alpha_t / dr;
  - no heat flux: q_0 ~ b-hat^mu (d_mu Theta + Theta a_mu) = 0 along the
    radial field, i.e. Theta alpha_t = constant (the redshifted temperature
    is uniform, not Theta);
  - no shear: b-hat^mu b-hat^nu nabla_mu u_nu = -(b-hat.u)(b-hat.a) = 0 and
    nabla_mu u^mu = 0, so dP_0 = 0;
with u = P/(gamma - 1) and rho = P/Theta.  With Theta = Theta_0 alpha_0/alpha
the momentum balance reads d ln P = -(alpha / (Theta_0 alpha_0) + gamma /
(gamma - 1)) d ln alpha, whose solution from P_0 at r = 200 is
  P = P_0 (alpha/alpha_0)^(-gamma/(gamma-1)) exp(-(alpha - alpha_0)/(Theta_0 alpha_0));
`pressure_ode` integrates the balance itself (eighth-order Dormand-Prince,
rtol 1e-13) as an independent check of that closed form.

Grid: modified Kerr-Schild coordinates with a = 0, X^1 = ln r, a thin band
about the equator (the solution does not depend on theta; the band's X^2
edges reflect), outflow at r = 200 and 300.  The field is a monopole,
sqrt(-g) B^1 independent of X^1, i.e. B^1 = C / r^3 in these coordinates,
so div B = 0 zone by zone.  The normal-observer velocity of the static
fluid is u~^1 = 2 u^t / (r^2 + 2 r), u^t = 1/alpha_t (Kerr-Schild, a = 0).
"""
from __future__ import annotations

import functools
import math

import numpy as np

from paper_1702_01106_b300 import inputs

GAMMA = 4.0 / 3.0
R_IN, R_OUT = 200.0, 300.0
RHO0, THETA0 = 1.0, 0.01          # at r = 200
B_C = 1e-2                         # B^1 = B_C / r^3: b^2 / P ~ 1e-8
TAU0 = 1e-3                        # tau_R = TAU0 r^(3/2): 2.8 at r = 200, 5.2 at 300


def alpha_t(r):
    return np.sqrt(1.0 - 2.0 / r)


def dlnalpha_dr(r):
    return 1.0 / (r * r * (1.0 - 2.0 / r))


def theta_of_r(r):
    return THETA0 * alpha_t(R_IN) / alpha_t(r)


def pressure(r):
    """The closed form of the momentum balance with Theta alpha_t constant."""
    a, a0 = alpha_t(np.asarray(r, dtype=float)), alpha_t(R_IN)
    return RHO0 * THETA0 * (a / a0) ** (-GAMMA / (GAMMA - 1.0)) * np.exp(-(a - a0) / (THETA0 * a0))


def pressure_ode(r):
    """dP/dr = -(rho + u + P) d ln alpha_t/dr integrated from r = 200."""
    from scipy.integrate import solve_ivp

    def rhs(rr, y):
        P = y[0]
        th = theta_of_r(rr)
        return [-(P / th + P / (GAMMA - 1.0) + P) * dlnalpha_dr(rr)]

    sol = solve_ivp(rhs, (R_IN, R_OUT), [RHO0 * THETA0], method="DOP853", rtol=1e-13, atol=1e-16,
                    dense_output=True)
    assert sol.status == 0
    return sol.sol(np.asarray(r, dtype=float))[0]


# ---------------------------------------------------------------- with a heat flux
# The second case: heat flowing outwards.  For the static fluid the
# relaxation equation leaves q = q_0 (its advection and nabla_mu u^mu vanish),
# so q_0 = -rho chi b-hat^r (dTheta/dr + Theta d ln alpha_t/dr) fixes dTheta/dr.
# The Killing energy flux sqrt(-g) T^r_t = sqrt(-g) q b-hat^r u_t is constant
# (the field carries none: b_t = 0 for a static fluid and a radial field), which
# fixes q(r) = F / (r^2 b-hat^r (-u_t)).  The radial momentum balance
# d(sqrt(-g) T^r_r)/dr = sqrt(-g) T^k_l Gamma^l_{r k}, with T^r_r = P + q b-hat^r u_r
# (u_r = g_rt u^t is not zero in Kerr-Schild coordinates) and T^k_l = w u^k u_l
# + P delta^k_l + q (b-hat^k u_l + u^k b-hat_l), fixes dP/dr.  Gamma of the
# Kerr-Schild metric (a = 0) comes from sympy, here; with F = 0 the balance
# reduces to the closed form above.


@functools.lru_cache(maxsize=None)
def _kerr_schild_r_connection():
    """(g_{mu nu}(r), Gamma^l_{r k}(r)) on the equator, Kerr-Schild, a = 0."""
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
    gam = [[sp.simplify(sum(gi[l, m] * (sp.diff(g[m, 1], X[k]) + sp.diff(g[m, k], X[1]) - sp.diff(g[1, k], X[m]))
                            for m in range(4)) / 2).subs(th, sp.pi / 2) for k in range(4)] for l in range(4)]
    return sp.lambdify(r, g.subs(th, sp.pi / 2), "numpy"), sp.lambdify(r, sp.Matrix(gam), "numpy")


def _static_frame(r):
    """u^mu, u_mu, b-hat^mu, b-hat_mu of the static fluid with a radial field."""
    gfun, _ = _kerr_schild_r_connection()
    gm = np.array(gfun(r), dtype=float)
    ucon = np.array([1.0 / alpha_t(r), 0.0, 0.0, 0.0])
    ucov = gm @ ucon
    v = np.array([-ucov[1] / ucov[0], 1.0, 0.0, 0.0])   # in the (t, r) plane, orthogonal to u
    bh = v / math.sqrt(v @ gm @ v)
    return ucon, ucov, bh, gm @ bh


def heat_flux(r, F):
    _, ucov, bh, _ = _static_frame(r)
    return F / (r * r * bh[1] * (-ucov[0]))


def _conducting_rhs(r, y, F, phi):
    Pg, th = y
    rho, u = Pg / th, Pg / (GAMMA - 1.0)
    w = rho + u + Pg
    ucon, ucov, bh, bhc = _static_frame(r)
    q = heat_flux(r, F)
    chi = phi * GAMMA * Pg / w * TAU0 * r ** 1.5
    dth = -q / (rho * chi * bh[1]) - th * dlnalpha_dr(r)
    T = w * np.outer(ucon, ucov) + Pg * np.eye(4) + q * (np.outer(bh, ucov) + np.outer(ucon, bhc))
    _, gam = _kerr_schild_r_connection()
    G = np.array(gam(r), dtype=float)                      # G[l, k] = Gamma^l_{r k}
    S = float(np.sum(T * G.T))                             # T^k_l Gamma^l_{r k}

    def qbu(x):
        _, uv, b, _ = _static_frame(x)
        return heat_flux(x, F) * b[1] * uv[1]

    h = 1e-3 * r
    dqbu = (qbu(r + h) - qbu(r - h)) / (2.0 * h)
    return [S - (2.0 / r) * (Pg + qbu(r)) - dqbu, dth]


@functools.lru_cache(maxsize=None)
def conducting_solution(F, phi=1.0):
    """Dense solution (P, Theta)(r) of the conducting atmosphere with energy
    flux F (F = 0: thermal equilibrium)."""
    from scipy.integrate import solve_ivp
    sol = solve_ivp(lambda x, y: _conducting_rhs(x, y, F, phi), (R_IN, R_OUT), [RHO0 * THETA0, THETA0],
                    method="DOP853", rtol=1e-12, atol=1e-16, dense_output=True)
    assert sol.status == 0
    return sol


def conducting_state(prob, F):
    """Primitives of the conducting atmosphere (q~ = q (tau_R/(chi rho Theta^2))^(1/2))."""
    x1, _, _ = inputs.zone_centers(prob)
    r = np.exp(x1[0, 0])
    Pg, th = conducting_solution(F, prob.phi).sol(r)
    rho, u = Pg / th, Pg / (GAMMA - 1.0)
    cs2 = GAMMA * Pg / (rho + u + Pg)
    q = np.array([heat_flux(x, F) for x in r])
    P, _ = atmosphere_state(prob)
    P[0], P[1] = rho, u
    P[8] = q / (th * np.sqrt(prob.phi * cs2 * rho))
    return P, r


def atmosphere_problem(n1, n2=4, tol=1e-12, conduction=True, viscosity=True):
    return inputs.Problem(dim=2, n=(n1, n2, 1), x_start=(math.log(R_IN), 0.45, 0.0),
                          x_end=(math.log(R_OUT), 0.55, 2 * math.pi),
                          bc=((inputs.BC_OUTFLOW, inputs.BC_OUTFLOW), (inputs.BC_REFLECT, inputs.BC_REFLECT),
                              (inputs.BC_PERIODIC, inputs.BC_PERIODIC)),
                          metric=inputs.METRIC_MKS_KERR, spin=0.0, h_mks=1.0, gamma=GAMMA,
                          conduction=conduction, viscosity=viscosity, higher_order=True,
                          phi=1.0, psi=1.0, tau_R=TAU0, tol=tol)


def atmosphere_state(prob):
    """Primitives [10, n3, n2, n1] on the zone centres, and r of each column."""
    x1, _, _ = inputs.zone_centers(prob)
    r = np.exp(x1[0, 0])
    Pg = pressure(r)
    th = theta_of_r(r)
    ut = 1.0 / alpha_t(r)
    P = np.zeros((10,) + tuple(prob.n[::-1]))
    P[0] = Pg / th
    P[1] = Pg / (GAMMA - 1.0)
    P[2] = 2.0 * ut / (r * r + 2.0 * r)
    P[5] = B_C / r ** 3
    return P, r


def atmosphere_dt(prob, cfl=0.5):
    """cfl x the smallest dX^1 / (coordinate light speed along X^1, at most 1/r)."""
    x1, _, _ = inputs.zone_centers(prob)
    r = np.exp(x1[0, 0])
    return cfl * float((prob.dx[0] * r).min())


def heat_target_without_redshift(prob, P):
    """|q~_0| the atmosphere would be driven to if the heat flux followed
    d_mu Theta alone (no Theta a_mu term): q_0 = -rho chi b-hat^r dTheta/dr
    with b-hat^r = alpha_t (the static observer's radial unit vector in
    Schwarzschild's r), chi = phi c_s^2 tau_R, rescaled by
    (tau_R / (chi rho Theta^2))^(1/2).  The scale a missing term would show."""
    x1, _, _ = inputs.zone_centers(prob)
    r = np.exp(x1[0, 0])
    rho, u = P[0, 0, 0], P[1, 0, 0]
    Pg = (GAMMA - 1.0) * u
    th = Pg / rho
    cs2 = GAMMA * Pg / (rho + u + Pg)
    tau = TAU0 * r ** 1.5
    chi = prob.phi * cs2 * tau
    dth = -theta_of_r(r) * dlnalpha_dr(r)                 # dTheta/dr of Theta alpha_t = const
    q0 = -rho * chi * alpha_t(r) * dth
    return np.abs(q0 * np.sqrt(tau / (chi * rho * th * th)))
