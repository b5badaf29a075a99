"""Hydrostatic conducting atmosphere (Section 8.2), the case in thermal
equilibrium: a static gas around a Schwarzschild black hole (M = 1) with a
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
