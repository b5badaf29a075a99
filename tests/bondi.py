"""Steady spherical accretion onto a Schwarzschild black hole (Michel 1972),
the exact solution for the hydrodynamic GR test: a polytrope p = K rho^gamma
flowing in radially with, in Schwarzschild coordinates (M = 1),
  rho u^r r^2 = C1                        (rest-mass flux)
  h^2 (1 - 2/r + (u^r)^2) = C2            (Bernoulli; h = 1 + gamma/(gamma-1) p/rho)
and passing smoothly through the sonic point r_c, where (u^r)^2 = 1/(2 r_c)
and the sound speed V^2 = gamma p/(rho h) equals u_c^2/(1 - 3 u_c^2).
Written here from these relations; rho = 1 at r_c."""
import math

import numpy as np

from paper_1702_01106_b300 import inputs


def michel_constants(gamma, rc):
    u2 = 1.0 / (2.0 * rc)
    V2 = u2 / (1.0 - 3.0 * u2)
    theta = V2 / (gamma * (1.0 - V2 / (gamma - 1.0)))    # p/rho at r_c, from V^2 = gamma theta / h
    K = theta                                             # rho_c = 1
    h = 1.0 + gamma / (gamma - 1.0) * theta
    C1 = -math.sqrt(u2) * rc * rc                         # inflow
    C2 = h * h * (1.0 - 2.0 / rc + u2)
    return K, C1, C2


def michel_rho(r, gamma, rc):
    """Density on the transonic branch (bisection on the Bernoulli relation
    with u^r from the mass flux: subsonic outside r_c, supersonic inside)."""
    K, C1, C2 = michel_constants(gamma, rc)

    def f(rho):
        h = 1.0 + gamma / (gamma - 1.0) * K * rho ** (gamma - 1.0)
        u = C1 / (rho * r * r)
        return h * h * (1.0 - 2.0 / r + u * u) - C2

    # f falls then rises in rho, with its minimum at the local sonic density
    # (a double root at r = r_c): locate it by golden-section search in log rho,
    # then bisect on the branch (subsonic outside r_c, supersonic inside)
    a, b = math.log(1e-8), math.log(1e4)
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    for _ in range(200):
        c, d = b - gr * (b - a), a + gr * (b - a)
        if f(math.exp(c)) < f(math.exp(d)):
            b = d
        else:
            a = c
    rmin = math.exp(0.5 * (a + b))
    if f(rmin) >= 0.0:
        return rmin            # at the sonic point the two branches meet
    a, b = (rmin, 1e4) if r > rc else (1e-8, rmin)
    fa = f(a)
    for _ in range(200):
        m = 0.5 * (a + b)
        fm = f(m)
        if (fm > 0) == (fa > 0):
            a, fa = m, fm
        else:
            b = m
    return 0.5 * (a + b)


def bondi_problem(n1, n2=4, r_in=2.5, r_out=20.0, tol=1e-12):
    """Schwarzschild (a = 0) in MKS coordinates, a thin equatorial band (the
    flow is radial; the band's X2 edges reflect), hydrodynamics only."""
    return inputs.Problem(dim=2, n=(n1, n2, 1), x_start=(math.log(r_in), 0.45, 0.0),
                          x_end=(math.log(r_out), 0.55, 2 * math.pi),
                          bc=((inputs.BC_OUTFLOW, inputs.BC_OUTFLOW), (inputs.BC_REFLECT, inputs.BC_REFLECT),
                              (inputs.BC_PERIODIC, inputs.BC_PERIODIC)),
                          metric=inputs.METRIC_MKS_KERR, spin=0.0, h_mks=1.0, gamma=4.0 / 3.0,
                          conduction=False, viscosity=False, higher_order=False, tol=tol)


def bondi_state(prob, rc=8.0):
    """Primitive state of the Michel solution on the zone centres: u^r from
    the mass flux, u^t_KS = u^t_BL + (2r/Delta) u^r, and the normal-observer
    velocity u~^1 = u^r/r + 2 u^t/(r^2 + 2 r) of Kerr-Schild with a = 0."""
    gamma = prob.gamma
    K, C1, _ = michel_constants(gamma, rc)
    x1, _, _ = inputs.zone_centers(prob)
    r = np.exp(x1[0, 0])
    rho = np.array([michel_rho(float(rr), gamma, rc) for rr in r])
    ur = C1 / (rho * r * r)
    ut_bl = np.sqrt(1.0 - 2.0 / r + ur * ur) / (1.0 - 2.0 / r)
    ut = ut_bl + 2.0 * r / (r * r - 2.0 * r) * ur
    P = np.zeros((10,) + tuple(prob.n[::-1]))
    P[0] = rho
    P[1] = K * rho ** gamma / (gamma - 1.0)
    P[2] = ur / r + 2.0 * ut / (r * r + 2.0 * r)
    return P


def bondi_dt(prob, cfl=0.5):
    """cfl x the smallest dX^1 / (coordinate light speed along X^1): the
    radial light speeds of Kerr-Schild (a = 0) in MKS, (-1, (1 - 2/r)/(1 + 2/r))/r."""
    x1, _, _ = inputs.zone_centers(prob)
    r = np.exp(x1[0, 0])
    return cfl * float((prob.dx[0] * r).min())
