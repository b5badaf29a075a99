"""Buoyancy instabilities with anisotropic conduction (Section 9.1): a
hydrostatic polytropic atmosphere around a Schwarzschild black hole (M = 1)
threaded by a weak field, with heat conducted along the field.
  - MTI (magneto-thermal instability): temperature falling outwards, field
    perpendicular to gravity (azimuthal); the radial field grows.
  - HBI (heat-flux-driven buoyancy instability): temperature rising
    outwards, field along gravity (radial); the perpendicular (azimuthal)
    field grows.
Written from the model and the linear theory the paper cites (Balbus 2000,
Quataert 2008); nothing here comes from the oracle or the CUDA path.

Equilibrium.  A static fluid moves along the Killing vector d_t, so its
four-acceleration is a_mu = d_mu ln alpha_t, alpha_t = (1 - 2/r)^(1/2), and
momentum balance reads dP/dr = -(rho + u + P) d ln alpha_t/dr.  With the
polytrope P = K rho^G (the paper's MTI: K = 1e-4, G = 4/3; HBI: K = 0.05,
G = 1/2), u = P/(gamma - 1) and Theta = P/rho = K rho^(G - 1),
dP/rho = G/(G - 1) dTheta, so
    G/(G - 1) dTheta / (1 + c Theta) = -d ln alpha_t,  c = gamma/(gamma - 1),
whose solution from Theta_0 at r = 200 is
    1 + c Theta = (1 + c Theta_0) (alpha_0/alpha_t)^(c (G - 1)/G).
`theta_ode` integrates the balance itself as an independent check.  Both
equilibria are Schwarzschild-stable (G < gamma = 5/3: the entropy rises
outwards); the MTI's temperature falls outwards, the HBI's rises.  The
paper gives no density scale: Theta_0 is chosen so that the linear theory's
growth time at r = 200 is the paper's dynamical time there (2500 M for the
MTI, 2000 M for the HBI).

Field and heat flux.  The field is B = 1e-3 / sqrt(-g) along phi (MTI, the
paper's weak azimuthal field) or along r (HBI); b^2/P ~ 1e-15, so magnetic
tension plays no part, and sqrt(-g) B is constant, so div B = 0.  The
initial heat flux vanishes (MTI: the field is perpendicular to the
temperature gradient; HBI: q~ starts at zero and relaxes to its target).
The closure follows the paper's choice chi = c_s R, tau_R = R/c_s: with
chi = phi c_s^2 tau_R this is phi = 1 and tau_R = R/c_s, which the library's
tau_R = tau_0 r^(3/2) follows over 200 <= r <= 300 (tau_0 fitted at
r = 250): to 4 % for the MTI, to 25 % for the HBI, whose sound speed rises
outwards.  Viscosity is off (the section names no viscosity for these runs).

Linear theory.  With conduction along the field much faster than the
dynamics, a weakly magnetised atmosphere is unstable where the temperature
falls along a field perpendicular to gravity (MTI) or rises along a field
parallel to it (HBI); the fastest modes, with wavevector nearly
perpendicular to gravity, grow at sigma = (g |d ln T/dz|)^(1/2).  Here
g = d ln alpha_t/dr and T = Theta.

Grid: modified Kerr-Schild coordinates with a = 0 and h = 1 (theta = pi X^2),
X^1 = ln r in [ln 200, ln 300], a thin band about the equator (reflecting X^2
edges; the equilibrium does not depend on theta) and phi = X^3 in [0, pi]
(periodic), the paper's half sphere in phi.  The paper holds rho, u and the
pressure fixed at the radial boundaries (constant-temperature boundaries
that keep driving the instability); the library's radial boundaries are
copies, so the run resets the outermost radial layers to the equilibrium
after every step (see `hold_boundaries`), which plays that part.
"""
from __future__ import annotations

import math

import numpy as np

from paper_1702_01106_b300 import inputs

GAMMA = 5.0 / 3.0            # the gas
R_IN, R_OUT = 200.0, 300.0
B_AMP = 1e-3                 # sqrt(-g) B, along phi (MTI) or r (HBI)
NOISE = 0.004                # seeded fluctuations of u~^1, in units of the local sound speed (see initial_state)
HOLD = 3                     # radial layers held at the equilibrium at each end


class Case:
    """One instability: the polytrope (K, G), Theta at r = 200, the field's
    direction (primitive index) and the component whose growth is measured."""

    def __init__(self, name, K, G, theta0, field, grows):
        self.name, self.K, self.G, self.theta0, self.field, self.grows = name, K, G, theta0, field, grows


MTI = Case("mti", 1e-4, 4.0 / 3.0, 1e-3, field=7, grows=5)    # azimuthal field; the radial field grows
HBI = Case("hbi", 0.05, 0.5, 2.5e-3, field=5, grows=7)        # radial field; the azimuthal field grows


def alpha_t(r):
    return np.sqrt(1.0 - 2.0 / np.asarray(r, dtype=float))


def gravity(r):
    """g = d ln alpha_t / dr."""
    r = np.asarray(r, dtype=float)
    return 1.0 / (r * r * (1.0 - 2.0 / r))


def theta_of_r(r, case=MTI):
    """Closed form of the hydrostatic polytrope (module docstring)."""
    c = GAMMA / (GAMMA - 1.0)
    e = c * (case.G - 1.0) / case.G
    return ((1.0 + c * case.theta0) * (alpha_t(R_IN) / alpha_t(r)) ** e - 1.0) / c


def theta_ode(r, case=MTI):
    """Momentum balance integrated from r = 200 (eighth-order Dormand-Prince)
    in P, with rho = (P/K)^(1/G): Theta = P / rho."""
    from scipy.integrate import solve_ivp

    def rhs(rr, y):
        P = y[0]
        rho = (P / case.K) ** (1.0 / case.G)
        return [-(rho + P / (GAMMA - 1.0) + P) * float(gravity(rr))]

    rho0 = (case.theta0 / case.K) ** (1.0 / (case.G - 1.0))
    sol = solve_ivp(rhs, (R_IN, R_OUT), [case.theta0 * rho0], method="DOP853", rtol=1e-13, atol=1e-18,
                    dense_output=True)
    assert sol.status == 0
    P = sol.sol(np.asarray(r, dtype=float))[0]
    return P / (P / case.K) ** (1.0 / case.G)


def sound_speed(r, case=MTI):
    th = theta_of_r(r, case)
    return np.sqrt(GAMMA * th / (1.0 + GAMMA / (GAMMA - 1.0) * th))


def growth_rate(r, case=MTI):
    """Fastest growth rate (g |d ln Theta/dr|)^(1/2) at r (centred
    difference of the closed form)."""
    r = np.asarray(r, dtype=float)
    h = 1e-4 * r
    dlnT = (np.log(theta_of_r(r + h, case)) - np.log(theta_of_r(r - h, case))) / (2.0 * h)
    return np.sqrt(gravity(r) * np.abs(dlnT))


def tau0(case=MTI):
    """tau_R = tau_0 r^(3/2) equal to R / c_s at r = 250."""
    return 250.0 / float(sound_speed(250.0, case)) / 250.0 ** 1.5


def problem(case=MTI, n1=64, n2=4, n3=128, tol=1e-10):
    return inputs.Problem(dim=3, n=(n1, n2, n3), x_start=(math.log(R_IN), 0.45, 0.0),
                          x_end=(math.log(R_OUT), 0.55, math.pi),
                          bc=((inputs.BC_OUTFLOW, inputs.BC_OUTFLOW), (inputs.BC_REFLECT, inputs.BC_REFLECT),
                              (inputs.BC_PERIODIC, inputs.BC_PERIODIC)),
                          metric=inputs.METRIC_MKS_KERR, spin=0.0, h_mks=1.0, gamma=GAMMA,
                          conduction=True, viscosity=False, higher_order=True,
                          phi=1.0, psi=1.0, tau_R=tau0(case), tol=tol)


def sqrt_g(prob, r, th):
    """sqrt(-g) of modified Kerr-Schild coordinates with a = 0, h = 1:
    r^2 sin(theta) (Kerr-Schild) times dr/dX^1 = r and dtheta/dX^2 = pi."""
    return r ** 3 * np.sin(th) * math.pi


def initial_state(prob, case=MTI, seed=11, noise=NOISE):
    """Primitives [10, n3, n2, n1] of the equilibrium with seeded u~^1
    fluctuations of `noise` times the local sound speed (the paper seeds
    about 4 %; 0.4 % keeps the linear phase going two e-folds longer before
    the field saturates, which is where the growth rate is measured); also
    returns r and theta of the zone centres."""
    x1, x2, _ = inputs.zone_centers(prob)
    r = np.exp(x1)
    th = math.pi * x2
    Theta = theta_of_r(r, case)
    rho = (Theta / case.K) ** (1.0 / (case.G - 1.0))
    Pg = rho * Theta
    ut = 1.0 / alpha_t(r)
    P = np.zeros((10,) + tuple(prob.n[::-1]))
    P[0] = rho
    P[1] = Pg / (GAMMA - 1.0)
    # the static fluid's normal-observer velocity in Kerr-Schild coordinates
    # (a = 0), per unit X^1 = ln r
    P[2] = 2.0 * ut / (r * r + 2.0 * r)
    rng = np.random.default_rng(seed)
    P[2] += noise * sound_speed(r, case) / r * rng.uniform(-1.0, 1.0, size=P[2].shape)
    P[case.field] = B_AMP / sqrt_g(prob, r, th)
    return P, r, th


def equilibrium(prob, case=MTI):
    """The state without the fluctuations (what the held layers are reset to)."""
    P, r, th = initial_state(prob, case, noise=0.0)
    return P


def time_step(prob, cfl=0.5):
    return inputs.torus_dt(prob, cfl)


def hold_boundaries(P_dev, P0_dev, layers=HOLD):
    """Reset the outermost `layers` radial layers at both ends to the
    equilibrium (device tensors [10, n3, n2, n1])."""
    P_dev[..., :layers] = P0_dev[..., :layers]
    P_dev[..., -layers:] = P0_dev[..., -layers:]


def growing_field_rms(P, r, case=MTI, lo=210.0, hi=290.0):
    """rms over the zones with lo < r < hi of the field component that the
    instability makes grow, in the local orthonormal frame on the equator:
    r B^1 (B^1 per unit ln r) for the MTI, r B^3 (B^3 per unit phi) for the
    HBI."""
    m = (r > lo) & (r < hi)
    return float(np.sqrt(np.mean((r[m] * P[case.grows][m]) ** 2)))
