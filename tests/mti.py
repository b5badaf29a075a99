"""Magneto-thermal instability (Section 9.1): a hydrostatic polytropic
atmosphere around a Schwarzschild black hole (M = 1) whose temperature falls
outwards, threaded by a weak azimuthal field, with heat conducted along the
field.  Written from the model and the linear theory the paper cites
(Balbus 2000); nothing here comes from the oracle or the CUDA path.

Equilibrium.  A static fluid moves along the Killing vector d_t, so its
four-acceleration is a_mu = d_mu ln alpha_t, alpha_t = (1 - 2/r)^(1/2), and
momentum balance reads dP/dr = -(rho + u + P) d ln alpha_t/dr.  With the
polytrope P = K rho^G (G = 4/3, K = 1e-4: the paper's MTI setup), u = P/(gamma - 1)
and Theta = P/rho = K rho^(G - 1), dP/rho = G/(G - 1) dTheta, so
    G/(G - 1) dTheta / (1 + c Theta) = -d ln alpha_t,  c = gamma/(gamma - 1),
whose solution from Theta_0 at r = 200 is
    1 + c Theta = (1 + c Theta_0) (alpha_0/alpha_t)^(c (G - 1)/G).
`theta_ode` integrates the balance itself as an independent check.  The
equilibrium is Schwarzschild-stable (G < gamma = 5/3: the entropy rises
outwards) but its temperature falls outwards.

Field and heat flux.  B^phi = 1e-3 / sqrt(-g) (the paper's weak azimuthal
field; b^2/P ~ 1e-15, so magnetic tension plays no part) is perpendicular
to the temperature gradient, so the initial heat flux and its target vanish.
The closure follows the paper's choice chi = c_s R, tau_R = R/c_s: with
chi = phi c_s^2 tau_R this is phi = 1 and tau_R = R/c_s, which the library's
tau_R = tau_0 r^(3/2) matches to within a few per cent over 200 <= r <= 300
(c_s^2 falls nearly as 1/r); tau_0 is fitted at r = 250.  Viscosity is off
(the section names no viscosity for this run).

Linear theory.  With conduction along the field much faster than the
dynamics, a weakly magnetised atmosphere is unstable where dT/dz < 0, and
the fastest modes (wavevector nearly along the field, displacement along
gravity) grow at sigma = (g |d ln T/dz|)^(1/2) (Balbus 2000).  Here
g = d ln alpha_t/dr and T = Theta; sigma^-1 is 2.5e3 M at r = 200 (the
paper's "dynamical time scale ~2500 M" there, and its fitted growth time
~2400 M) and 4.3e3 M at r = 300.

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
G_POLY = 4.0 / 3.0           # the atmosphere's polytropic index (Schwarzschild-stable: G < gamma)
K_POLY = 1e-4
R_IN, R_OUT = 200.0, 300.0
THETA0 = 1e-3                # Theta at r = 200 (rho_0 = (Theta_0/K)^(1/(G-1)) = 1000, P_0 = 1)
B_PHI = 1e-3                 # B^phi = B_PHI / sqrt(-g)
NOISE = 0.004                # seeded fluctuations of u~^1, in units of the local sound speed (see mti_state)
HOLD = 3                     # radial layers held at the equilibrium at each end


def alpha_t(r):
    return np.sqrt(1.0 - 2.0 / np.asarray(r, dtype=float))


def gravity(r):
    """g = d ln alpha_t / dr."""
    r = np.asarray(r, dtype=float)
    return 1.0 / (r * r * (1.0 - 2.0 / r))


def theta_of_r(r):
    """Closed form of the hydrostatic polytrope (module docstring)."""
    c = GAMMA / (GAMMA - 1.0)
    e = c * (G_POLY - 1.0) / G_POLY
    return ((1.0 + c * THETA0) * (alpha_t(R_IN) / alpha_t(r)) ** e - 1.0) / c


def theta_ode(r):
    """Momentum balance integrated from r = 200 (eighth-order Dormand-Prince)
    in P, with rho = (P/K)^(1/G): Theta = P / rho."""
    from scipy.integrate import solve_ivp

    def rhs(rr, y):
        P = y[0]
        rho = (P / K_POLY) ** (1.0 / G_POLY)
        return [-(rho + P / (GAMMA - 1.0) + P) * float(gravity(rr))]

    rho0 = (THETA0 / K_POLY) ** (1.0 / (G_POLY - 1.0))
    sol = solve_ivp(rhs, (R_IN, R_OUT), [THETA0 * rho0], method="DOP853", rtol=1e-13, atol=1e-18,
                    dense_output=True)
    assert sol.status == 0
    P = sol.sol(np.asarray(r, dtype=float))[0]
    return P / (P / K_POLY) ** (1.0 / G_POLY)


def sound_speed(r):
    th = theta_of_r(r)
    return np.sqrt(GAMMA * th / (1.0 + GAMMA / (GAMMA - 1.0) * th))


def growth_rate(r):
    """Fastest MTI growth rate (g |d ln Theta/dr|)^(1/2) at r (centred
    difference of the closed form)."""
    r = np.asarray(r, dtype=float)
    h = 1e-4 * r
    dlnT = (np.log(theta_of_r(r + h)) - np.log(theta_of_r(r - h))) / (2.0 * h)
    return np.sqrt(gravity(r) * np.abs(dlnT))


def tau0():
    """tau_R = tau_0 r^(3/2) equal to R / c_s at r = 250."""
    return 250.0 / float(sound_speed(250.0)) / 250.0 ** 1.5


def mti_problem(n1=64, n2=4, n3=128, tol=1e-10):
    return inputs.Problem(dim=3, n=(n1, n2, n3), x_start=(math.log(R_IN), 0.45, 0.0),
                          x_end=(math.log(R_OUT), 0.55, math.pi),
                          bc=((inputs.BC_OUTFLOW, inputs.BC_OUTFLOW), (inputs.BC_REFLECT, inputs.BC_REFLECT),
                              (inputs.BC_PERIODIC, inputs.BC_PERIODIC)),
                          metric=inputs.METRIC_MKS_KERR, spin=0.0, h_mks=1.0, gamma=GAMMA,
                          conduction=True, viscosity=False, higher_order=True,
                          phi=1.0, psi=1.0, tau_R=tau0(), tol=tol)


def sqrt_g(prob, r, th):
    """sqrt(-g) of modified Kerr-Schild coordinates with a = 0, h = 1:
    r^2 sin(theta) (Kerr-Schild) times dr/dX^1 = r and dtheta/dX^2 = pi."""
    return r ** 3 * np.sin(th) * math.pi


def mti_state(prob, seed=11, noise=NOISE):
    """Primitives [10, n3, n2, n1] of the equilibrium with seeded u~^1
    fluctuations of `noise` times the local sound speed (the paper seeds
    about 4 %; 0.4 % keeps the linear phase going two e-folds longer before
    the field saturates, which is where the growth rate is measured); also
    returns r and theta of the zone centres."""
    x1, x2, _ = inputs.zone_centers(prob)
    r = np.exp(x1)
    th = math.pi * x2
    Theta = theta_of_r(r)
    rho = (Theta / K_POLY) ** (1.0 / (G_POLY - 1.0))
    Pg = rho * Theta
    ut = 1.0 / alpha_t(r)
    P = np.zeros((10,) + tuple(prob.n[::-1]))
    P[0] = rho
    P[1] = Pg / (GAMMA - 1.0)
    # the static fluid's normal-observer velocity in Kerr-Schild coordinates
    # (a = 0), per unit X^1 = ln r
    P[2] = 2.0 * ut / (r * r + 2.0 * r)
    rng = np.random.default_rng(seed)
    P[2] += noise * sound_speed(r) / r * rng.uniform(-1.0, 1.0, size=P[2].shape)
    P[7] = B_PHI / sqrt_g(prob, r, th)
    return P, r, th


def equilibrium(prob):
    """The state without the fluctuations (what the held layers are reset to)."""
    P, r, th = mti_state(prob, noise=0.0)
    return P


def mti_dt(prob, cfl=0.5):
    return inputs.torus_dt(prob, cfl)


def hold_boundaries(P_dev, P0_dev, layers=HOLD):
    """Reset the outermost `layers` radial layers at both ends to the
    equilibrium (device tensors [10, n3, n2, n1])."""
    P_dev[..., :layers] = P0_dev[..., :layers]
    P_dev[..., -layers:] = P0_dev[..., -layers:]


def radial_field_rms(P, r, lo=210.0, hi=290.0):
    """rms of the radial field b^r ~ r B^1 (B^1 per unit ln r) over the
    zones with lo < r < hi."""
    m = (r > lo) & (r < hi)
    return float(np.sqrt(np.mean((r[m] * P[5][m]) ** 2)))
