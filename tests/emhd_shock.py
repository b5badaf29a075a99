"""Steady structure of the EMHD shock (Section 8.1.3): the continuous
solution that joins the two states of Table 2 when the pressure anisotropy
relaxes on tau_R = 0.1 with nu = psi c_s^2 tau_R, psi = 3 (gamma = 4/3).
Written here from the model equations of Section 2 (the stress tensor
Eq. fullSEtens, q^mu and Pi^mu nu, the targets Eqs. q0def and dP0def and the
rescaled relaxation equations q_evol_rescaled and dP_evol_rescaled); nothing
here comes from the oracle or the CUDA path.

One dimension, flat space, no time dependence, the field along the flow.
With w = u^1 and gamma_u = u^t = (1 + w^2)^(1/2), b^mu = B^1 (w, gamma_u, 0, 0)
and b-hat^mu = (w, gamma_u, 0, 0).  The conservation laws keep the x-fluxes
rho w, T^{1t} and T^{11} at their upstream values, and the rescaled
relaxation equations become, for X = q~ or dP~,
    d(X w)/dx - (X / 2) dw/dx = -(X - X_0) / tau_R,
with, from b-hat^mu (d_mu Theta + Theta a_mu) and b-hat^mu b-hat^nu d_mu u_nu,
    q_0  = -rho chi (gamma_u Theta' + Theta w w' / gamma_u),
    dP_0 = 3 rho nu (w' - w'/3) = 2 rho nu w'.
Every equation is linear in the derivatives Y' of Y = (rho, u, w, q~, dP~),
so the structure obeys A(Y) Y' = f(Y): the three flux rows and the two
relaxation rows, evaluated from their definitions (derivatives of the fluxes
and of Theta by the complex step, exact to rounding).

The paper solves the same steady equations as a boundary-value problem by a
global Newton iteration on eighth-order central differences.  Here the
structure is integrated instead (an eighth-order Dormand-Prince method,
relative tolerance 1e-13) from the upstream state along its one unstable
direction, which with conduction off is the only way to leave it; the
integration ends at the downstream state, the shift is fixed by putting x = 0
where rho is halfway between the two states.

Heat conduction: with phi = 5 the heat-flux mode travels at
v_q = ((gamma - 1) phi)^(1/2) c_s = 0.563 upstream (the v_q of Eq. modcs),
slower than the upstream flow (0.707), so it cannot run ahead of the shock:
the upstream state becomes a saddle of the steady equations (one unstable
and one stable direction) and its unstable direction misses the downstream
state.  The structure is therefore taken with conduction off; the paper
reports that heat conduction plays a marginal part inside this shock.
"""
from __future__ import annotations

import functools

import numpy as np

from paper_1702_01106_b300 import inputs

GAMMA = 4.0 / 3.0
TAU_R = 0.1
PSI = 3.0
PHI = 5.0
B1 = 1e-5
LEFT = np.array([1.0, 1.0, 1.0, 0.0, 0.0])          # rho, u, u^1, q~, dP~ (Table 2)
RIGHT_PRINTED = np.array([3.08312999, 4.94577705, 0.32434571, 0.0, 0.0])
_H = 1e-30                                           # complex step


class _Model:
    def __init__(self, conduction: bool, phi: float = PHI, higher_order: bool = True):
        self.cond = conduction
        self.phi = phi
        self.ho = 1.0 if higher_order else 0.0

    # thermodynamics and the closure of Section 4
    def thermo(self, Y):
        rho, u, w, qt, dPt = Y
        Pg = (GAMMA - 1.0) * u
        cs2 = GAMMA * Pg / (rho + u + Pg)
        Theta = Pg / rho
        nu = PSI * cs2 * TAU_R
        chi = self.phi * cs2 * TAU_R
        sq = np.sqrt(TAU_R / (chi * rho * Theta * Theta))    # q~ = q sq      (Eq. q)
        sp = np.sqrt(TAU_R / (nu * rho * Theta))             # dP~ = dP sp    (Eq. dP)
        return Pg, Theta, chi, nu, sq, sp

    def fluxes(self, Y):
        """(rho u^1, T^{1t}, T^{11}) from Eq. fullSEtens with q^mu = q b-hat^mu and
        Pi^{mu nu} = -dP (b-hat^mu b-hat^nu - h^{mu nu}/3)."""
        rho, u, w, qt, dPt = Y
        Pg, Theta, chi, nu, sq, sp = self.thermo(Y)
        q = qt / sq if self.cond else 0.0 * qt
        dP = dPt / sp
        gu = np.sqrt(1.0 + w * w)
        ucon = [gu, w]
        bcon = [B1 * w, B1 * gu]
        bsq = -bcon[0] * bcon[0] + bcon[1] * bcon[1]
        bhat = [w, gu]
        gcon = [[-1.0, 0.0], [0.0, 1.0]]

        def T(m, n):
            h = gcon[m][n] + ucon[m] * ucon[n]
            return ((rho + u + 0.5 * bsq) * ucon[m] * ucon[n] + (Pg + 0.5 * bsq) * h - bcon[m] * bcon[n]
                    + q * (bhat[m] * ucon[n] + bhat[n] * ucon[m]) - dP * (bhat[m] * bhat[n] - h / 3.0))

        return np.array([rho * w, T(1, 0), T(1, 1)])

    def _ddir(self, fun, Y, dY):
        """Directional derivative of fun at Y along dY (complex step)."""
        return np.imag(fun(Y.astype(complex) + 1j * _H * dY)) / _H

    def equations(self, Y, dY):
        """The five steady equations E(Y, Y') (zero on the structure)."""
        rho, u, w, qt, dPt = Y
        Pg, Theta, chi, nu, sq, sp = self.thermo(Y)
        gu = np.sqrt(1.0 + w * w)
        dw = dY[2]
        dTheta = self._ddir(lambda Z: (GAMMA - 1.0) * Z[1] / Z[0], Y, dY)
        E = np.empty(5)
        E[:3] = self._ddir(self.fluxes, Y, dY)
        if self.cond:
            q0 = -rho * chi * (gu * dTheta + Theta * w * dw / gu)
            E[3] = w * dY[3] + qt * dw - self.ho * 0.5 * qt * dw + (qt - sq * q0) / TAU_R
        else:
            E[3] = dY[3]
        dP0 = 3.0 * rho * nu * (dw - dw / 3.0)
        E[4] = w * dY[4] + dPt * dw - self.ho * 0.5 * dPt * dw + (dPt - sp * dP0) / TAU_R
        return E

    def slope(self, Y):
        f = -self.equations(Y, np.zeros(5))
        A = np.empty((5, 5))
        for k in range(5):
            e = np.zeros(5)
            e[k] = 1.0
            A[:, k] = self.equations(Y, e) + f
        return np.linalg.solve(A, f)

    def jacobian(self, Y, h=1e-7):
        """d(Y')/dY at Y (central differences), for the fixed-point analysis."""
        J = np.empty((5, 5))
        for k in range(5):
            e = np.zeros(5)
            e[k] = h
            J[:, k] = (self.slope(Y + e) - self.slope(Y - e)) / (2 * h)
        return J


def model(conduction: bool = False, phi: float = PHI, higher_order: bool = True) -> _Model:
    return _Model(conduction, phi, higher_order)


def fixed_point_rates(Y, conduction: bool, phi: float = PHI):
    """The nonzero eigenvalues of d(Y')/dY at a uniform state (growth rates in
    x of the steady perturbations on the constant-flux surface)."""
    ev = np.linalg.eigvals(model(conduction, phi).jacobian(np.asarray(Y, dtype=float)))
    return np.sort(ev.real[np.abs(ev) > 1e-6 * np.abs(ev).max()])


@functools.lru_cache(maxsize=None)
def structure():
    """(x, Y(x)) of the structure on a dense table, x = 0 at the midpoint in
    rho; Y upstream and downstream of the table is the end state."""
    from scipy.integrate import solve_ivp

    m = model(conduction=False)
    J = m.jacobian(LEFT)
    ev, V = np.linalg.eig(J)
    k = int(np.argmax(ev.real))
    v = V[:, k].real
    v = v * np.sign(v[0]) / np.abs(v).max()       # compressive side: rho rises
    Y0 = LEFT + 1e-13 * v
    span = 8.0
    sol = solve_ivp(lambda x, y: m.slope(y), (0.0, span), Y0, method="DOP853",
                    rtol=1e-13, atol=1e-16, dense_output=True)
    assert sol.status == 0
    x = np.linspace(0.0, span, 160001)
    Y = sol.sol(x)
    mid = 0.5 * (LEFT[0] + Y[0, -1])
    i = int(np.argmax(Y[0] > mid))
    # refine the midpoint on the dense output (bisection)
    a, b = x[i - 1], x[i]
    for _ in range(80):
        c = 0.5 * (a + b)
        if sol.sol(c)[0] > mid:
            b = c
        else:
            a = c
    xc = 0.5 * (a + b)
    return x - xc, Y, sol, xc


def profile(xs):
    """Y = (rho, u, u^1, q~, dP~) of the structure at the points xs."""
    x, Y, sol, xc = structure()
    xs = np.asarray(xs, dtype=float)
    out = np.empty((5, xs.size))
    inside = (xs >= x[0]) & (xs <= x[-1])
    out[:, inside] = sol.sol(xs[inside] + xc)
    out[:, xs < x[0]] = LEFT[:, None]
    out[:, xs > x[-1]] = Y[:, -1:]
    return out


def shock_structure_problem(n, tol=1e-12, x_range=(-1.0, 3.0)):
    """1-D run through the structure: outflow boundaries, conduction off,
    viscosity and the higher-order term on, tau_R = 0.1, psi = 3."""
    return inputs.Problem(dim=2, n=(n, 1, 1), x_start=(x_range[0], 0.0, 0.0), x_end=(x_range[1], 1.0, 1.0),
                          bc=((inputs.BC_OUTFLOW, inputs.BC_OUTFLOW), (inputs.BC_PERIODIC, inputs.BC_PERIODIC),
                              (inputs.BC_PERIODIC, inputs.BC_PERIODIC)),
                          gamma=GAMMA, conduction=False, viscosity=True, higher_order=True,
                          tau_R=TAU_R, phi=PHI, psi=PSI, tol=tol)


def structure_state(prob):
    """Primitives [10, 1, 1, n] of the structure at the zone centres, and x."""
    n = prob.n[0]
    x = prob.x_start[0] + (np.arange(n) + 0.5) * prob.dx[0]
    Y = profile(x)
    P = np.zeros((10, n))
    P[0], P[1], P[2] = Y[0], Y[1], Y[2]
    P[5] = B1
    P[8], P[9] = Y[3], Y[4]
    return P.reshape(10, 1, 1, n), x
