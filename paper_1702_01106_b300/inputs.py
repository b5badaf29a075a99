"""Seeded synthetic inputs and problem descriptions for the implicit EMHD step.

This module is shared by the CUDA path and by the test oracle.  It holds no
arithmetic of the method itself: only problem parameters, grids and initial
states, each following the paper's test setups (Section 8) or the workload
recipes stated in the design notes.  Random numbers come from numpy's
counter-based Philox generator, seeded per field.

State layout everywhere: float64 array P[10, n3, n2, n1] (X1 fastest) with the
fields (rho, u, u1, u2, u3, B1, B2, B3, q~, dP~); q~ and dP~ are the rescaled
heat flux and pressure anisotropy of Section 4 (Eqs. q, dP).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

NVAR = 10
FIELDS = ("rho", "u", "u1", "u2", "u3", "B1", "B2", "B3", "qt", "dPt")

BC_PERIODIC, BC_OUTFLOW, BC_REFLECT = 0, 1, 2
RECON_MC, RECON_WENO5 = 0, 1
METRIC_MINKOWSKI = 0


@dataclass
class Problem:
    """Grid, physics and solver parameters of one run."""

    dim: int = 2
    n: tuple = (64, 64, 1)
    x_start: tuple = (0.0, 0.0, 0.0)
    x_end: tuple = (1.0, 1.0, 1.0)
    bc: tuple = ((BC_PERIODIC, BC_PERIODIC),) * 3
    metric: int = METRIC_MINKOWSKI
    recon: int = RECON_MC
    theta: float = 2.0          # generalized minmod parameter (2 = MC)
    conduction: bool = True
    viscosity: bool = True
    higher_order: bool = True
    gamma: float = 4.0 / 3.0
    phi: float = 1.0
    psi: float = 1.0
    tau_R: float = 1.0
    tol: float = 1e-10
    eps_fd: float = 2.0 ** -26
    k_max: int = 30
    ls_max: int = 10
    spin: float = 0.0
    h_mks: float = 0.3

    @property
    def dx(self):
        return tuple((self.x_end[d] - self.x_start[d]) / self.n[d] for d in range(3))

    @property
    def zones(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def zone_centers(prob: Problem):
    """Coordinates (x1, x2, x3) of zone centres, each shaped [n3, n2, n1]."""
    ax = [prob.x_start[d] + (np.arange(prob.n[d]) + 0.5) * prob.dx[d] for d in range(3)]
    x3, x2, x1 = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return x1, x2, x3


# ---------------------------------------------------------------- linear mode
# Table 1 (Section 8.1.1): background state and the eigenvector of the
# propagating, decaying EMHD mode with k = (2 pi, 4 pi), gamma = 4/3,
# tau_R = 1, chi = nu = c_s^2 tau_R.  The q and dP entries are the physical
# heat flux and pressure anisotropy.
TABLE1_BACKGROUND = np.array([1.0, 2.0, 0.0, 0.0, 0.0, 0.1, 0.3, 0.0, 0.0, 0.0])
TABLE1_EIGENVECTOR = np.array([
    -0.518522524082246 - 0.1792647678001878j,
    0.5516170736393813 + 0.0j,
    0.008463122479547856 + 0.011862022608466367j,
    -0.16175466371870734 - 0.034828080823603294j,
    0.0 + 0.0j,
    -0.05973794979640743 - 0.03351707506150924j,
    0.02986897489820372 + 0.016758537530754618j,
    0.0 + 0.0j,
    0.5233486841539436 + 0.04767672501939603j,
    0.2909106062057657 + 0.02159452055336572j,
])
TABLE1_OMEGA = -0.5533585207638141 - 3.6262571286888425j
TABLE1_K = (2.0 * math.pi, 4.0 * math.pi)


def linear_mode_problem(n: int = 64, **kw) -> Problem:
    """Config: 2-D Minkowski linear mode on [0,1]^2, periodic (Section 8.1.1)."""
    base = dict(dim=2, n=(n, n, 1), gamma=4.0 / 3.0, tau_R=1.0, phi=1.0, psi=1.0)
    base.update(kw)
    return Problem(**base)


def rescaled_eigenvector(prob: Problem) -> np.ndarray:
    """Table 1 eigenvector with its q, dP entries expressed in the rescaled
    primitives q~ = q (tau_R/(chi rho Theta^2))^(1/2), dP~ = dP (tau_R/(nu rho
    Theta))^(1/2) at the background (Eqs. q, dP with chi = phi c_s^2 tau_R,
    nu = psi c_s^2 tau_R), which is exact to first order in the amplitude."""
    rho, u = TABLE1_BACKGROUND[0], TABLE1_BACKGROUND[1]
    g = prob.gamma
    pg = (g - 1.0) * u
    theta = pg / rho
    cs = math.sqrt(g * pg / (rho + g * u))
    v = TABLE1_EIGENVECTOR.copy()
    v[8] = v[8] / (cs * theta * math.sqrt(prob.phi * rho))
    v[9] = v[9] / (cs * math.sqrt(prob.psi * rho * theta))
    return v


def linear_mode_state(prob: Problem, amp: float = 1e-4, phase: float = 0.0, t: float = 0.0) -> np.ndarray:
    """P = P0 + Re(A dP exp(i(k.x + phase) + omega t)) on the zone centres."""
    x1, x2, _ = zone_centers(prob)
    v = rescaled_eigenvector(prob)
    wave = np.exp(1j * (TABLE1_K[0] * x1 + TABLE1_K[1] * x2 + phase) + TABLE1_OMEGA * t)
    P = np.empty((NVAR,) + x1.shape)
    for a in range(NVAR):
        P[a] = TABLE1_BACKGROUND[a] + np.real(amp * v[a] * wave)
    return P


def linear_mode_phase(seed: int = 1) -> float:
    """Seeded phase 2 pi U(0,1) of the linear-mode workload."""
    return 2.0 * math.pi * float(np.random.Generator(np.random.Philox(seed)).random())


# ---------------------------------------------------------------- turbulent box
def turbulent_box_problem(n: int = 1024, **kw) -> Problem:
    """Config: 2-D special-relativistic EMHD box, periodic, gamma = 4/3,
    tau_R = 1, phi = psi = 1, MC reconstruction, dt = 0.5/n."""
    base = dict(dim=2, n=(n, n, 1), gamma=4.0 / 3.0, tau_R=1.0, phi=1.0, psi=1.0)
    base.update(kw)
    return Problem(**base)


def turbulent_box_state(prob: Problem, seed_rho: int = 2, seed_vel: int = 3, kmax: int = 8,
                        vrms: float = 0.1, rho_noise: float = 1e-3) -> np.ndarray:
    """rho = 1 + 1e-3 N(0,1); u = 1; B = (0.2, 0.1, 0); u1, u2 = sums over
    0 < |n| <= kmax of a_n cos(2 pi n.x + phi_n), a_n ~ N(0,1), phi_n ~ U(0, 2pi),
    each rescaled to rms vrms; u3 = q~ = dP~ = 0."""
    n1, n2 = prob.n[0], prob.n[1]
    rng_r = np.random.Generator(np.random.Philox(seed_rho))
    rng_v = np.random.Generator(np.random.Philox(seed_vel))
    P = np.zeros((NVAR, 1, n2, n1))
    P[0, 0] = 1.0 + rho_noise * rng_r.standard_normal((n2, n1))
    P[1] = 1.0
    P[5] = 0.2
    P[6] = 0.1
    modes = [(a, b) for a in range(-kmax, kmax + 1) for b in range(-kmax, kmax + 1)
             if 0 < a * a + b * b <= kmax * kmax]
    for comp in (2, 3):
        amps = rng_v.standard_normal(len(modes))
        phases = 2.0 * math.pi * rng_v.random(len(modes))
        # Sum of cosines evaluated exactly on the zone centres with an inverse FFT.
        spec = np.zeros((n2, n1), dtype=complex)
        for (a, b), am, ph in zip(modes, amps, phases):
            # cos(2pi(a x + b y) + ph) at x = (i + 1/2)/n1, y = (j + 1/2)/n2
            shift = np.exp(1j * (ph + math.pi * (a / n1 + b / n2)))
            spec[b % n2, a % n1] += 0.5 * am * shift
            spec[(-b) % n2, (-a) % n1] += 0.5 * am * np.conj(shift)
        field = np.real(np.fft.ifft2(spec) * (n1 * n2))
        field *= vrms / math.sqrt(np.mean(field * field))
        P[comp, 0] = field
    return P


def batched_boxes(seed_size: int = 6, seed_angle: int = 7, count: int = 64,
                  sides=(128, 256, 512, 1024), amp: float = 1e-4):
    """Config: `count` independent 2-D boxes with sides drawn uniformly from
    `sides`; each has the linear-mode initial state with its background field
    rotated by a seeded angle (|B| kept); dt = 0.5/side."""
    rs = np.random.Generator(np.random.Philox(seed_size))
    ra = np.random.Generator(np.random.Philox(seed_angle))
    out = []
    bmag = math.hypot(0.1, 0.3)
    for _ in range(count):
        side = int(sides[int(rs.integers(0, len(sides)))])
        ang = 2.0 * math.pi * float(ra.random())
        prob = linear_mode_problem(side)
        P = linear_mode_state(prob, amp=amp)
        P[5] = P[5] - 0.1 + bmag * math.cos(ang)
        P[6] = P[6] - 0.3 + bmag * math.sin(ang)
        out.append((prob, P, 0.5 / side))
    return out
