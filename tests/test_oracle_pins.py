"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden), closed forms, textbook special cases, library
routines, brute force on tiny inputs, or convergence rates.  None needs a GPU.
"""
import math

import numpy as np
import pytest

from paper_1702_01106_b300 import inputs
from tests.oracle_helpers import read_golden, random_zone_state, zone_vector, minkowski_derived


def _dispersion(orc, prob, P0, k):
    """Eigenvalues/vectors omega of the linearised system for P ~ exp(i k.x + omega t):
    omega (dU/dP - dS/dP_t) dP = -[i k_j (dF^j/dP - dS/dP_j) - dS/dP] dP."""
    MU, A, SP, SD = orc.linearize(prob, P0)
    M = MU - SD[0]
    K = -SP.astype(complex)
    for j in range(len(k)):
        K = K + 1j * k[j] * (A[j] - SD[j + 1])
    w, V = np.linalg.eig(-np.linalg.solve(M, K))
    return w, V


# ---------------------------------------------------------------- Table 1
def test_linear_mode_eigenvalue_and_eigenvector(orc):
    rows = read_golden("table1_linear_mode.txt")
    omega = complex(float(rows[0][1]), float(rows[0][2]))
    P0 = np.array([float(r[1]) for r in rows[1:]])
    ev = np.array([complex(float(r[2]), float(r[3])) for r in rows[1:]])
    prob = inputs.linear_mode_problem(8)
    w, V = _dispersion(orc, prob, P0, (2 * math.pi, 4 * math.pi))
    i = int(np.argmin(np.abs(w - omega)))
    assert abs(w[i] - omega) < 1e-9 * abs(omega)
    # the table lists physical q, dP; the oracle's primitives are q~, dP~
    rho, u, g = P0[0], P0[1], prob.gamma
    pg = (g - 1) * u
    cs = math.sqrt(g * pg / (rho + g * u))
    v = V[:, i].copy()
    v[8] *= cs * (pg / rho) * math.sqrt(prob.phi * rho)
    v[9] *= cs * math.sqrt(prob.psi * pg)
    v = v / v[1] * ev[1]
    assert np.max(np.abs(v - ev)) < 1e-9
    assert abs(np.linalg.norm(ev) - 1.0) < 1e-9           # a unit eigenvector
    assert abs(2 * math.pi * ev[5] + 4 * math.pi * ev[6]) < 1e-12  # k . dB = 0


def test_linear_mode_all_modes_stable(orc):
    """Causal, stable theory: no linear mode grows (all Re omega <= 0)."""
    prob = inputs.linear_mode_problem(8)
    for k in [(2 * math.pi, 4 * math.pi), (10.0, 0.0), (0.0, 7.0), (30.0, -20.0)]:
        w, _ = _dispersion(orc, prob, inputs.TABLE1_BACKGROUND, k)
        assert np.max(w.real) < 1e-10


def test_printed_induction_sign_makes_alfven_waves_grow(orc):
    """The induction flux sign reading: flipping the sign of the B-flux block
    (the printed form) gives a real, growing omega; the oracle's form does not."""
    prob = inputs.linear_mode_problem(8)
    P0 = inputs.TABLE1_BACKGROUND
    MU, A, SP, SD = orc.linearize(prob, P0)
    k = (2 * math.pi, 4 * math.pi)
    A2 = A.copy()
    A2[:, 5:8, :] *= -1.0
    M = MU - SD[0]
    K = -SP + 1j * k[0] * (A2[0] - SD[1]) + 1j * k[1] * (A2[1] - SD[2])
    w = np.linalg.eigvals(-np.linalg.solve(M, K))
    assert np.max(w.real) > 1.0


@pytest.mark.slow
def test_linear_mode_second_order_convergence(orc):
    """Section 8.1.1: the L1 error against the exact decaying mode at t = 0.5
    falls at second order."""
    errs = []
    for n in (16, 32, 64):
        prob = inputs.linear_mode_problem(n, tol=1e-12)
        P = inputs.linear_mode_state(prob, amp=1e-4)
        dt = 0.5 / n
        for _ in range(n):
            P, it, st, _ = orc.step(prob, P, dt)
            assert (st == 0).all()
        exact = inputs.linear_mode_state(prob, amp=1e-4, t=0.5)
        errs.append(np.abs(P - exact).mean())
    order1 = math.log2(errs[0] / errs[1])
    order2 = math.log2(errs[1] / errs[2])
    assert order1 > 1.8 and order2 > 1.8, errs
    assert errs[2] < 1e-2 * 1e-4  # well below the amplitude


# ---------------------------------------------------------------- firehose
def test_firehose_growth_rate(orc):
    rows = {r[0]: float(r[1]) for r in read_golden("firehose.txt")}
    prob = inputs.linear_mode_problem(8, tau_R=1e6)
    rho, u, g = 1.0, 2.0, prob.gamma
    pg = (g - 1) * u
    cs = math.sqrt(g * pg / (rho + g * u))
    P0 = np.array([rho, u, 0, 0, 0, 0.1, 0, 0, 0, -0.011 / (cs * math.sqrt(prob.psi * pg))])
    w, V = _dispersion(orc, prob, P0, (2 * math.pi, 0.0))
    i = int(np.argmax(w.real))
    assert abs(w[i].imag) < 1e-10
    # Gamma = 0.10367 here; the paper's 0.1036 matches it truncated to four
    # digits.  The printed eigenvector fixes the digit: A/B = Gamma/(k B^1) for
    # this Alfven mode, and 0.1628/0.9867 = 0.16499 matches 0.10367/(0.2 pi)
    # = 0.16500 while the rounded reading 0.10360 would give 0.16488.
    assert 0.0 <= w[i].real - rows["growth"] < 1e-4
    ratio = abs(V[3, i] / V[6, i])
    assert abs(ratio - rows["A"] / rows["B"]) < 6e-5
    assert abs(ratio - w[i].real / (2 * math.pi * 0.1)) < 1e-9


# ---------------------------------------------------------------- Table 2
def test_shock_jump_conditions_table2(orc):
    rows = read_golden("table2_shock_states.txt")
    L = np.zeros(10); R = np.zeros(10)
    for a, r in enumerate(rows):
        L[a], R[a] = float(r[1]), float(r[2])
    prob = inputs.linear_mode_problem(8, conduction=False, viscosity=False, higher_order=False)
    _, FL, _ = orc.point(prob, L)
    _, FR, _ = orc.point(prob, R)
    for a in range(5):
        assert abs(FL[0][a] - FR[0][a]) <= 2e-8 * max(1.0, abs(FL[0][a])), (a, FL[0][a], FR[0][a])
    assert abs(FL[0][0] - 1.0) < 1e-12                     # mass flux rho u^1 = 1
    # printed four-digit fluxes (Section 8.1.2 discussion): momentum 2.6667, energy 3.2998
    assert abs(FL[0][2] - 2.6667) < 1e-4
    assert abs(-FL[0][1] - 3.2998) < 1e-4


# ---------------------------------------------------------------- wave speeds
def test_sound_speed_velocity_addition(orc):
    """Closures and field off: the bound is c_s, boosted by relativistic velocity addition."""
    prob = inputs.linear_mode_problem(8, conduction=False, viscosity=False)
    rng = np.random.default_rng(5)
    for _ in range(20):
        rho, u = rng.uniform(0.2, 3), rng.uniform(0.2, 3)
        ux = rng.uniform(-2, 2)
        P = np.array([rho, u, ux, 0, 0, 0, 0, 0, 0, 0])
        _, _, c = orc.point(prob, P)
        g = prob.gamma
        cs = math.sqrt(g * (g - 1) * u / (rho + g * u))
        v = ux / math.sqrt(1 + ux * ux)
        cp = (v + cs) / (1 + v * cs)
        cm = (v - cs) / (1 - v * cs)
        assert abs(c[0][1] - cp) < 1e-13 and abs(c[0][0] - cm) < 1e-13
        # transverse direction: v_y = 0, speeds +- cs / gamma-factor form
        assert abs(c[1][1] + c[1][0]) < 1e-13


@pytest.mark.parametrize("row", read_golden("wave_speed_limits.txt"))
def test_psi_max_causality_limit(orc, row):
    g, psi_max, digits = float(row[0]), float(row[1]), int(row[2])

    def vmax(psi):
        prob = inputs.linear_mode_problem(8, gamma=g, phi=psi, psi=psi)
        P = np.array([1e-12, 1.0, 0, 0, 0, 0, 0, 0, 0, 0])  # c_s^2 -> gamma - 1
        _, _, c = orc.point(prob, P)
        return c[0][1]

    lo, hi = 0.01, 5.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if vmax(mid) < 1.0:
            lo = mid
        else:
            hi = mid
    assert round(lo, digits) == pytest.approx(psi_max, abs=0.6 * 10 ** (-digits) + 1e-12)


# ---------------------------------------------------------------- Jacobian
def test_fd_jacobian_matches_complex_step(orc):
    prob = inputs.linear_mode_problem(8)
    rng = np.random.default_rng(11)
    for _ in range(10):
        Pn = random_zone_state(rng)
        PE = Pn * (1 + 1e-3 * rng.standard_normal(10))
        zc = zone_vector(orc, prob, Pn, PE, 0.01, divF=rng.normal(0, 0.1, 10),
                         dTh=np.r_[0, rng.normal(0, 0.1, 3)], du=np.vstack([np.zeros(4), rng.normal(0, 0.1, (3, 4))]),
                         divu=0.05)
        P = Pn * (1 + 1e-2 * rng.standard_normal(10))
        Jfd = orc.zone_jacobian(prob, zc, P, "fd")
        Jcs = orc.zone_jacobian(prob, zc, P, "cs")
        scale = np.abs(Jcs).max()
        # one-sided differences: truncation error O(eps) of the column scale
        assert np.abs(Jfd - Jcs).max() < 8 * prob.eps_fd * scale
        # the magnetic rows depend only on B (and linearly)
        assert np.all(Jcs[5:8, :5] == 0) and np.all(Jcs[5:8, 8:] == 0)


def test_fd_column_of_a_small_component(orc):
    """small() (Section 3.1) perturbs a component just above 5 eps by eps of
    itself, i.e. by 5 eps^2: with the default eps that column still stands
    far enough above the residual's rounding to match the complex-step
    column to 1e-4 of the Jacobian's scale (at eps = 2^-26 the same columns
    were off by 1-2 % of it)."""
    prob = inputs.linear_mode_problem(8)
    eps = prob.eps_fd
    rng = np.random.default_rng(13)
    for sgn in (1.0, -1.0):
        Pn = random_zone_state(rng)
        Pn[8] = sgn * 6 * eps
        Pn[9] = -sgn * 6 * eps
        PE = Pn.copy()
        zc = zone_vector(orc, prob, Pn, PE, 0.01, divF=rng.normal(0, 0.1, 10),
                         dTh=np.r_[0, rng.normal(0, 0.1, 3)], du=np.vstack([np.zeros(4), rng.normal(0, 0.1, (3, 4))]),
                         divu=0.05)
        Jfd = orc.zone_jacobian(prob, zc, Pn, "fd")
        Jcs = orc.zone_jacobian(prob, zc, Pn, "cs")
        scale = np.abs(Jcs).max()
        assert np.abs(Jfd[:, 8:] - Jcs[:, 8:]).max() < 1e-4 * scale


def test_fd_columns_of_a_cold_zone(orc):
    """A cold, tenuous zone (rho = 1e-7, u = 1e-11, as in the torus
    atmosphere): the rho and u columns of the FD Jacobian (Section 3.1) match
    the complex-step columns to 1e-4 of their scale.  An absolute step of
    eps on u (small() taken for every component below 5 eps) moves u by
    5e4 times itself, and that column is off by order one."""
    prob = inputs.linear_mode_problem(8)
    rng = np.random.default_rng(17)
    Pn = np.array([1e-7, 1e-11, 0.01, -0.02, 0.005, 1e-6, 2e-6, 0.0, 1e-9, -1e-9])
    zc = zone_vector(orc, prob, Pn, Pn.copy(), 0.01, divF=1e-8 * rng.normal(0, 1, 10))
    Jfd = orc.zone_jacobian(prob, zc, Pn, "fd")
    Jcs = orc.zone_jacobian(prob, zc, Pn, "cs")
    for col in (0, 1):
        scale = np.abs(Jcs[:, col]).max()
        assert np.abs(Jfd[:, col] - Jcs[:, col]).max() < 1e-4 * scale, col


def test_complex_step_matches_central_differences(orc):
    """Independent check of the complex-step Jacobian itself."""
    prob = inputs.linear_mode_problem(8)
    rng = np.random.default_rng(12)
    Pn = random_zone_state(rng)
    zc = zone_vector(orc, prob, Pn, Pn, 0.02, divu=0.1)
    P = Pn * 1.01
    Jcs = orc.zone_jacobian(prob, zc, P, "cs")
    Jc = np.zeros((10, 10))
    for j in range(10):
        h = 1e-5 * max(1.0, abs(P[j]))
        e = np.zeros(10); e[j] = h
        Jc[:, j] = (orc.zone_residual(prob, zc, P + e) - orc.zone_residual(prob, zc, P - e)) / (2 * h)
    assert np.abs(Jc - Jcs).max() < 1e-7 * np.abs(Jcs).max()


# ---------------------------------------------------------------- LU
def test_lu_solve_matches_lapack_and_pivots(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        J = rng.standard_normal((10, 10))
        b = rng.standard_normal(10)
        x, rc = orc.lu_solve(J, b)
        assert rc == 0
        assert np.allclose(x, np.linalg.solve(J, b), rtol=1e-10, atol=1e-12)
    # zero leading pivots need row exchanges
    J = np.eye(10)[::-1] * np.arange(1, 11)
    b = np.arange(10.0)
    x, rc = orc.lu_solve(J, b)
    assert rc == 0 and np.allclose(J @ x, b)
    x, rc = orc.lu_solve(np.zeros((10, 10)), b)
    assert rc == 1


# ---------------------------------------------------------------- Newton
def _manufactured(orc, prob, rng, noise):
    Pstar = random_zone_state(rng)
    Pn = Pstar * (1 + noise * rng.standard_normal(10))
    PE = Pn.copy()
    zc = zone_vector(orc, prob, Pn, PE, 0.01, divF=np.zeros(10),
                     dTh=np.r_[0, rng.normal(0, 0.1, 3)], du=np.vstack([np.zeros(4), rng.normal(0, 0.1, (3, 4))]),
                     divu=0.02)
    r = orc.zone_residual(prob, zc, Pstar)
    scale = zc[59:69]
    zc[10:20] = -r / scale          # divF := -R(P*), so that R(P*) = 0
    return Pstar, Pn, zc


def test_newton_manufactured_root(orc):
    prob = inputs.linear_mode_problem(8, tol=1e-13)
    rng = np.random.default_rng(21)
    for _ in range(25):
        Pstar, Pn, zc = _manufactured(orc, prob, rng, 1e-2)
        assert np.abs(orc.zone_residual(prob, zc, Pstar)).max() < 1e-14
        P, iters, status, evals = orc.zone_newton(prob, zc, Pn)
        assert status == 0, status
        assert 1 <= iters <= 8
        assert np.abs(P - Pstar).max() < 1e-10 * (1 + np.abs(Pstar).max())


def _paper_newton(orc, prob, zc, P):
    """Section 3 written out independently: Newton with the FD Jacobian of
    Section 3.1 (LAPACK solve) and the quadratic backtracking of Section 3.2."""
    r = orc.zone_residual(prob, zc, P); evals = 1
    f = r @ r
    k = 0
    while np.abs(r).max() > prob.tol and k < prob.k_max:
        J = orc.zone_jacobian(prob, zc, P, "fd"); evals += 10
        d = np.linalg.solve(J, -r)
        lam = 1.0
        for t in range(prob.ls_max + 1):
            Pt = P + lam * d
            rt = orc.zone_residual(prob, zc, Pt); evals += 1
            ft = rt @ rt
            if math.sqrt(ft) < math.sqrt(f) * (1 - 1e-4 * lam) or t == prob.ls_max:
                break
            ln = f / (ft + (2 * lam - 1) * f) * lam * lam if math.isfinite(ft) else 0.0
            lam = ln if (ln > 0 and math.isfinite(ln)) else 0.5 * lam
        P, r, f = Pt, rt, ft
        k += 1
    return P, k, evals


def test_newton_loop_matches_independent_restatement(orc):
    prob = inputs.linear_mode_problem(8, tol=1e-12)
    rng = np.random.default_rng(31)
    backtracked = 0
    for _ in range(30):
        Pstar, Pn, zc = _manufactured(orc, prob, rng, 0.5)
        Pn[0] = abs(Pn[0]); Pn[1] = abs(Pn[1])
        P1, it1, st1, ev1 = orc.zone_newton(prob, zc, Pn)
        P2, it2, ev2 = _paper_newton(orc, prob, zc, Pn.copy())
        if st1 != 0:
            continue
        assert it1 == it2 and ev1 == ev2
        assert np.abs(P1 - P2).max() < 1e-9 * (1 + np.abs(P2).max())
        backtracked += ev1 != 1 + 11 * it1
    assert backtracked > 0  # some starts needed the line search


def test_line_search_step_is_quadratic_minimiser():
    """Section 3.2: lambda_new minimises the quadratic through f(0), f'(0) = -2 f(0), f(lambda)."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        f0, lam = rng.uniform(0.1, 5), rng.uniform(0.05, 1)
        fl = f0 * rng.uniform(1.0, 3)                   # a rejected trial: the model is convex
        c = (fl - f0 + 2 * f0 * lam) / lam ** 2        # q(x) = f0 - 2 f0 x + c x^2
        xmin = f0 / c
        assert c > 0 and abs(xmin - f0 / (fl + (2 * lam - 1) * f0) * lam * lam) < 1e-12 * xmin
        assert xmin < 0.5 * lam + 1e-12                 # a rejected step at least halves lambda


def test_ideal_hydro_inversion_matches_bisection(orc):
    """With B = q = dP = 0 and closures off, one stage with no fluxes is the
    classic primitive recovery; compare with a bisection on the pressure."""
    prob = inputs.linear_mode_problem(8, conduction=False, viscosity=False, higher_order=False, tol=1e-14)
    g = prob.gamma
    rng = np.random.default_rng(41)
    for _ in range(20):
        Pstar = np.zeros(10)
        Pstar[0] = rng.uniform(0.3, 3); Pstar[1] = rng.uniform(0.3, 3); Pstar[2:5] = rng.normal(0, 0.6, 3)
        Ustar, _, _ = orc.point(prob, Pstar)
        Pn = Pstar.copy(); Pn[:5] *= 1 + 0.03 * rng.standard_normal(5)
        zc = zone_vector(orc, prob, Pn, Pn, 0.01)
        zc[0:10] = Ustar                               # U(P_n) := U*, no fluxes: root is U(P) = U*
        th, ut, ucov = minkowski_derived(Pn, g)
        P, iters, status, _ = orc.zone_newton(prob, zc, Pn)
        assert status == 0
        # textbook inversion: D = rho W, S_i = w W^2 v_i, E = w W^2 - p, w = rho + gamma u
        D, E, S = Ustar[0], -Ustar[1], Ustar[2:5]

        def resid(p):
            v = S / (E + p)
            W = 1 / math.sqrt(1 - v @ v)
            rho = D / W
            w = (E + p) / W ** 2
            return (g - 1) * (w - rho) / g - p, rho, (w - rho) / g, W * v

        lo, hi = 1e-12, 50.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if resid(mid)[0] > 0:
                lo = mid
            else:
                hi = mid
        _, rho, u, uvec = resid(0.5 * (lo + hi))
        ref = np.r_[rho, u, uvec]
        assert np.abs(P[:5] - ref).max() < 1e-12 * (1 + np.abs(ref).max())


# ---------------------------------------------------------------- reconstruction
def test_mc_reconstruction(orc):
    prob = inputs.linear_mode_problem(8)
    line = 0.3 + 0.7 * np.arange(-3, 4)
    lo, hi = orc.recon(prob, line)
    assert lo == pytest.approx(0.3 - 0.35, abs=1e-15) and hi == pytest.approx(0.3 + 0.35, abs=1e-15)
    lo, hi = orc.recon(prob, np.array([0, 0, 0, 1.0, 0.5, 0, 0]))     # extremum: flat
    assert lo == 1.0 and hi == 1.0
    lo, hi = orc.recon(prob, np.array([0, 0, 0.0, 1.0, 1.1, 0, 0]))    # MC limits to 2*0.1
    assert hi == pytest.approx(1.1) and lo == pytest.approx(0.9)
    lo, hi = orc.recon(inputs.linear_mode_problem(8, theta=1.0), np.array([0, 0, 0.0, 1.0, 1.1, 0, 0]))
    assert hi == pytest.approx(1.05)                                     # minmod


def test_weno5_reconstruction_order(orc):
    prob = inputs.linear_mode_problem(8, recon=inputs.RECON_WENO5)
    lo, hi = orc.recon(prob, 0.3 + 0.7 * np.arange(-3, 4))
    assert lo == pytest.approx(-0.05, abs=1e-14) and hi == pytest.approx(0.65, abs=1e-14)
    errs = []
    for n in (40, 80, 160):
        h = 1.0 / n
        x0 = 0.1
        # cell averages of sin(2 pi x) on cells centred at x0 + m h
        avg = lambda m: (np.cos(2 * np.pi * (x0 + (m - 0.5) * h)) - np.cos(2 * np.pi * (x0 + (m + 0.5) * h))) / (2 * np.pi * h)
        line = np.array([avg(m) for m in range(-3, 4)])
        lo, hi = orc.recon(prob, line)
        errs.append(abs(hi - np.sin(2 * np.pi * (x0 + 0.5 * h))))
    assert math.log2(errs[0] / errs[1]) > 4.5 and math.log2(errs[1] / errs[2]) > 4.5


def test_ppm_reconstruction(orc):
    """PPM: exact on linear data; flat at an extremum; the overshoot
    constraint; third order on a smooth monotone profile (the limited
    slopes cap it below the unlimited fourth order)."""
    prob = inputs.linear_mode_problem(8, recon=inputs.RECON_PPM)
    lo, hi = orc.recon(prob, 0.3 + 0.7 * np.arange(-3, 4))
    assert lo == pytest.approx(-0.05, abs=1e-14) and hi == pytest.approx(0.65, abs=1e-14)
    lo, hi = orc.recon(prob, np.array([0, 0, 0.2, 1.0, 0.5, 0, 0]))
    assert lo == 1.0 and hi == 1.0
    # a steep step next to a flat zone: the interpolant is monotone on the zone
    lo, hi = orc.recon(prob, np.array([0, 0, 0.0, 0.1, 1.0, 1.0, 1.0]))
    assert min(lo, hi) >= 0.0 - 1e-15 and max(lo, hi) <= 1.0 + 1e-15
    assert (hi - 0.1) * (0.1 - lo) >= 0
    errs = []
    for n in (40, 80, 160):
        h = 1.0 / n
        x0 = 0.1
        avg = lambda m: (np.cos(2 * np.pi * (x0 + (m - 0.5) * h)) - np.cos(2 * np.pi * (x0 + (m + 0.5) * h))) / (2 * np.pi * h)
        line = np.array([avg(m) for m in range(-3, 4)])
        lo, hi = orc.recon(prob, line)
        errs.append(abs(hi - np.sin(2 * np.pi * (x0 + 0.5 * h))))
    assert math.log2(errs[0] / errs[1]) > 2.5 and math.log2(errs[1] / errs[2]) > 2.5


# ---------------------------------------------------------------- grid invariants
def _corner_divb(P, dx):
    B1, B2 = P[5, 0], P[6, 0]
    d1 = (B1 + np.roll(B1, 1, 0) - np.roll(B1, 1, 1) - np.roll(np.roll(B1, 1, 0), 1, 1)) / (2 * dx[0])
    d2 = (B2 + np.roll(B2, 1, 1) - np.roll(B2, 1, 0) - np.roll(np.roll(B2, 1, 0), 1, 1)) / (2 * dx[1])
    return d1 + d2


def test_flux_ct_keeps_corner_divergence(orc):
    prob = inputs.turbulent_box_problem(32, tol=1e-13)
    P = inputs.turbulent_box_state(prob)
    rng = np.random.default_rng(9)
    P[5:7] += 1e-2 * rng.standard_normal(P[5:7].shape)    # start with a non-zero corner divergence
    d0 = _corner_divb(P, prob.dx)
    dt = 0.5 / 32
    for _ in range(3):
        P, it, st, _ = orc.step(prob, P, dt)
        assert (st == 0).all()
    d1 = _corner_divb(P, prob.dx)
    assert np.abs(d0).max() > 1e-2
    assert np.abs(d1 - d0).max() < 1e-12 * np.abs(P[5:7]).max() / prob.dx[0]


def test_periodic_box_conserves_mass_and_energy_momentum(orc):
    prob = inputs.turbulent_box_problem(24, tol=1e-14)
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / 24

    def totals(P):
        tot = np.zeros(5); mag = np.zeros(5)
        for z in range(prob.zones):
            U, _, _ = orc.point(prob, P.reshape(10, -1)[:, z])
            tot += U[:5]; mag += np.abs(U[:5])
        return tot, mag

    t0, m0 = totals(P)
    P1, it, st, _ = orc.step(prob, P, dt)
    assert (st == 0).all()
    t1, _ = totals(P1)
    assert np.all(np.abs(t1 - t0) <= 1e-12 * m0)


def test_flop_count_file_matches_oracle():
    """tests/golden/flop_counts.txt is what make_flop_counts.py writes now."""
    from tests.golden import make_flop_counts
    stored = {}
    for line in open(make_flop_counts.OUT):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            stored[k] = int(v)
    assert stored == make_flop_counts.counts()


# ---------------------------------------------------------------- HLLE (Section 2.4.2)
def _zigzag_line(n, base, amp):
    """States of n zones along X1 alternating base + amp, base - amp: every
    zone is a local extremum of every field, so the limited reconstruction
    is flat and the face states are the neighbouring zone values."""
    P = np.zeros((10, 1, 1, n))
    sgn = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    for v in range(10):
        P[v, 0, 0] = base[v] + amp[v] * sgn
    return P


def test_hlle_equals_llf_when_the_bounds_are_symmetric(orc):
    """With no flow along either direction the grid-frame speeds of each face
    state are +-c, so the HLLE bounds are c_R = c_L = max c, the LLF speed; the
    HLLE flux (c_R F^- + c_L F^+ - c_R c_L (U^+ - U^-))/(c_R + c_L) then is the
    LLF flux (F^- + F^+)/2 - c (U^+ - U^-)/2.  Random rest-frame states
    (u^1 = u^2 = 0, everything else varying, both closures on) on a ragged
    2-D grid, flux-CT included."""
    rng = np.random.default_rng(31)
    prob = inputs.linear_mode_problem(8).with_(n=(9, 6, 1))
    P = np.zeros((10, 1, 6, 9))
    P[0] = rng.uniform(0.5, 2.0, P[0].shape)
    P[1] = rng.uniform(0.2, 3.0, P[1].shape)
    P[4] = rng.normal(0.0, 0.4, P[4].shape)
    P[5:8] = rng.normal(0.0, 0.3, P[5:8].shape)
    P[8:10] = rng.normal(0.0, 0.1, P[8:10].shape)
    F_llf = orc.fluxes(prob, P)
    F_hlle = orc.fluxes(prob.with_(riemann=inputs.FLUX_HLLE), P)
    scale = np.abs(F_llf).max(axis=(2, 3, 4), keepdims=True) + 1e-300
    assert (np.abs(F_hlle - F_llf) / scale).max() < 1e-14
    # the pin has teeth: a dissipation term of the wrong sign would differ
    assert np.abs(F_llf[0, 0]).max() > 1e-3


@pytest.mark.parametrize("direction", [+1, -1])
def test_hlle_is_the_upwind_flux_of_a_supersonic_face(orc, direction):
    """When every wave at a face moves the same way (all c^+- > 0), c_L = 0
    and HLLE returns the flux of the upwind state, F(P^-) (left state); for
    flow to -X1 it returns F(P^+).  Zig-zag data make the face states the
    zone values themselves, so the expected flux is the pointwise flux of
    the upwind zone.  Cold, fast flow (|u~^1| = 3, v ~ 0.95) with the
    closures on keeps every speed of one sign (checked)."""
    n = 8
    base = np.array([1.0, 0.01, 3.0 * direction, 0.2, -0.1, 0.05, 0.02, -0.03, 0.01, -0.02])
    amp = np.array([0.1, 0.002, 0.1, 0.05, 0.03, 0.0, 0.01, 0.01, 0.005, 0.004])
    prob = inputs.Problem(dim=1, n=(n, 1, 1), riemann=inputs.FLUX_HLLE)
    P = _zigzag_line(n, base, amp)
    F = orc.fluxes(prob, P)[0]                  # [10, 1, 1, n], low face of each zone
    Pz = P.reshape(10, n)
    for i in range(n):
        up = Pz[:, (i - 1) % n] if direction > 0 else Pz[:, i]
        dn = Pz[:, i] if direction > 0 else Pz[:, (i - 1) % n]
        _, Fup, cup = orc.point(prob, up)
        _, Fdn, cdn = orc.point(prob, dn)
        c = np.r_[cup[0], cdn[0]]
        assert (c > 0).all() if direction > 0 else (c < 0).all()
        want = Fup[0].copy()
        want[5] = 0.0                           # F^1[B^1] = 0 (flux-CT)
        got = F[:, 0, 0, i]
        assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max(), (i, got - want)
        # and not the downstream state's flux: the face states differ
        assert np.abs(Fdn[0][:5] - Fup[0][:5]).max() > 1e-3
