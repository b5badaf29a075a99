"""Pins of the oracle's modified Kerr-Schild geometry (Section 2.1) and the
torus floors against closed forms of the Kerr metric and geodesic motion."""
import math

import numpy as np
import pytest

from paper_1702_01106_b300 import inputs


def _prob(a=0.9375, h=0.3):
    return inputs.torus_problem(8, 8, 1, spin=a, h=h)


def _theta(prob, X2):
    return math.pi * X2 + 0.5 * (1 - prob.h_mks) * math.sin(2 * math.pi * X2)


def _dtheta(prob, X2):
    return math.pi * (1 + (1 - prob.h_mks) * math.cos(2 * math.pi * X2))


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9375])
def test_sqrt_minus_g_closed_form(orc, a):
    """sqrt(-g) = Sigma sin(theta) (Kerr-Schild) times r dtheta/dX^2 (MKS)."""
    prob = _prob(a)
    for X1 in (math.log(1.5), math.log(6.0), math.log(30.0)):
        for X2 in (0.1, 0.37, 0.5, 0.8):
            geo = orc.geometry(prob, [X1, X2, 0.3])
            r, th = math.exp(X1), _theta(prob, X2)
            sig = r * r + a * a * math.cos(th) ** 2
            want = sig * math.sin(th) * r * _dtheta(prob, X2)
            assert abs(geo["sqrtg"] - want) <= 1e-12 * want
            assert np.allclose(geo["gcov"] @ geo["gcon"], np.eye(4), atol=1e-12)


def test_schwarzschild_components(orc):
    """a = 0: g_tt = -(1 - 2/r), g_11 = (1 + 2/r) r^2, g_t1 = 2, lapse (1 + 2/r)^(-1/2)."""
    prob = _prob(0.0)
    for r in (2.5, 7.0, 20.0):
        geo = orc.geometry(prob, [math.log(r), 0.4, 0.0])
        g = geo["gcov"]
        assert abs(g[0, 0] + (1 - 2 / r)) < 1e-14
        assert abs(g[1, 1] - (1 + 2 / r) * r * r) < 1e-12 * r * r
        assert abs(g[0, 1] - 2.0) < 1e-14
        assert abs(geo["alpha"] - 1 / math.sqrt(1 + 2 / r)) < 1e-14


def test_horizon_where_g11_vanishes(orc):
    """g^{rr} = Delta/Sigma vanishes on the outer horizon r_+ = 1 + (1 - a^2)^(1/2)."""
    a = 0.9375
    prob = _prob(a)
    rp = 1 + math.sqrt(1 - a * a)
    geo = orc.geometry(prob, [math.log(rp), 0.3, 0.0])
    assert abs(geo["gcon"][1, 1]) < 1e-12
    geo = orc.geometry(prob, [math.log(1.2 * rp), 0.3, 0.0])
    assert geo["gcon"][1, 1] > 0


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9375])
def test_circular_orbits_are_geodesics(orc, a):
    """Prograde circular equatorial orbits have Omega = 1/(r^{3/2} + a)
    (Bardeen, Press & Teukolsky 1972): the radial geodesic equation
    Gamma^1_tt + 2 Gamma^1_tphi Omega + Gamma^1_phiphi Omega^2 = 0 holds."""
    prob = _prob(a)
    for r in (4.0, 6.0, 12.0, 30.0):
        geo = orc.geometry(prob, [math.log(r), 0.5, 0.0])
        G = geo["Gam"]
        om = 1.0 / (r ** 1.5 + a)
        res = G[1, 0, 0] + 2 * G[1, 0, 3] * om + G[1, 3, 3] * om * om
        assert abs(res) < 1e-13 * max(abs(G[1, 0, 0]), 1e-300)


def test_connection_against_finite_differences(orc):
    """Gamma from dual numbers vs 4th-order centred differences of g (h = 1e-4)."""
    prob = _prob()
    X = np.array([math.log(5.0), 0.31, 0.0])
    geo = orc.geometry(prob, X)
    h = 1e-4
    dg = np.zeros((4, 4, 4))
    for d in (1, 2):
        e = np.zeros(3); e[d - 1] = h
        f = [orc.geometry(prob, X + s * e)["gcov"] for s in (-2, -1, 1, 2)]
        dg[d] = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
    gi = geo["gcon"]
    G = 0.5 * (np.einsum("lk,mkn->lmn", gi, dg) + np.einsum("lk,nkm->lmn", gi, dg)
               - np.einsum("lk,kmn->lmn", gi, dg))
    assert np.abs(G - geo["Gam"]).max() < 1e-8 * np.abs(G).max()


def test_minkowski_tau_and_kerr_tau(orc):
    prob = _prob()
    r = 9.0
    geo = orc.geometry(prob, [math.log(r), 0.5, 0.0])
    assert abs(geo["tauR"] - r ** 1.5) < 1e-12 * r ** 1.5
    flat = inputs.linear_mode_problem(8).with_(tau_R=2.5)
    assert orc.geometry(flat, [0.1, 0.2, 0.3])["tauR"] == 2.5


def test_floors(orc):
    """rho and u are raised to 1e-5 r^{-3/2}, 1e-7 r^{-5/2}; dP is clamped to
    [-b^2, b^2/2] (checked by re-evaluating it after the clamp)."""
    prob = _prob()
    r = 4.0
    X = [math.log(r), 0.5, 0.0]
    P = np.array([1e-9, 1e-12, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    out = orc.floors(prob, X, P)
    assert out[0] == pytest.approx(1e-5 * r ** -1.5, rel=1e-15)
    assert out[1] == pytest.approx(1e-7 * r ** -2.5, rel=1e-15)
    P = np.array([1.0, 0.5, 0.01, 0.0, 0.02, 0.05, 0.01, 0.0, 0.0, 50.0])
    out = orc.floors(prob, X, P)
    assert out[9] < 50.0 and out[:9].tolist() == P[:9].tolist()
    P[9] = -50.0
    out2 = orc.floors(prob, X, P)
    assert out2[9] > -50.0
    # ratio of the clamped values is the ratio of the thresholds: (b^2/2)/(-b^2)
    assert out[9] / out2[9] == pytest.approx(-0.5, rel=1e-12)
    P[9] = 1e-6
    assert orc.floors(prob, X, P)[9] == 1e-6      # inside the band: unchanged


def test_polar_faces_carry_no_flux(orc):
    """Faces on the axis (theta = 0, pi) have sqrt(-g) = 0: the oracle's X2
    fluxes there vanish for every field."""
    prob = inputs.torus_problem(12, 10, 1)
    P = inputs.torus_state(prob)
    F = orc.fluxes(prob, P)              # [dim, 10, n3, n2, n1], low face of each zone
    assert np.abs(F[1, :, :, 0, :]).max() == 0.0
