"""The EMHD shock (Section 8.1.3): the steady structure joining the two
states of Table 2 (tau_R = 0.1, psi = 3, gamma = 4/3), obtained from the
model's steady equations in tests/emhd_shock.py, checked against the printed
right state, then used as the initial condition of the scheme: the oracle's
steady residual of the structure and its drift from it after t = 1 fall with
resolution (the paper's check of the IVP against the BVP solution), and the
CUDA path follows the oracle and converges the same way at up to 4096
zones."""
import math

import numpy as np
import pytest

from tests import emhd_shock as es


def test_structure_reaches_the_printed_right_state():
    """Integrated from the upstream state, the structure ends on the printed
    downstream state of Table 2 to all its eight decimals, with q~ = dP~ = 0."""
    _, Y, _, _ = es.structure()
    end = Y[:, -1]
    assert np.all(np.round(end[:3], 8) == es.RIGHT_PRINTED[:3]), end
    assert abs(end[4]) < 1e-12


def test_structure_keeps_the_fluxes():
    m = es.model(conduction=False)
    _, Y, _, _ = es.structure()
    ref = m.fluxes(es.LEFT)
    drift = max(np.abs(m.fluxes(Y[:, i]) - ref).max() for i in range(0, Y.shape[1], 499))
    assert drift < 1e-11


def test_structure_is_a_compressive_viscous_profile():
    """rho rises and u^1 falls monotonically; dP~ < 0 inside (compression along
    b-hat makes the parallel pressure the larger); the profile is within 1e-9
    of the upstream state 0.4 before its midpoint and within 1e-11 of the
    downstream state 3 after it."""
    x = np.linspace(-0.4, 3.0, 3401)
    Y = es.profile(x)
    assert np.all(np.diff(Y[0]) >= -1e-13) and np.all(np.diff(Y[2]) <= 1e-13)
    assert np.all(Y[4] <= 1e-13) and Y[4].min() < -0.5
    assert np.abs(Y[:, 0] - es.LEFT).max() < 1e-9
    _, Yt, _, _ = es.structure()
    assert np.abs(Y[:, -1] - Yt[:, -1]).max() < 1e-11


def test_fixed_points_and_the_heat_flux_mode():
    """Conduction off: the upstream state has one unstable direction and the
    downstream state one stable direction, so the structure leaving upstream
    is unique up to a shift.  With phi = 5 the heat-flux mode (speed
    ((gamma - 1) phi)^(1/2) c_s of Eq. modcs) is slower than the upstream flow
    and the upstream state turns into a saddle: the reading that takes the
    structure with conduction off."""
    up = es.fixed_point_rates(es.LEFT, conduction=False)
    _, Y, _, _ = es.structure()
    down = es.fixed_point_rates(Y[:, -1], conduction=False)
    assert up.size == 1 and up[0] > 0 and down.size == 1 and down[0] < 0
    upc = es.fixed_point_rates(es.LEFT, conduction=True)
    assert upc.size == 2 and upc[0] < 0 < upc[1]
    g = es.GAMMA
    cs2 = g * (g - 1) / (1 + g)                      # rho = u = 1
    vq = math.sqrt((g - 1) * es.PHI * cs2)
    v1 = 1 / math.sqrt(2)                            # u^1 = 1
    assert vq < v1 < math.sqrt(es.PSI * cs2)


def test_oracle_steady_residual_of_the_structure_falls(orc):
    """The oracle's residual of the structure with no time change (P = P_n =
    P^E: flux divergence minus sources, with the slope-limited targets of the
    relaxation terms) is its truncation error: the L1 norm of every row falls
    by 8x or more from 256 to 1024 zones.  A dropped or misplaced dissipative
    term (Pi's sign, the 3 rho nu factor, the higher-order term) leaves it
    order one."""
    norms = {}
    for n in (256, 1024):
        prob = es.shock_structure_problem(n)
        P, _ = es.structure_state(prob)
        R = orc.residual(prob, P, P, 0.25 * prob.dx[0], P, scaled=False).reshape(10, -1)
        norms[n] = np.abs(R).sum(axis=1) * prob.dx[0]
        assert np.abs(R[3:9]).max() == 0.0
    for a in (0, 1, 2, 9):
        assert norms[256][a] > 8 * norms[1024][a], (a, norms[256][a], norms[1024][a])
    assert norms[1024][[0, 1, 2, 9]].max() < 3e-3


def _drift(P, P0, dx):
    return np.abs(P - P0).reshape(10, -1)[[0, 1, 2, 9]].sum(axis=1) * dx


def test_oracle_stays_on_the_structure(orc):
    """Started on the structure, the scheme stays on it: after t = 1 (ten
    relaxation times) the L1 drift falls by 2.8x or more (order 1.5) per
    doubling from 128 to 512 zones, to below 3e-4 in rho."""
    d = []
    for n in (128, 256, 512):
        prob = es.shock_structure_problem(n)
        P0, _ = es.structure_state(prob)
        P = P0.copy()
        dt = 0.25 * prob.dx[0]
        for _ in range(int(round(1.0 / dt))):
            P, _, st, _ = orc.step(prob, P, dt)
            assert st.max() == 0
        d.append(_drift(P, P0, prob.dx[0]))
    assert np.all(d[0] > 2.8 * d[1]) and np.all(d[1] > 2.8 * d[2]), d
    assert d[2][0] < 3e-4


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_structure_parity_and_convergence(orc, precision):
    """The CUDA path from the structure: at 512 zones within 1e-9 of the
    oracle (float64 solver at tol 1e-14 after 20 steps, mixed solver at
    tol 1e-10 after one); from 1024 to 4096 zones, where the steep upstream
    foot (e-folding length 0.0055) is resolved, its L1 drift after t = 1
    falls by 3x or more per doubling."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_01106_b300.grim import Grim
    from tests.gpu_helpers import rel_field_err
    dev = torch.device("cuda:0")
    tol = 1e-12 if precision == 0 else 1e-10

    prob = es.shock_structure_problem(512, tol=1e-14 if precision == 0 else tol)
    P0, _ = es.structure_state(prob)
    dt = 0.25 * prob.dx[0]
    g = Grim(prob, precision=precision)
    a = torch.from_numpy(P0).to(dev)
    ref = P0.copy()
    for _ in range(20 if precision == 0 else 1):
        g.step(a, a, dt)
        ref, _, st, _ = orc.step(prob.with_(tol=1e-14), ref, dt)
        assert st.max() == 0
    assert g.stats()["failed"] == 0
    assert rel_field_err(a.cpu().numpy(), ref).max() < 1e-9
    g.close()

    d = []
    for n in (1024, 2048, 4096):
        prob = es.shock_structure_problem(n, tol=tol)
        P0, _ = es.structure_state(prob)
        dt = 0.25 * prob.dx[0]
        g = Grim(prob, precision=precision)
        a = torch.from_numpy(P0).to(dev)
        for _ in range(int(round(1.0 / dt))):
            g.step(a, a, dt)
        assert g.stats()["failed"] == 0
        d.append(_drift(a.cpu().numpy(), P0, prob.dx[0]))
        g.close()
    for k in range(2):
        assert np.all(d[k] > 3 * d[k + 1]), (k, d)
