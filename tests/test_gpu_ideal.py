"""Ideal MHD (conduction and viscosity off): zones whose q~, dP~ and their
residual rows are zero solve the 5x5 block of rho, u, u^i (Section 8.2's
ideal-MHD solve) instead of the 7x7 EMHD block, with the same root as the
oracle's 10x10 solve.  The mixed solver's float32 Jacobian costs 2 n + 1
residual evaluations an update with centred differences over n columns, so
its counters show which block each update took: 11 for 5x5, 15 for 7x7."""
import numpy as np
import pytest

from tests.shock_setup import shock_problem, shock_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _run(prob, P, precision, dt, steps, dev):
    from paper_1702_01106_b300.grim import Grim
    g = Grim(prob, precision=precision)
    a = torch.from_numpy(P).to(dev)
    for _ in range(steps):
        g.step(a, a, dt)
    s = g.stats()
    g.close()
    return a.cpu().numpy(), s


@pytest.mark.parametrize("precision", [0, 1])
def test_ideal_mhd_takes_the_5x5_block(dev, orc, precision):
    from tests.gpu_helpers import rel_field_err
    prob = shock_problem(256, tol=1e-14 if precision == 0 else 1e-10)
    P, _ = shock_state(prob)
    dt = 0.25 * prob.dx[0]
    got, s = _run(prob, P, precision, dt, 1, dev)
    ref, _, st, _ = orc.step(prob.with_(tol=1e-14), P, dt)
    assert st.max() == 0 and s["failed"] == 0
    assert rel_field_err(got, ref).max() < (1e-12 if precision == 0 else 1e-9)
    if precision == 1:
        assert s["lu32"] > 0 and s["evals32"] == 11 * s["lu32"]
    else:
        # 5 FD columns and one or two line-search trials an update (7 columns
        # would make it at least 8)
        assert s["lu64"] > 0 and 6 * s["lu64"] <= s["evals64"] - s["zones"] < 8 * s["lu64"]


def test_ideal_mode_keeps_the_7x7_block_where_q_is_nonzero(dev, orc):
    """The same shock with q~ and dP~ nonzero in its first 32 zones (they relax
    to zero): those zones and their neighbours (whose explicit q~ and dP~
    fluxes are not zero) take the 7x7 block, the rest the 5x5 one, and the
    step matches the oracle's."""
    from tests.gpu_helpers import rel_field_err
    prob = shock_problem(256, tol=1e-14)
    P, _ = shock_state(prob)
    P = P.copy()
    P[8, ..., :32] = 1e-3
    P[9, ..., :32] = -2e-3
    dt = 0.25 * prob.dx[0]
    got, s = _run(prob, P, 0, dt, 1, dev)
    ref, _, st, _ = orc.step(prob, P, dt)
    assert st.max() == 0 and s["failed"] == 0
    assert rel_field_err(got, ref).max() < 1e-12
    _, s32 = _run(prob.with_(tol=1e-10), P, 1, dt, 1, dev)
    assert 11 * s32["lu32"] < s32["evals32"] < 15 * s32["lu32"]


def test_emhd_keeps_the_7x7_block(dev):
    from paper_1702_01106_b300 import inputs
    prob = inputs.turbulent_box_problem(32, tol=1e-10)
    P = inputs.turbulent_box_state(prob)
    _, s = _run(prob, P, 1, 0.5 / 32, 1, dev)
    assert s["lu32"] > 0 and s["evals32"] == 15 * s["lu32"]
