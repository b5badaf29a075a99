"""Table 2 (Section 8.1.2): the steady ideal-MHD shock stays in place.  A 1-D
run from the two printed states keeps the captured shock within half a zone
of x = 0 over three crossing times of the domain, leaves the supersonic
upstream state untouched, and holds the downstream plateau near the printed
density (the subsonic downstream flow leaves through a copy boundary, which
lets its state drift by a few per cent); the oracle at 64 zones, the CUDA
path at 256."""
import numpy as np
import pytest

from tests.shock_setup import shock_position, shock_problem, shock_state, shock_states


def _check(P, x, dx):
    L, R = shock_states()
    rho = P[0, 0, 0]
    xs = shock_position(rho, x, L, R)
    assert abs(xs) < 0.5 * dx, xs / dx
    up = P[:, 0, 0, x < -4 * dx]
    assert np.abs(up - L[:, None]).max() < 1e-12
    down = rho[x > 4 * dx]
    assert np.abs(down / R[0] - 1).max() < 0.05


def test_shock_steady_oracle(orc):
    n = 64
    prob = shock_problem(n)
    P, x = shock_state(prob)
    dt = 0.25 * prob.dx[0]
    for _ in range(400):
        P, _, st, _ = orc.step(prob, P, dt)
        assert st.max() == 0
    _check(P, x, prob.dx[0])


@pytest.mark.gpu
def test_shock_steady_gpu(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_01106_b300.grim import Grim
    dev = torch.device("cuda:0")
    n = 256
    prob = shock_problem(n)
    P, x = shock_state(prob)
    dt = 0.25 * prob.dx[0]
    g = Grim(prob)
    a = torch.from_numpy(P).to(dev)
    for _ in range(1600):
        g.step(a, a, dt)
    s = g.stats()
    assert s["failed"] == 0
    _check(a.cpu().numpy(), x, prob.dx[0])
    # the first 100 steps agree with the oracle
    n2 = 64
    prob2 = shock_problem(n2, tol=1e-14)
    P2, _ = shock_state(prob2)
    g2 = Grim(prob2)
    b = torch.from_numpy(P2).to(dev)
    ref = P2
    for _ in range(20):
        g2.step(b, b, 0.25 * prob2.dx[0])
        ref, _, _, _ = orc.step(prob2, ref, 0.25 * prob2.dx[0])
    from tests.gpu_helpers import rel_field_err
    assert rel_field_err(b.cpu().numpy(), ref).max() < 1e-11
    g.close()
    g2.close()


def test_ideal_rows_vanish_for_any_fluid_state(orc):
    """The premise of the ideal-MHD 5x5 Newton block: with conduction and
    viscosity off and q~ = dP~ = 0 everywhere, the q~ and dP~ rows of the
    stage residual are exactly zero whatever rho, u and u^i are, so their
    Newton update is zero."""
    prob = shock_problem(32)
    Pn, _ = shock_state(prob)
    rng = np.random.default_rng(5)
    PE = Pn * (1 + 1e-2 * rng.standard_normal(Pn.shape))
    PE[5:] = Pn[5:]
    for _ in range(3):
        Pk = Pn * (1 + 1e-1 * rng.standard_normal(Pn.shape))
        Pk[5:] = Pn[5:]
        R = orc.residual(prob, Pn, PE, 0.01, Pk).reshape(10, -1)
        assert np.all(R[8:] == 0.0) and np.abs(R[:5]).max() > 0
