"""Steps and stages written over their own P_n.

grim_step allows P_out == P_in and grim_stage P_out == P_n.  The start of a
stage is written into P_out before the Newton solves, yet two parts of the
stage read P_n after that: the learned start's fallback (a zone whose
learned start has a larger residual than P_n restarts from P_n) and, in the
general-metric path, the revert of a zone whose solve failed (back to P_n
before the floors).  So an in-place step must give exactly the result of the
same step into a separate buffer, in both of those cases.
"""
import numpy as np
import pytest

from paper_1702_01106_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _t(P, dev):
    return torch.from_numpy(np.ascontiguousarray(P)).to(dev)


def _same_in_place(g, P, dt, dev, steps):
    a = _t(P, dev)
    b = torch.empty_like(a)
    c = a.clone()
    for _ in range(steps):
        g.step(a, b, dt)
        a, b = b, a
        g.step(c, c, dt)
    torch.cuda.synchronize()
    return torch.equal(a, c)


@pytest.mark.parametrize("graphs", [False, True])
def test_kerr_torus_in_place_with_failed_zones(dev, graphs):
    """The 16 x 12 x 6 torus at tol 1e-14: surface zones stall below their
    round-off floor every stage, fail, and are reverted to P_n and floored."""
    from paper_1702_01106_b300.grim import Grim
    prob = inputs.torus_problem(16, 12, 6, tol=1e-14)
    P = inputs.torus_state(prob)
    dt = inputs.torus_dt(prob)
    g = Grim(prob)
    g.use_graphs(graphs)
    g.reset_stats()
    assert _same_in_place(g, P, dt, dev, 3)
    assert g.stats()["failed"] > 0
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_learned_start_in_place_with_fallbacks(dev, precision):
    """An untrained network's start loses to P_n in most zones: those zones
    restart from P_n, which an in-place step must still have."""
    from paper_1702_01106_b300.grim import MLP, Grim
    prob = inputs.turbulent_box_problem(32, tol=1e-12).with_(n=(48, 40, 1))
    P = inputs.turbulent_box_state(prob)
    m = MLP(seed=3)
    g = Grim(prob, precision=precision)
    g.set_guess(m, accept=1e-9)
    g.reset_stats()
    assert _same_in_place(g, P, 0.25 / 32, dev, 2)
    s = g.stats()
    assert s["fallbacks"] > 0.1 * s["zones"]
    g.close()
    m.close()


def test_stage_in_place(dev):
    """grim_stage with P_out == P_n (the torus at tol 1e-14, failed zones
    reverted to P_n) equals the same stage into a separate buffer."""
    from paper_1702_01106_b300.grim import Grim
    prob = inputs.torus_problem(16, 12, 6, tol=1e-14)
    P = inputs.torus_state(prob)
    dt = inputs.torus_dt(prob)
    g = Grim(prob)
    a = _t(P, dev)
    h = torch.empty_like(a)
    g.stage(a, a, 0.5 * dt, h)
    out = torch.empty_like(a)
    st = torch.zeros(prob.zones, dtype=torch.uint8, device=dev)
    g.stage(a, h, dt, out, status=st)
    assert (st != 0).any()
    g.stage(a, h, dt, a)
    torch.cuda.synchronize()
    assert torch.equal(a, out)
    g.close()
