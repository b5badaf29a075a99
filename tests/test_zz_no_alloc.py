"""grim_step_static: the step for callers that cannot allocate device memory.

Callers that own all device memory through their own pool, or that must not
call cudaMalloc after start-up, use grim_step_static, whose scratch is a
static device array.  Its results must equal grim_step's, call after call,
and the oracle's; it must also work in place and allocate nothing.  This
file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_1702_01106_b300 import inputs
from tests.gpu_helpers import rel_field_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("precision", [0, 1])
def test_static_step_matches_context_step_twice(dev, precision):
    from paper_1702_01106_b300.grim import Grim, step_static
    prob = inputs.turbulent_box_problem(32, tol=1e-14).with_(n=(72, 40, 1))
    P = torch.from_numpy(inputs.turbulent_box_state(prob)).to(dev)
    dt = 0.5 / 72
    g = Grim(prob, precision=precision)
    ref1 = torch.empty_like(P)
    ref2 = torch.empty_like(P)
    g.step(P, ref1, dt)
    g.step(ref1, ref2, dt)
    out1 = torch.empty_like(P)
    out2 = torch.empty_like(P)
    assert step_static(prob, P, out1, dt, precision) == 0
    assert step_static(prob, out1, out2, dt, precision) == 0
    torch.cuda.synchronize()
    assert rel_field_err(out1.cpu().numpy(), ref1.cpu().numpy()).max() < 1e-12
    assert rel_field_err(out2.cpu().numpy(), ref2.cpu().numpy()).max() < 1e-12
    g.close()


def test_static_step_rejects_grids_beyond_its_limit(dev):
    from paper_1702_01106_b300.grim import STATIC_MAX_ZONES, step_static
    prob = inputs.turbulent_box_problem(32).with_(n=(STATIC_MAX_ZONES + 1, 1, 1))
    P = torch.zeros((10, 1, 1, 1), dtype=torch.float64, device=dev)
    assert step_static(prob, P, P, 0.01) == -4   # GRIM_ESIZE, nothing launched


@pytest.mark.parametrize("precision,recon", [(0, inputs.RECON_MC), (0, inputs.RECON_WENO5), (1, inputs.RECON_MC)])
def test_static_step_matches_the_oracle(dev, orc, precision, recon):
    """The fused tile kernel that only this entry point runs, against the
    oracle directly: float64 at tol 1e-14 within 1e-12, the mixed solver at
    tol 1e-12 within 1e-9 (ragged 72 x 40 grid, several 16 x 16 tiles)."""
    from paper_1702_01106_b300.grim import step_static, step_static_stats
    tol = 1e-14 if precision == 0 else 1e-12
    prob = inputs.turbulent_box_problem(32, tol=tol, recon=recon).with_(n=(72, 40, 1))
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / 72
    out = torch.empty((10, 1, 40, 72), dtype=torch.float64, device=dev)
    assert step_static(prob, torch.from_numpy(P).to(dev), out, dt, precision) == 0
    s = step_static_stats()
    ref, _, st, _ = orc.step(prob.with_(tol=1e-14), P, dt)
    assert st.max() == 0 and s["failed"] == 0 and s["zones"] == 2 * prob.zones
    assert rel_field_err(out.cpu().numpy(), ref).max() < (1e-12 if precision == 0 else 1e-9)


def test_static_step_in_place(dev, orc):
    """P_out == P_in: the result equals the out-of-place step's and the
    oracle's."""
    from paper_1702_01106_b300.grim import step_static
    prob = inputs.turbulent_box_problem(32, tol=1e-14).with_(n=(40, 36, 1))
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / 40
    a = torch.from_numpy(P).to(dev)
    b = torch.empty_like(a)
    assert step_static(prob, a, b, dt) == 0
    assert step_static(prob, a, a, dt) == 0
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    ref, _, _, _ = orc.step(prob, P, dt)
    assert rel_field_err(a.cpu().numpy(), ref).max() < 1e-12


def test_static_step_allocates_nothing(dev):
    """After the first call (which looks up the static array's address),
    further calls leave the device's free memory unchanged."""
    from paper_1702_01106_b300.grim import step_static
    prob = inputs.turbulent_box_problem(32, tol=1e-12).with_(n=(64, 48, 1))
    a = torch.from_numpy(inputs.turbulent_box_state(prob)).to(dev)
    b = torch.empty_like(a)
    assert step_static(prob, a, b, 0.5 / 64) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert step_static(prob, b, a, 0.5 / 64) == 0
        assert step_static(prob, a, b, 0.5 / 64) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
