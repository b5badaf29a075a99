"""grim_step_static: the step for callers that cannot allocate device memory.

Callers that own all device memory through their own pool, or that must not
call cudaMalloc after start-up, use grim_step_static, whose scratch is a
static device array.  Its results must equal grim_step's, call after call.
This file is collected last so that a run stopping at the first failure has
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
