"""Batched boxes of different sizes: a batched step (eager, then replayed
from a graph) equals grim_step on each box, and the counters add up."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_step_equals_per_box_steps(dev, precision):
    from paper_1702_01106_b300.grim import Batch, Grim
    boxes = inputs.batched_boxes(count=7, sides=(16, 32, 48, 64))
    probs = [b[0] for b in boxes]
    dts = [b[2] for b in boxes]
    steps = 4
    ref, zones, iters = [], 0, 0
    for prob, P, dt in boxes:
        g = Grim(prob, precision=precision)
        a = torch.from_numpy(P).to(dev)
        for _ in range(steps):
            g.step(a, a, dt)
        s = g.stats()
        zones += s["zones"]
        iters += s["iters"]
        ref.append(a.cpu().numpy())
        g.close()
    bt = Batch(probs, precision=precision)
    A = [torch.from_numpy(b[1]).to(dev) for b in boxes]
    B = [torch.empty_like(a) for a in A]
    for _ in range(steps):           # ping-pong: eager, capture a->b, capture b->a, replay
        bt.step(A, B, dts)
        A, B = B, A
    s = bt.stats()
    for i in range(len(boxes)):
        assert np.array_equal(A[i].cpu().numpy(), ref[i]), i
    assert s["zones"] == zones and s["iters"] == iters and s["failed"] == 0
    assert s["launches"] > 0
    bt.close()


def test_batched_step_learned_guess_and_without_graphs(dev):
    """Graphs off gives the same result; a learned guess set on every box
    keeps the boxes converged."""
    from paper_1702_01106_b300.grim import Batch, MLP, GRIM_MIXED
    boxes = inputs.batched_boxes(count=3, sides=(16, 32))
    probs = [b[0] for b in boxes]
    dts = [b[2] for b in boxes]
    outs = []
    for graphs in (True, False):
        bt = Batch(probs, precision=GRIM_MIXED)
        bt.use_graphs(graphs)
        A = [torch.from_numpy(b[1]).to(dev) for b in boxes]
        for _ in range(3):
            bt.step(A, A, dts)
        outs.append([a.cpu().numpy() for a in A])
        bt.close()
    for x, y in zip(*outs):
        assert np.array_equal(x, y)
    m = MLP(seed=3)
    bt = Batch(probs, precision=GRIM_MIXED)
    bt.set_guess(m, accept=1e-3)
    A = [torch.from_numpy(b[1]).to(dev) for b in boxes]
    for _ in range(2):
        bt.step(A, A, dts)
    s = bt.stats()
    assert s["failed"] == 0 and s["max_res"] <= probs[0].tol
    bt.close()
    m.close()
