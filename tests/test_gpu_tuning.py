"""Launch shapes, zone compaction, CUDA graphs and the autotuner: none of
them may change a result bit, and the counters must add up."""
import json
import os

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


def _run(prob, P, dt, dev, precision, steps=2, graphs=False, **tune):
    from paper_1702_01106_b300.grim import Grim
    g = Grim(prob, precision=precision)
    if tune:
        g.set_tuning(**tune)
    g.use_graphs(graphs)
    a = torch.from_numpy(P).to(dev)
    b = torch.empty_like(a)
    for _ in range(steps):
        g.step(a, b, dt)
        a, b = b, a
    s = g.stats()
    out = a.cpu().numpy()
    g.close()
    return out, s


@pytest.mark.parametrize("precision", [0, 1])
def test_compaction_and_block_shapes_agree(dev, precision):
    """Every Newton block size and cut, with and without the compaction
    rounds, and every explicit block size, reaches the same root: solved to
    the round-off tolerance the states agree to 1e-12 (field-scaled;
    separately compiled kernels may contract multiply-adds differently, so
    bits can differ), every zone is solved once and none fails; the mean
    update count is unchanged."""
    from tests.gpu_helpers import rel_field_err
    prob = inputs.turbulent_box_problem(96).with_(n=(96, 80, 1), tol=1e-14)
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / 96
    ref, sref = _run(prob, P, dt, dev, precision, newton_kcut=prob.k_max + 1, newton_rounds=0)
    assert sref["failed"] == 0
    for rounds in (0, 1):
        for bs in (32, 64, 128):
            for kcut, fbs, zbs in ((1, 256, 64), (2, 64, 256), (3, 128, 128), (prob.k_max, 128, 128)):
                out, s = _run(prob, P, dt, dev, precision, newton_bs=bs, newton_kcut=kcut, faces_bs=fbs,
                              zone_bs=zbs, newton_rounds=rounds)
                err = rel_field_err(out.reshape(10, -1), ref.reshape(10, -1)).max()
                assert err < 1e-12, (rounds, bs, kcut, err)
                assert s["zones"] == sref["zones"] and s["failed"] == 0, (rounds, bs, kcut)
                assert abs(s["iters"] - sref["iters"]) <= 0.01 * sref["iters"], (rounds, bs, kcut)
                assert s["max_res"] <= prob.tol


@pytest.mark.parametrize("precision", [0, 1])
def test_compaction_rounds_on_the_torus(dev, precision):
    """The general-metric kernels with the compaction rounds against the
    one-pass kernel on the 16 x 12 x 6 Kerr torus (floors on, tol 1e-12):
    the same zone-by-zone update counts and failures in every stage, and
    the same state to 1e-12 after three steps; with the cut at one update
    the rounds hand the slow zones to the queue kernel as the one-pass
    kernel does."""
    from paper_1702_01106_b300.grim import Grim
    from tests.gpu_helpers import rel_field_err
    prob = inputs.torus_problem(16, 12, 6, tol=1e-12)
    P = inputs.torus_state(prob)
    dt = inputs.torus_dt(prob)
    runs = {}
    for rounds, kcut in ((0, prob.k_max), (1, prob.k_max), (1, 1), (1, 3)):
        g = Grim(prob, precision=precision)
        g.set_tuning(newton_rounds=rounds, newton_kcut=kcut)
        a = torch.from_numpy(P).to(dev)
        h = torch.empty_like(a)
        b = torch.empty_like(a)
        it = torch.zeros(prob.zones, dtype=torch.uint8, device=dev)
        st = torch.zeros_like(it)
        per_stage = []
        for _ in range(3):
            g.stage(a, a, 0.5 * dt, h, iters=it, status=st)
            per_stage.append((it.cpu().numpy().copy(), st.cpu().numpy() != 0))
            g.stage(a, h, dt, b, iters=it, status=st)
            per_stage.append((it.cpu().numpy().copy(), st.cpu().numpy() != 0))
            a, b = b, a
        runs[(rounds, kcut)] = (a.cpu().numpy(), per_stage, g.stats())
        g.close()
    ref, ref_stages, sref = runs[(0, prob.k_max)]
    assert sref["failed"] > 0 or precision == 1
    for key, (out, stages, s) in runs.items():
        for (i0, f0), (i1, f1) in zip(ref_stages, stages):
            assert np.array_equal(f0, f1), key
            assert np.array_equal(i0[~f0], i1[~f1]), key
        assert rel_field_err(out.reshape(10, -1), ref.reshape(10, -1)).max() < 1e-12, key
        assert s["zones"] == sref["zones"] and s["failed"] == sref["failed"], key
        assert s["iters"] == sref["iters"] and s["evals64"] == sref["evals64"], key


def test_compaction_moves_slow_zones_to_the_queue(dev):
    """With the cut at one update, the zones that need more finish in the
    queue kernel: same per-zone update histogram as the in-order kernel and
    one launch more per stage."""
    prob = inputs.turbulent_box_problem(64)
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / 64
    ref, sref = _run(prob, P, dt, dev, 1, steps=1, newton_kcut=prob.k_max + 1)
    out, s = _run(prob, P, dt, dev, 1, steps=1, newton_kcut=1)
    assert sum(sref["hist"][2:]) > 0                # some zones need more than one update
    assert s["launches"] == sref["launches"] + 2
    assert s["zones"] == sref["zones"] and s["failed"] == 0
    assert abs(s["iters"] - sref["iters"]) <= 0.01 * sref["iters"]


def test_graph_replay_is_bit_identical(dev):
    """Steps replayed from captured graphs (two graphs: a->b and b->a, plus an
    in-place one) equal eager steps; the launch count still adds up."""
    from paper_1702_01106_b300.grim import Grim
    prob = inputs.turbulent_box_problem(64)
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / 64
    ref, sref = _run(prob, P, dt, dev, 1, steps=6)
    out, s = _run(prob, P, dt, dev, 1, steps=6, graphs=True)
    assert np.array_equal(out, ref)
    assert s["launches"] == sref["launches"] and s["iters"] == sref["iters"]
    g = Grim(prob, precision=1)
    g.use_graphs(True)
    a = torch.from_numpy(P).to(dev)
    for _ in range(6):
        g.step(a, a, dt)
    assert np.array_equal(a.cpu().numpy(), ref)
    g.close()


def test_autotune_picks_a_valid_shape_and_caches_it(dev, tmp_path):
    from paper_1702_01106_b300.grim import Grim
    prob = inputs.turbulent_box_problem(128)
    P = torch.from_numpy(inputs.turbulent_box_state(prob)).to(dev)
    P0 = P.clone()
    dt = 0.5 / 128
    path = str(tmp_path / "tune.jsonl")
    g = Grim(prob, precision=1)
    t, ms = g.autotune(P, dt, path)
    assert torch.equal(P, P0)                      # the state is not modified
    assert t["newton_bs"] in (32, 64, 128) and t["newton_kcut"] >= 1 and t["newton_rounds"] in (0, 1)
    assert t["faces_bs"] in (64, 128, 256) and t["zone_bs"] in (64, 128, 256)
    assert ms > 0 and g.tuning() == t
    assert g.stats()["zones"] == 0                 # statistics reset
    lines = open(path).read().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert {k: rec[k] for k in t} == t and "prec1" in rec["key"]
    g.close()
    g2 = Grim(prob, precision=1)
    t2, ms2 = g2.autotune(P, dt, path)             # served from the cache
    assert t2 == t and abs(ms2 - ms) < 1e-3
    g2.close()
    g3 = Grim(prob, precision=0)                   # another key: appended
    g3.autotune(P, dt, path)
    assert len(open(path).read().splitlines()) == 2
    g3.close()
    os.remove(path)
