"""The learned initial guess on the GPU: device gradients and inference
against the numpy reference, and the end-to-end gain of a trained network."""
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


def _norm(rng):
    return np.concatenate([rng.normal(0, 1, 32), rng.uniform(0.5, 2, 32), rng.normal(0, 1, 16),
                           rng.uniform(0.5, 2, 16)]).astype(np.float32)


def test_device_gradient_matches_reference(dev):
    from paper_1702_01106_b300.grim import MLP
    from oracle import mlp_ref
    rng = np.random.default_rng(3)
    m = MLP(seed=11)
    params, _ = m.get_params()
    params = params + rng.normal(0, 0.05, params.size).astype(np.float32)  # non-zero biases everywhere
    norm = _norm(rng)
    m.set_params(params, norm)
    M = 512
    X = rng.normal(0, 1, (M, 32)).astype(np.float32) * norm[32:64] + norm[:32]
    Y = rng.normal(0, 1, (M, 16)).astype(np.float32) * norm[80:96] + norm[64:80]
    g, loss = m.gradient(torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev))
    lref, gref = mlp_ref.loss_and_grad(params, norm, X, Y, bf16_round=True)
    assert abs(loss - lref) <= 1e-3 * lref
    o = 0
    for no, ni in mlp_ref.SIZES:
        for n in (no * ni, no):
            a, b = g[o:o + n], gref[o:o + n]
            assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-12, (o, n)
            o += n
    m.close()


def test_features_are_the_stage_increment(dev, orc):
    """Features of a stage: [0..9] minus the oracle's scaled residual at P_n
    (the explicit increment in the residual's row scaling), [10..19] the
    Minkowski metric, [20..29] P_n, [30..31] zero."""
    from paper_1702_01106_b300.grim import Grim
    prob = inputs.turbulent_box_problem(32).with_(n=(48, 40, 1), k_max=0)
    P = inputs.turbulent_box_state(prob)
    g = Grim(prob, precision=1)
    a = torch.from_numpy(P).to(dev)
    out = torch.empty_like(a)
    dts = 0.25 / 32
    g.stage(a, a, dts, out)
    X = torch.empty((prob.zones, 32), dtype=torch.float32, device=dev)
    g.mlp_sample(a, None, X)
    X = X.cpu().numpy().astype(np.float64)
    r = orc.residual(prob, P, P, dts, P).reshape(10, -1)
    for f in range(10):
        scale = np.abs(r[f]).max()
        assert np.abs(X[:, f] + r[f]).max() <= 1e-6 * scale + 1e-30, f
    eta = np.array([-1, 0, 0, 0, 1, 0, 0, 1, 0, 1], np.float64)   # g_tt, g_tx, .., g_zz
    assert np.array_equal(X[:, 10:20], np.broadcast_to(eta, (prob.zones, 10)))
    from tests.gpu_helpers import learned_pn_features
    Pf = learned_pn_features(P)           # log rho, log u, q~ and dP~ over |X| + rho
    assert np.abs(X[:, 20:30] - Pf).max() <= 1e-6 * np.abs(Pf).max()
    assert not X[:, 30:].any()
    g.close()


def test_learned_start_equals_reference_prediction(dev):
    """With k_max = 0 the stage returns its start: P_n + y times the field's
    unit (P_n for rho and u, |X_n| + rho_n for q~ and dP~, 1 for u^i), y the
    network's output on the stage's features (magnetic components from
    flux-CT)."""
    from paper_1702_01106_b300.grim import MLP, Grim
    from oracle import mlp_ref
    rng = np.random.default_rng(4)
    prob = inputs.turbulent_box_problem(32).with_(n=(48, 40, 1), k_max=0)
    P = inputs.turbulent_box_state(prob)
    m = MLP(seed=5)
    params, _ = m.get_params()
    norm = np.zeros(96, np.float32)
    norm[32:64] = 1.0
    norm[64:80] = 0.0
    norm[80:96] = 1e-5    # small corrections keep every start admissible
    norm[32:42] = 1e-3
    norm[52:62] = rng.uniform(0.1, 1, 10).astype(np.float32)
    m.set_params(params, norm)
    g = Grim(prob, precision=1)
    g.set_guess(m, accept=1e30)
    a = torch.from_numpy(P).to(dev)
    out = torch.empty_like(a)
    dts = 0.25 / 32
    g.stage(a, a, dts, out)
    X = torch.empty((prob.zones, 32), dtype=torch.float32, device=dev)
    g.mlp_sample(a, None, X)
    pred = mlp_ref.predict(params, norm, X.cpu().numpy(), bf16_round=True)
    from tests.gpu_helpers import learned_units
    got = out.cpu().numpy().reshape(10, -1)
    Pn = P.reshape(10, -1)
    unit = learned_units(Pn)
    for o in (0, 1, 2, 3, 4, 8, 9):
        # the device SiLU uses the hardware tanh approximation (relative error
        # ~2^-11) and a different float32 summation order, which can flip the
        # bfloat16 rounding of an activation (one part in 2^8)
        scale = np.abs(pred[:, o]).max() + 1e-6
        dgot = (got[o] - Pn[o]) / unit[o]
        diff = np.abs(dgot - pred[:, o]) / scale
        assert diff.max() <= 3e-2, o
        assert np.median(diff) <= 3e-3, o
    g.close()
    m.close()


def test_trained_guess_saves_newton_iterations(dev, orc):
    """Trained on converged stages of one 256^2 turbulent box (2^20 samples),
    the learned start removes Newton iterations on a held-out box (at this
    resolution the plain start needs 2-3 per stage); results stay within 1e-9
    of the oracle (sampled zones)."""
    from paper_1702_01106_b300 import guess
    from paper_1702_01106_b300.grim import Grim, GRIM_MIXED
    n = 256
    prob = inputs.turbulent_box_problem(n)
    dt = 0.5 / n
    P = inputs.turbulent_box_state(prob)
    X, Y, _ = guess.collect(prob, P, dt, 8, dev)
    m, losses = guess.train(X, Y, steps=6000)
    assert losses[-1] < 0.9 * losses[0]
    P2 = inputs.turbulent_box_state(prob, seed_rho=4, seed_vel=5)   # held out
    iters, outs = {}, {}
    for learned in (False, True):
        g = Grim(prob, precision=GRIM_MIXED)
        if learned:
            g.set_guess(m, accept=1e-7)
        a = torch.from_numpy(P2).to(dev)
        out = torch.empty_like(a)
        g.step(a, out, dt)
        s = g.stats()
        assert s["failed"] == 0 and s["max_res"] <= prob.tol
        iters[learned] = s["iters"] / s["zones"]
        outs[learned] = out.cpu().numpy()
        if learned:
            assert s["fallbacks"] < 0.05 * s["zones"]
        g.close()
    assert iters[False] > 2.2 and iters[True] < iters[False] - 0.2, iters
    zs = np.random.default_rng(9).choice(prob.zones, 64, replace=False)
    ref, _, _, _ = orc.step_sampled(prob.with_(tol=1e-14), P2, dt, zs)
    assert rel_field_err(outs[True].reshape(10, -1)[:, zs], ref).max() < 1e-9
    m.close()
