"""Parity of the general-metric path (3-D grids, modified Kerr-Schild) with
the FP64 oracle, through the C ABI."""
import math

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


def _t(P, dev):
    return torch.from_numpy(np.ascontiguousarray(P)).to(dev)


def _box3d(n=(12, 10, 8), tol=1e-14, seed=11):
    """3-D periodic box: the linear-mode state plus seeded noise (1e-3) on
    every field, so that all three directions carry structure."""
    prob = inputs.linear_mode_problem(n[0], tol=tol).with_(dim=3, n=n)
    P = inputs.linear_mode_state(prob, amp=1e-4, phase=inputs.linear_mode_phase(1))
    rng = np.random.Generator(np.random.Philox(seed))
    P = P + 1e-3 * rng.standard_normal(P.shape) * np.array([1, 1, 1, 1, 1, 1, 1, 1, 0, 0])[:, None, None, None]
    return prob, P


def _torus(n1, n2, n3, tol=1e-14):
    prob = inputs.torus_problem(n1, n2, n3, tol=tol)
    return prob, inputs.torus_state(prob)


@pytest.mark.parametrize("precision", [0, 1])
def test_gr_residual_parity_kerr(dev, orc, precision):
    """The stage residual on the torus against the oracle's, per row relative
    to |r| + 1.  Float64 within 1e-11.  The mixed solver forms its face
    states (the MC values from float-float slopes) and fluxes in float-float,
    about 48 significant bits: at the torus surface, where the flux
    divergence is ~1e3 times what a zone holds, a rounding of 2^-47 of the
    face values is ~1e3 x 2^-47 ~ 1e-11 of the scaled residual, so its bound
    is 2e-11."""
    from paper_1702_01106_b300.grim import Grim
    prob, Pn = _torus(20, 16, 1)
    rng = np.random.default_rng(5)
    PE = Pn * (1 + 1e-3 * rng.standard_normal(Pn.shape))
    Pk = Pn * (1 + 1e-3 * rng.standard_normal(Pn.shape))
    dts = 0.5 * inputs.torus_dt(prob)
    g = Grim(prob, precision=precision)
    R = torch.empty_like(_t(Pn, dev))
    g.residual(_t(Pn, dev), _t(PE, dev), dts, _t(Pk, dev), R)
    ref = orc.residual(prob, Pn, PE, dts, Pk)
    # torus-surface zones carry scaled residuals up to ~1e3 at P_n
    bound = 1e-11 if precision == 0 else 2e-11
    assert (np.abs(R.cpu().numpy() - ref) / (np.abs(ref) + 1.0)).max() < bound
    g.close()


@pytest.mark.parametrize("shape,tol,bound", [((20, 16, 1), 1e-12, 1e-11), ((16, 12, 6), 1e-12, 1e-11),
                                             ((12, 10, 4), 1e-12, 1e-11)])
def test_gr_stage_parity_kerr(dev, orc, shape, tol, bound):
    """One stage of the torus: the same zones fail to find an admissible root
    (torus-surface zones whose explicit update has none) and revert to their
    start; every zone agrees with the oracle to `bound`.  The grids are
    solved to 1e-12: torus-surface zones carry scaled residual terms of
    order 1e3, whose rounding (~1e-13) is the floor below which they cannot
    converge; near that floor the cold gas's Jacobian columns (relative
    steps on u ~ 1e-3 rho) carry rounding of ~1e-4, and the two codes'
    different rounding decides which marginal zones stall.  At 1e-12 every
    zone converges or finds no admissible root alike."""
    from paper_1702_01106_b300.grim import Grim
    prob, Pn = _torus(*shape, tol=tol)
    dts = 0.5 * inputs.torus_dt(prob)
    g = Grim(prob)
    out = torch.empty_like(_t(Pn, dev))
    st = torch.zeros(prob.zones, dtype=torch.uint8, device=dev)
    g.stage(_t(Pn, dev), _t(Pn, dev), dts, out, status=st)
    ref, _, rst, _ = orc.stage(prob, Pn, Pn, dts)
    assert np.array_equal(st.cpu().numpy() != 0, rst != 0)
    assert (rst != 0).mean() < 0.1
    err = rel_field_err(out.cpu().numpy(), ref).max()
    assert err < bound, err
    g.close()


def test_gr_step_3d_minkowski(dev, orc):
    from paper_1702_01106_b300.grim import Grim
    prob, P = _box3d()
    dt = 0.5 / 12
    g = Grim(prob)
    out = torch.empty_like(_t(P, dev))
    g.step(_t(P, dev), out, dt)
    ref, _, st, _ = orc.step(prob, P, dt)
    assert st.max() == 0 and g.stats()["failed"] == 0
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-12
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_gr_step_3d_kerr(dev, orc, precision):
    """One step of a 3-D torus (floors on), both codes at tol 1e-12 (above the
    torus-surface zones' round-off floor, see test_gr_stage_parity_kerr):
    float64 within 1e-10 of the oracle (two stages at tol 1e-12; the energy
    row fixes the cold gas's u only to ~tol rho/u, about 1e2 tol), mixed
    precision within 1e-9; failures (zones without an admissible root,
    reverted to their start) are few."""
    from paper_1702_01106_b300.grim import Grim
    prob, P = _torus(16, 12, 6, tol=1e-12)
    dt = inputs.torus_dt(prob)
    g = Grim(prob, precision=precision)
    out = torch.empty_like(_t(P, dev))
    g.step(_t(P, dev), out, dt)
    s = g.stats()
    ref, _, st, _ = orc.step(prob, P, dt)
    assert s["failed"] < 0.05 * s["zones"]
    err = rel_field_err(out.cpu().numpy(), ref).max()
    assert err < (1e-10 if precision == 0 else 1e-9), err
    g.close()


def _corner_div(prob, P, sqrtg):
    """Corner divergence of sqrt(-g) B^i (the quantity flux-CT keeps):
    at corner (i-1/2, j-1/2, k-1/2) the difference along d of sqrt(-g) B^d
    averaged over the zones adjacent along the other active directions."""
    dim = prob.dim
    F = [sqrtg * P[5 + d] for d in range(dim)]
    axes = {0: 2, 1: 1, 2: 0}                     # array axis of direction d ([n3, n2, n1])
    div = 0.0
    for d in range(dim):
        f = F[d]
        diff = f - np.roll(f, 1, axis=axes[d])
        for e in range(dim):
            if e != d:
                diff = 0.5 * (diff + np.roll(diff, 1, axis=axes[e]))
        div = div + diff / prob.dx[d]
    return div


def test_gr_3d_flux_ct_keeps_divergence(dev):
    """3-D periodic box: the corner divergence of B is unchanged to round-off
    over 3 steps (flux-CT on all three planes)."""
    from paper_1702_01106_b300.grim import Grim
    prob, P = _box3d(n=(12, 10, 8), tol=1e-12)
    d0 = _corner_div(prob, P, 1.0)
    g = Grim(prob)
    a = _t(P, dev)
    for _ in range(3):
        g.step(a, a, 0.5 / 12)
    d1 = _corner_div(prob, a.cpu().numpy(), 1.0)
    scale = np.abs(P[5:8]).max() / min(prob.dx[:3])
    assert np.abs(d1 - d0).max() < 1e-12 * scale
    g.close()


def test_gr_kerr_conservation_of_mass(dev):
    """Axisymmetric Kerr torus with periodic X1 and X3 is not available (the
    horizon); instead: a 3-D Minkowski box conserves sum sqrt(-g) rho u^t to
    round-off with tol at the round-off floor."""
    from paper_1702_01106_b300.grim import Grim
    prob, P = _box3d(tol=1e-14)
    g = Grim(prob)
    a = _t(P, dev)

    def mass(Q):
        v2 = Q[2] ** 2 + Q[3] ** 2 + Q[4] ** 2
        return float((Q[0] * np.sqrt(1 + v2)).sum())

    m0 = mass(P)
    for _ in range(2):
        g.step(a, a, 0.5 / 12)
    assert abs(mass(a.cpu().numpy()) - m0) < 1e-12 * abs(m0)
    g.close()


@pytest.mark.parametrize("recon", [inputs.RECON_MC, inputs.RECON_PPM])
def test_gr_step_hlle(dev, orc, recon):
    """HLLE on the general-metric path: one step of the 3-D box within 1e-12
    of the oracle, and one stage of the axisymmetric torus (tol 1e-12, the
    same failed zones) within 1e-11 (MC and PPM)."""
    from paper_1702_01106_b300.grim import Grim
    prob, P = _box3d()
    prob = prob.with_(riemann=inputs.FLUX_HLLE, recon=recon)
    g = Grim(prob)
    out = torch.empty_like(_t(P, dev))
    g.step(_t(P, dev), out, 0.5 / 12)
    ref, _, st, _ = orc.step(prob, P, 0.5 / 12)
    assert st.max() == 0
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-12
    g.close()
    prob, Pn = _torus(20, 16, 1, tol=1e-12)
    prob = prob.with_(riemann=inputs.FLUX_HLLE, recon=recon)
    dts = 0.5 * inputs.torus_dt(prob)
    g = Grim(prob)
    out = torch.empty_like(_t(Pn, dev))
    st = torch.zeros(prob.zones, dtype=torch.uint8, device=dev)
    g.stage(_t(Pn, dev), _t(Pn, dev), dts, out, status=st)
    ref, _, rst, _ = orc.stage(prob, Pn, Pn, dts)
    assert np.array_equal(st.cpu().numpy() != 0, rst != 0)
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-11
    g.close()


def test_gr_full_size_torus_sampled_parity(dev, orc):
    """The 192 x 192 x 128 Kerr torus in the benchmark's configuration (tol
    1e-10, float64 and mixed): zones sampled across the torus, its surface,
    the atmosphere, the inner boundary and the axis agree with the oracle's
    step of those zones (solved to 1e-14) within 1e-9; no zone fails."""
    from paper_1702_01106_b300.grim import Grim
    prob = inputs.torus_problem(192, 192, 128)
    P = inputs.torus_state(prob)
    dt = inputs.torus_dt(prob)
    n1, n2, n3 = prob.n
    rng = np.random.default_rng(17)
    pick = [(0, 96, 0), (n1 - 1, 96, 5), (60, 0, 7), (60, n2 - 1, n3 - 1), (70, 96, 64), (45, 80, 3)]
    pick += [tuple(int(x) for x in rng.integers(0, [n1, n2, n3])) for _ in range(18)]
    zs = np.array([(k * n2 + j) * n1 + i for i, j, k in pick], dtype=np.int64)
    ref, _, st, _ = orc.step_sampled(prob.with_(tol=1e-14), P, dt, zs)
    for precision in (0, 1):
        g = Grim(prob, precision=precision)
        out = torch.empty_like(_t(P, dev))
        g.step(_t(P, dev), out, dt)
        s = g.stats()
        assert s["failed"] == 0 and s["max_res"] <= prob.tol
        got = out.cpu().numpy().reshape(10, -1)[:, zs]
        assert rel_field_err(got, ref).max() < 1e-9
        g.close()


@pytest.mark.parametrize("shape", [(9, 7, 3), (5, 11, 2), (13, 1, 1)])
def test_gr_odd_grids_minkowski(dev, orc, shape):
    """Ragged 3-D grids (and a one-zone-wide 2-D one) on the general-metric
    path: one float64 step within 1e-12 of the oracle."""
    from paper_1702_01106_b300.grim import Grim
    n = shape
    dim = 3 if n[2] > 1 else 2
    prob, P = _box3d(n=n)
    prob = prob.with_(dim=dim)
    if dim == 2:
        prob = prob.with_(metric=inputs.METRIC_MINKOWSKI)
        P = P[:, :1]
    g = Grim(prob)
    out = torch.empty_like(_t(P, dev))
    g.step(_t(P, dev), out, 0.5 / 13)
    ref, _, st, _ = orc.step(prob, P, 0.5 / 13)
    assert st.max() == 0 and g.stats()["failed"] == 0
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-12
    g.close()


def test_gr_learned_start_equals_reference_prediction(dev):
    """The learned start in a general metric (the torus, floors off): with
    k_max = 0 a stage returns its start, P_n + y times the field's unit (P_n
    for rho and u, |X_n| + rho_n for q~ and dP~, 1 for the velocities), y the
    network's output on the stage's features (the residual at P_n, the
    zone's g_{mu nu}, P_n in those units), with the magnetic components from
    flux-CT.  Zones whose start is worse than P_n fall back to P_n; the rest
    carry the prediction."""
    from paper_1702_01106_b300.grim import MLP, Grim
    from oracle import mlp_ref
    prob, P = _torus(20, 16, 1)
    prob = prob.with_(k_max=0, floors=False)
    a = _t(P, dev)
    out = torch.empty_like(a)
    dts = 0.5 * inputs.torus_dt(prob)
    g = Grim(prob, precision=1)
    g.stage(a, a, dts, out)                      # the stage's constants, plain start
    X = torch.empty((prob.zones, 32), dtype=torch.float32, device=dev)
    g.mlp_sample(a, None, X)
    Xh = X.cpu().numpy()
    assert np.ptp(Xh[:, 10:20], axis=0).max() > 0   # the metric varies over the torus
    m = MLP(seed=7)
    params, _ = m.get_params()
    norm = np.zeros(96, np.float32)
    norm[:32] = Xh.mean(axis=0)
    norm[32:64] = np.maximum(Xh.std(axis=0), 1e-6)
    norm[80:96] = 1e-9    # small corrections keep every start admissible
    m.set_params(params, norm)
    g.set_guess(m, accept=1e30)
    g.reset_stats()
    g.stage(a, a, dts, out)
    nfb = g.stats()["fallbacks"]
    pred = mlp_ref.predict(params, norm, Xh, bf16_round=True)
    got = out.cpu().numpy().reshape(10, -1)
    Pn = P.reshape(10, -1)
    fields = [0, 1, 2, 3, 4, 8, 9]
    from tests.gpu_helpers import learned_units
    unit = learned_units(Pn)
    kept = ~np.all(got[fields] == Pn[fields], axis=0)
    assert (~kept).sum() == nfb and nfb <= 0.02 * prob.zones, nfb
    for o in fields:
        scale = np.abs(pred[kept, o]).max() + 1e-30
        dgot = (got[o, kept] - Pn[o, kept]) / unit[o, kept]
        diff = np.abs(dgot - pred[kept, o]) / scale
        assert diff.max() <= 3e-2, o
        assert np.median(diff) <= 3e-3, o
    g.close()
    m.close()


def test_gr_trained_guess_keeps_the_answer(dev, orc):
    """Trained on converged stages of a small 3-D torus, the learned start
    leaves the answer where the plain start puts it: the Newton updates stay
    within a tenth of the plain start's, as few zones fail (torus-surface
    zones without an admissible root), and the result stays within 1e-9 of
    the oracle (sampled zones inside the torus).  On this grid the learned
    start does not save updates (the benchmark reports the full-size
    torus)."""
    from paper_1702_01106_b300 import guess
    from paper_1702_01106_b300.grim import Grim, GRIM_MIXED
    prob, P = _torus(24, 24, 8, tol=1e-12)   # as test_gr_step_3d_kerr's mixed case
    dt = inputs.torus_dt(prob)
    X, Y, P1 = guess.collect(prob, P, dt, 4, dev)
    P1 = P1.cpu().numpy()
    m, losses = guess.train(X, Y, steps=4000)
    assert losses[-1] < 0.9 * losses[0]
    iters, outs, fails = {}, {}, {}
    for learned in (False, True):
        g = Grim(prob, precision=GRIM_MIXED)
        if learned:
            g.set_guess(m, accept=1e-3)
        a = torch.from_numpy(P1).to(dev)
        out = torch.empty_like(a)
        g.step(a, out, dt)
        s = g.stats()
        assert s["failed"] <= 0.02 * s["zones"], s
        iters[learned] = s["iters"] / s["zones"]
        fails[learned] = s["failed"]
        outs[learned] = out.cpu().numpy()
        g.close()
    assert iters[True] < iters[False] + 0.1, iters
    assert fails[True] <= fails[False] + 0.005 * prob.zones, fails
    rho = P1.reshape(10, -1)[0]
    inside = np.nonzero(rho > 0.05 * rho.max())[0]
    zs = np.random.default_rng(10).choice(inside, 48, replace=False)
    ref, _, _, _ = orc.step_sampled(prob.with_(tol=1e-14), P1, dt, zs)
    assert rel_field_err(outs[True].reshape(10, -1)[:, zs], ref).max() < 1e-9
    m.close()
