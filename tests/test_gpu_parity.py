"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Grids span several 16x16 tiles with ragged tails; the full-size workload is
checked on sampled zones in the launch configuration the benchmark times.
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


def _g(prob, precision=0):
    from paper_1702_01106_b300.grim import Grim
    return Grim(prob, precision=precision)


def _t(P, dev):
    return torch.from_numpy(np.ascontiguousarray(P)).to(dev)


def _ragged_turbulent(n1=40, n2=24, tol=1e-14, **kw):
    prob = inputs.turbulent_box_problem(32, tol=tol, **kw).with_(n=(n1, n2, 1))
    P = inputs.turbulent_box_state(inputs.turbulent_box_problem(32).with_(n=(n1, n2, 1)))
    return prob, P


def test_residual_parity(dev, orc):
    prob, Pn = _ragged_turbulent()
    rng = np.random.default_rng(1)
    PE = Pn * (1 + 1e-3 * rng.standard_normal(Pn.shape))
    Pk = Pn * (1 + 1e-3 * rng.standard_normal(Pn.shape))
    dts = 0.25 / 32
    g = _g(prob)
    R = torch.empty_like(_t(Pn, dev))
    for scaled in (True, False):
        g.residual(_t(Pn, dev), _t(PE, dev), dts, _t(Pk, dev), R, scaled=scaled)
        ref = orc.residual(prob, Pn, PE, dts, Pk, scaled=scaled)
        got = R.cpu().numpy()
        if scaled:
            assert np.abs(got - ref).max() < 1e-13
        else:
            err = np.abs(got - ref).reshape(10, -1).max(axis=1)
            mag = np.abs(ref).reshape(10, -1).max(axis=1) + 1.0 / dts
            assert np.all(err < 1e-12 * mag), err / mag


@pytest.mark.parametrize("recon", [inputs.RECON_MC, inputs.RECON_WENO5, inputs.RECON_PPM])
def test_stage_parity(dev, orc, recon):
    prob, Pn = _ragged_turbulent(recon=recon)
    dts = 0.25 / 32
    g = _g(prob)
    out = torch.empty_like(_t(Pn, dev))
    it = torch.zeros(prob.zones, dtype=torch.uint8, device=dev)
    st = torch.zeros(prob.zones, dtype=torch.uint8, device=dev)
    g.stage(_t(Pn, dev), _t(Pn, dev), dts, out, iters=it, status=st)
    ref, rit, rst, _ = orc.stage(prob, Pn, Pn, dts)
    assert int(st.max()) == 0 and rst.max() == 0
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-12
    assert np.abs(it.cpu().numpy().astype(int) - rit).max() <= 1


def test_one_step_linear_mode(dev, orc):
    prob = inputs.linear_mode_problem(48, tol=1e-14)
    P = inputs.linear_mode_state(prob, amp=1e-4, phase=inputs.linear_mode_phase(1))
    dt = 0.5 / 48
    g = _g(prob)
    out = torch.empty_like(_t(P, dev))
    g.step(_t(P, dev), out, dt)
    ref, _, st, _ = orc.step(prob, P, dt)
    assert st.max() == 0
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-12
    s = g.stats()
    assert s["failed"] == 0 and s["zones"] == 2 * prob.zones


def test_many_steps_turbulent(dev, orc):
    """100 steps on a ragged grid beside the oracle's (tol 1e-14): the
    float64 path (tol 1e-14) and the mixed solver (tol 1e-12; its float32
    Jacobian converges linearly, so 1e-12 is where it still converges in a
    few updates) both within 1e-9 per primitive after 100 steps.  Each
    step's root is fixed to ~kappa tol, so 100 steps accumulate at most
    ~100 kappa tol ~ 1e-10."""
    prob, P = _ragged_turbulent(40, 24, tol=1e-14)
    dt = 0.5 / 40
    g = _g(prob)
    gm = _g(prob.with_(tol=1e-12), precision=1)
    a = _t(P, dev)
    b = torch.empty_like(a)
    am = _t(P, dev)
    bm = torch.empty_like(am)
    ref = P.copy()
    errs = []
    for n in range(100):
        g.step(a, b, dt)
        a, b = b, a
        gm.step(am, bm, dt)
        am, bm = bm, am
        ref, _, st, _ = orc.step(prob, ref, dt)
        assert st.max() == 0
        if n in (0, 9, 99):
            errs.append((rel_field_err(a.cpu().numpy(), ref).max(), rel_field_err(am.cpu().numpy(), ref).max()))
    assert errs[0][0] < 1e-12
    assert errs[-1][0] < 1e-9 and errs[-1][1] < 1e-9, errs
    assert g.stats()["failed"] == 0
    sm = gm.stats()
    assert sm["failed"] == 0 and sm["max_res"] <= 1e-12 and sm["evals32"] > 0


def _corner_div_2d(prob, P):
    """Corner divergence of B on a periodic 2-D grid (the quantity flux-CT
    keeps, Section 4.2): at corner (i-1/2, j-1/2) the differences of B^1
    along x^1 and of B^2 along x^2, each averaged over the two zones
    adjacent along the other direction."""
    B1, B2 = P[5, 0], P[6, 0]                       # [n2][n1]
    d1 = B1 - np.roll(B1, 1, axis=1)
    d1 = 0.5 * (d1 + np.roll(d1, 1, axis=0))
    d2 = B2 - np.roll(B2, 1, axis=0)
    d2 = 0.5 * (d2 + np.roll(d2, 1, axis=1))
    return d1 / prob.dx[0] + d2 / prob.dx[1]


@pytest.mark.parametrize("precision", [0, 1])
def test_flux_ct_keeps_divergence_100_steps(dev, precision):
    """100 steps of the periodic ragged box, float64 and the mixed solver:
    flux-CT leaves the corner divergence of B unchanged to round-off (each
    step adds only float64 rounding: the edge EMFs are doubles also when the
    mixed solver forms the face fluxes in float-float)."""
    prob, P = _ragged_turbulent(40, 24, tol=1e-12)
    dt = 0.5 / 40
    g = _g(prob, precision=precision)
    a = _t(P, dev)
    d0 = _corner_div_2d(prob, P)
    for _ in range(100):
        g.step(a, a, dt)
    d1 = _corner_div_2d(prob, a.cpu().numpy())
    scale = np.abs(P[5:7]).max() / min(prob.dx[:2])
    assert np.abs(d1 - d0).max() < 1e-12 * scale
    assert g.stats()["failed"] == 0
    g.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-14), (1, 1e-12)])
def test_periodic_box_conserves_mass_energy_momentum(dev, orc, precision, tol):
    """20 steps of the periodic 24^2 box, float64 and the mixed solver: the
    totals of rho u^t, T^t_t and T^t_i (from the oracle's U(P)) move by no
    more than the solver tolerance allows.  A full stage ends with every
    zone's scaled residual |r_a| <= tol, r_a = (U_a(P) - U*_a) / (|U_a(P_n)|
    + |U_0(P_n)|), and the totals of U* equal those of U(P_n) on a periodic
    grid (the flux differences telescope), so a step moves total a by at
    most tol sum(|U_a| + |U_0|); the bound takes twice that."""
    prob = inputs.turbulent_box_problem(24, tol=tol)
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / 24
    steps = 20

    def totals(Q):
        tot, mag = np.zeros(5), np.zeros(5)
        for z in range(prob.zones):
            U, _, _ = orc.point(prob, Q.reshape(10, -1)[:, z])
            tot += U[:5]
            mag += np.abs(U[:5])
        return tot, mag

    t0, m0 = totals(P)
    g = _g(prob, precision=precision)
    a = _t(P, dev)
    for _ in range(steps):
        g.step(a, a, dt)
    assert g.stats()["failed"] == 0
    t1, _ = totals(a.cpu().numpy())
    bound = 2.0 * steps * tol * (m0 + m0[0])
    assert np.all(np.abs(t1 - t0) <= bound), np.abs(t1 - t0) / bound
    g.close()


def test_in_place_step(dev, orc):
    prob, P = _ragged_turbulent(24, 40)
    g = _g(prob)
    a = _t(P, dev)
    g.step(a, a, 0.5 / 40)
    ref, _, _, _ = orc.step(prob, P, 0.5 / 40)
    assert rel_field_err(a.cpu().numpy(), ref).max() < 1e-12


def test_mixed_precision_matches_fp64(dev, orc):
    """FP32 Jacobian/LU, FP64 residual and test: at tol 1e-10 every zone
    reaches max|r| <= 1e-10 and the primitives stay within 1e-9 of the FP64 oracle."""
    prob, P = _ragged_turbulent(40, 24, tol=1e-10)
    dt = 0.5 / 40
    g = _g(prob, precision=1)
    out = torch.empty_like(_t(P, dev))
    g.step(_t(P, dev), out, dt)
    s = g.stats()
    assert s["failed"] == 0 and s["max_res"] <= 1e-10 and s["evals32"] > 0
    ref, _, _, _ = orc.step(prob.with_(tol=1e-14), P, dt)
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-9


@pytest.mark.parametrize("shape", [(1, 1), (1, 17), (17, 1), (16, 16), (33, 17)])
def test_small_and_degenerate_grids(dev, orc, shape):
    prob, P = _ragged_turbulent(*shape, tol=1e-14)
    g = _g(prob)
    out = torch.empty_like(_t(P, dev))
    g.step(_t(P, dev), out, 0.01)
    ref, _, _, _ = orc.step(prob, P, 0.01)
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-12


def test_full_size_sampled_parity(dev, orc):
    """The 1024^2 turbulent box in the benchmark's configuration (tol 1e-10):
    sampled zones against the oracle, and the residual bound everywhere."""
    prob = inputs.turbulent_box_problem(1024)
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / 1024
    for precision in (0, 1):
        g = _g(prob, precision)
        out = torch.empty_like(_t(P, dev))
        g.step(_t(P, dev), out, dt)
        s = g.stats()
        assert s["failed"] == 0 and s["max_res"] <= prob.tol
        rng = np.random.default_rng(7 + precision)
        zs = np.concatenate([rng.choice(prob.zones, 48, replace=False), [0, 1023, prob.zones - 1]])
        ref, _, st, _ = orc.step_sampled(prob.with_(tol=1e-14), P, dt, zs)
        got = out.cpu().numpy().reshape(10, -1)[:, zs]
        assert rel_field_err(got, ref).max() < 1e-9
        g.close()


def test_reciprocal_matches_ieee_division(dev):
    """The Newton-Raphson reciprocal used for FD divisors and LU pivots stays
    within one rounding of IEEE division over 2^-300..2^300."""
    from paper_1702_01106_b300.grim import math_selftest
    assert math_selftest(1 << 20) <= 2.0 ** -52


@pytest.mark.parametrize("bc", [((1, 1), (2, 2), (0, 0)), ((2, 1), (0, 0), (0, 0)), ((0, 0), (1, 2), (0, 0))])
def test_stage_parity_non_periodic_boundaries(dev, orc, bc):
    """Outflow (copy) and reflecting boundaries applied by the tile/face loaders."""
    prob, Pn = _ragged_turbulent(20, 18, tol=1e-14)
    prob = prob.with_(bc=bc)
    dts = 0.25 / 32
    g = _g(prob)
    out = torch.empty_like(_t(Pn, dev))
    g.stage(_t(Pn, dev), _t(Pn, dev), dts, out)
    ref, _, rst, _ = orc.stage(prob, Pn, Pn, dts)
    assert rst.max() == 0
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-12


@pytest.mark.parametrize("recon", [inputs.RECON_MC, inputs.RECON_WENO5, inputs.RECON_PPM])
def test_stage_parity_hlle(dev, orc, recon):
    """The HLLE flux (Section 2.4.2) on the flat path: one stage within 1e-12
    of the oracle."""
    prob, Pn = _ragged_turbulent(recon=recon, riemann=inputs.FLUX_HLLE)
    dts = 0.25 / 32
    g = _g(prob)
    out = torch.empty_like(_t(Pn, dev))
    g.stage(_t(Pn, dev), _t(Pn, dev), dts, out)
    ref, _, rst, _ = orc.stage(prob, Pn, Pn, dts)
    assert rst.max() == 0
    assert rel_field_err(out.cpu().numpy(), ref).max() < 1e-12
    g.close()


@pytest.mark.parametrize("recon", [inputs.RECON_MC, inputs.RECON_WENO5])
def test_mixed_residual_float_float_faces(dev, orc, recon):
    """The mixed solver evaluates face states and fluxes in float-float
    (about 48 significant bits): its stage residual agrees with the float64
    oracle's to 1e-12 (absolute, scaled rows of order 1e-3)."""
    prob, Pn = _ragged_turbulent(recon=recon)
    rng = np.random.default_rng(2)
    PE = Pn * (1 + 1e-3 * rng.standard_normal(Pn.shape))
    Pk = Pn * (1 + 1e-3 * rng.standard_normal(Pn.shape))
    dts = 0.25 / 32
    g = _g(prob, precision=1)
    R = torch.empty_like(_t(Pn, dev))
    g.residual(_t(Pn, dev), _t(PE, dev), dts, _t(Pk, dev), R)
    ref = orc.residual(prob, Pn, PE, dts, Pk)
    assert np.abs(R.cpu().numpy() - ref).max() < 1e-12
    g.close()


@pytest.mark.parametrize("bscale", [1e-20, 1e-34, 0.0])
def test_mixed_residual_weak_field(dev, orc, bscale):
    """A field far below the float range's square root (b^2 underflows a
    float) or zero: the float-float face states form b-hat from b scaled by
    a power of two, so the mixed solver's residual still agrees with the
    float64 oracle's to 1e-12 (an unscaled b-hat overflowed to ~1e41)."""
    prob, Pn = _ragged_turbulent()
    Pn = Pn.copy()
    Pn[5:8] *= bscale
    rng = np.random.default_rng(3)
    PE = Pn * (1 + 1e-3 * rng.standard_normal(Pn.shape))
    Pk = Pn * (1 + 1e-3 * rng.standard_normal(Pn.shape))
    dts = 0.25 / 32
    g = _g(prob, precision=1)
    R = torch.empty_like(_t(Pn, dev))
    g.residual(_t(Pn, dev), _t(PE, dev), dts, _t(Pk, dev), R)
    ref = orc.residual(prob, Pn, PE, dts, Pk)
    got = R.cpu().numpy()
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() < 1e-12
    g.close()
