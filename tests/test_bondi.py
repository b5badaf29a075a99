"""Michel accretion (Section 8.2's Bondi test, hydrodynamic part): the exact
steady transonic inflow onto a Schwarzschild black hole (sonic point
r_c = 8, gamma = 4/3), run through the modified Kerr-Schild scheme with its
geometric source.  The flow stays steady to truncation error: the mean
density error in 3 < r < 12 after t = 5 falls with the radial resolution
(4x from 32 to 64 zones on the oracle; 2.5x from 64 to 128 through the CUDA
path, where the limiter and the copy boundary at r = 20 set the rate) and
sits at a few 1e-6.  Then the viscous inflow of the same section: the
pressure anisotropy carried by the flow, against reference profiles from
the steady relaxation ODE along the flow (tests/bondi_viscous.py), with and
without the higher-order term."""
import numpy as np
import pytest

from paper_1702_01106_b300 import inputs
from tests.bondi import bondi_dt, bondi_problem, bondi_state


def _err(prob, P, P0):
    x1, _, _ = inputs.zone_centers(prob)
    r = np.exp(x1[0, 0])
    m = (r > 3) & (r < 12)
    return float(np.mean(np.abs(P[0, 0, 1, m] / P0[0, 0, 1, m] - 1)))


def test_bondi_steady_oracle(orc):
    errs = []
    for n1 in (32, 64):
        prob = bondi_problem(n1)
        P0 = bondi_state(prob)
        P = P0.copy()
        dt = bondi_dt(prob)
        for _ in range(int(round(5.0 / dt))):
            P, _, st, _ = orc.step(prob, P, dt)
            assert st.max() == 0
        errs.append(_err(prob, P, P0))
    assert errs[1] < 5e-5 and errs[0] / errs[1] > 4, errs


@pytest.mark.gpu
def test_bondi_steady_gpu(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_01106_b300.grim import Grim
    from tests.gpu_helpers import rel_field_err
    dev = torch.device("cuda:0")
    errs = []
    for n1 in (64, 128):
        prob = bondi_problem(n1)
        P0 = bondi_state(prob)
        dt = bondi_dt(prob)
        g = Grim(prob)
        a = torch.from_numpy(P0).to(dev)
        for _ in range(int(round(5.0 / dt))):
            g.step(a, a, dt)
        assert g.stats()["failed"] == 0
        g.close()
        errs.append(_err(prob, a.cpu().numpy(), P0))
    assert errs[1] < 5e-6 and errs[0] / errs[1] > 2.5, errs
    # and 20 steps agree with the oracle
    prob = bondi_problem(32, tol=1e-14)
    P0 = bondi_state(prob)
    dt = bondi_dt(prob)
    g = Grim(prob)
    a = torch.from_numpy(P0).to(dev)
    ref = P0
    for _ in range(20):
        g.step(a, a, dt)
        ref, _, _, _ = orc.step(prob, ref, dt)
    assert rel_field_err(a.cpu().numpy(), ref).max() < 1e-11
    g.close()


# ---------------------------------------------------------------- viscous inflow
def _dp_err(prob, P, higher_order):
    """Mean |dP~ - reference| over 3 < r < 12, relative to the reference's
    largest value there."""
    from tests import bondi_viscous as bv
    x1, _, _ = inputs.zone_centers(prob)
    r = np.exp(x1[0, 0])
    m = (r > 3) & (r < 12)
    ref = bv.reference(higher_order).sol(r)[0]
    return float(np.abs(P[9, 0, 1] - ref)[m].mean() / np.abs(ref[m]).max())


def test_viscous_bondi_reference():
    """The reference profile's ingredients: the shear bhat bhat nabla u is
    the same scalar in Boyer-Lindquist and Kerr-Schild coordinates (1e-8);
    the higher-order term changes the profile by order one (so the
    comparisons below can tell it is there); and where tau_R is short the
    profile sits near its Braginskii target."""
    from tests import bondi_viscous as bv
    for r in (2.6, 3.0, 5.0, 7.5, 12.0, 30.0):
        S, _ = bv.shear_bl(r)
        assert abs(bv.shear_ks(r) / S - 1) < 1e-8
    rr = np.array([3.0, 5.0, 8.0])
    ho, plain = bv.reference(True).sol(rr)[0], bv.reference(False).sol(rr)[0]
    assert np.all(np.abs(plain / ho - 1) > 0.2)
    y0 = np.array([bv.target(x)[0] for x in rr])
    assert np.all(np.abs(ho / y0 - 1) < 0.25)


@pytest.mark.parametrize("higher_order", [True, False])
def test_viscous_bondi_oracle(orc, higher_order):
    """Section 8.2's viscous Bondi check on the oracle (feedback of dP on the
    flow negligible, psi = 1e-6; tests/bondi_viscous.py): started on the
    reference profile, after t = 30 the mean error of dP~ in 3 < r < 12
    falls 3x or more from 32 to 64 radial zones and is below 2e-4 of the
    profile, while the profile with the higher-order term toggled is 1e-1
    away."""
    from tests import bondi_viscous as bv
    errs = []
    for n1 in (32, 64):
        prob = bv.viscous_bondi_problem(n1, higher_order)
        P, _ = bv.viscous_bondi_state(prob, higher_order)
        dt = bondi_dt(prob)
        for _ in range(int(round(30.0 / dt))):
            P, _, st, _ = orc.step(prob, P, dt)
            assert st.max() == 0
        errs.append(_dp_err(prob, P, higher_order))
    assert errs[0] > 3 * errs[1] and errs[1] < 2e-4, errs
    assert _dp_err(prob, P, not higher_order) > 0.1


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_viscous_bondi_gpu(orc, precision):
    """The viscous Bondi check through the CUDA path (float64 and mixed, with
    the higher-order term and without): 20 steps of the 32-zone run within
    1e-10 of the oracle (mixed: 1e-9), and after t = 30 the error of dP~
    against the reference falls 3x or more per doubling from 64 to 256
    radial zones."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_01106_b300.grim import Grim
    from tests import bondi_viscous as bv
    from tests.gpu_helpers import rel_field_err
    dev = torch.device("cuda:0")
    prob = bv.viscous_bondi_problem(32, tol=1e-13 if precision == 0 else 1e-12)
    P0, _ = bv.viscous_bondi_state(prob)
    dt = bondi_dt(prob)
    g = Grim(prob, precision=precision)
    a = torch.from_numpy(P0).to(dev)
    ref = P0
    for _ in range(20):
        g.step(a, a, dt)
        ref, _, st, _ = orc.step(prob.with_(tol=1e-13), ref, dt)
        assert st.max() == 0
    assert rel_field_err(a.cpu().numpy(), ref).max() < (1e-10 if precision == 0 else 1e-9)
    g.close()
    for ho in (True, False):
        errs = []
        for n1 in (64, 128, 256):
            prob = bv.viscous_bondi_problem(n1, ho, tol=1e-12)
            P0, _ = bv.viscous_bondi_state(prob, ho)
            dt = bondi_dt(prob)
            g = Grim(prob, precision=precision)
            a = torch.from_numpy(P0).to(dev)
            for _ in range(int(round(30.0 / dt))):
                g.step(a, a, dt)
            assert g.stats()["failed"] == 0
            errs.append(_dp_err(prob, a.cpu().numpy(), ho))
            g.close()
        assert errs[0] > 3 * errs[1] and errs[1] > 3 * errs[2], (ho, errs)
        assert _dp_err(prob, a.cpu().numpy(), not ho) > 0.1
