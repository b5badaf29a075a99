"""Magneto-thermal instability (Section 9.1) through the CUDA path, checked
against the linear theory the paper cites (tests/mti.py has the setup and
the theory), and the setup itself checked on the CPU."""
import numpy as np
import pytest

from tests import mti


def test_equilibrium_closed_form_and_ode_agree():
    r = np.linspace(mti.R_IN, mti.R_OUT, 21)
    assert np.abs(mti.theta_of_r(r) / mti.theta_ode(r) - 1.0).max() < 1e-11


def test_linear_theory_gives_the_papers_dynamical_time():
    """The fastest local growth time 1/sigma at r = 200 is the paper's
    "dynamical time scale ~2500 M" there (Section 9.1, caption of the MTI
    growth figure); the temperature falls outwards while the entropy rises
    (unstable to the MTI, stable to convection)."""
    assert abs(1.0 / float(mti.growth_rate(200.0)) / 2500.0 - 1.0) < 0.05
    r = np.linspace(mti.R_IN, mti.R_OUT, 11)
    th = mti.theta_of_r(r)
    rho = (th / mti.K_POLY) ** (1.0 / (mti.G_POLY - 1.0))
    entropy = np.log(rho * th / rho ** mti.GAMMA)
    assert np.all(np.diff(th) < 0) and np.all(np.diff(entropy) > 0)
    # the library's tau_R = tau_0 r^(3/2) follows R / c_s over the domain
    ratio = mti.tau0() * r ** 1.5 / (r / mti.sound_speed(r))
    assert np.abs(ratio - 1.0).max() < 0.05


def _run(prob, dev, t_end, sample=500.0):
    """Steps from the seeded equilibrium with the outer radial layers held;
    returns the sample times, the rms radial field and the statistics."""
    torch = pytest.importorskip("torch")
    from paper_1702_01106_b300.grim import Grim
    P, r, _ = mti.mti_state(prob)
    dt = mti.mti_dt(prob)
    g = Grim(prob)
    g.use_graphs(True)
    a = torch.from_numpy(P).to(dev)
    b = torch.empty_like(a)
    eq = torch.from_numpy(mti.equilibrium(prob)).to(dev)
    every = max(1, int(sample / dt))
    times, brms = [], []
    for n in range(int(t_end / dt) + 1):
        if n % every == 0:
            times.append(n * dt)
            brms.append(mti.radial_field_rms(a.cpu().numpy(), r))
        g.step(a, b, dt)
        a, b = b, a
        mti.hold_boundaries(a, eq)
    s = g.stats()
    g.close()
    return np.array(times), np.array(brms), s


def _rate(t, b, t0, t1):
    m = (t >= t0) & (t <= t1)
    return np.polyfit(t[m], np.log(b[m]), 1)[0]


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.gpu
def test_mti_grows_at_the_linear_rate(dev):
    """64 x 4 x 256 zones (r, theta band, phi in [0, pi]), float64, to
    t = 24 000 M.  After the seeded transient the radial field grows
    exponentially: the rates over 15 000-19 500 M and 19 500-24 000 M agree
    to 15 %, over two e-folds.  The rate lies between the slowest and the
    fastest local rate of linear theory on the domain (r = 300: 4.3e3 M;
    r = 200: 2.5e3 M), as a global mode pinned by the held layers must.
    Measured: about 4.0e3 M (the paper fits 2.4e3 M at 128 zones in each
    of r, theta and phi; the rate here rises with the azimuthal resolution,
    from 4.4e3 M at 128 zones in phi)."""
    prob = mti.mti_problem(n1=64, n3=256)
    t, b, s = _run(prob, dev, 24000.0)
    assert s["failed"] == 0 and s["max_res"] <= prob.tol
    s1, s2 = _rate(t, b, 15000.0, 19500.0), _rate(t, b, 19500.0, 24000.0)
    assert abs(s1 / s2 - 1.0) < 0.15, (s1, s2)
    sigma = _rate(t, b, 15000.0, 24000.0)
    assert b[-1] > 5.0 * b[t >= 15000.0][0]                 # at least e^1.6 in the window
    assert float(mti.growth_rate(mti.R_OUT)) < sigma < float(mti.growth_rate(mti.R_IN)), 1.0 / sigma


@pytest.mark.gpu
def test_mti_needs_conduction(dev):
    """The same atmosphere with conduction off is Schwarzschild-stable: the
    radial field does not grow exponentially (over 15 000-24 000 M its rate
    stays below a quarter of the slowest local MTI rate)."""
    prob = mti.mti_problem(n1=64, n3=128).with_(conduction=False)
    t, b, s = _run(prob, dev, 24000.0)
    assert s["failed"] == 0
    assert _rate(t, b, 15000.0, 24000.0) < 0.25 * float(mti.growth_rate(mti.R_OUT))
