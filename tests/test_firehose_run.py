"""Firehose instability (Section 8.1.4) through the full nonlinear scheme:
the printed setup (with B^2 = B cos(2 pi x^1), the reading that keeps
div B = 0) grows at the rate of linear theory, Gamma = 0.10367 (the printed
0.1036 truncated).  The oracle on a coarse grid, the CUDA path on finer
grids (the error of the fitted rate falls with resolution)."""
import math

import numpy as np
import pytest

from paper_1702_01106_b300 import inputs

GAMMA_LINEAR = 0.10367   # the dispersion relation's root (test_oracle_pins.test_firehose_growth_rate)


def firehose(n, alpha=1e-4):
    prob = inputs.Problem(dim=2, n=(n, 1, 1), tau_R=1e6, gamma=4.0 / 3.0, phi=1.0, psi=1.0, tol=1e-12)
    x = (np.arange(n) + 0.5) / n
    rho, u, g = 1.0, 2.0, prob.gamma
    pg = (g - 1) * u
    cs = math.sqrt(g * pg / (rho + g * u))
    P = np.zeros((10, 1, 1, n))
    P[0], P[1], P[5] = rho, u, 0.1
    P[3] = 0.1628 * alpha * np.sin(2 * np.pi * x)
    P[6] = 0.9867 * alpha * np.cos(2 * np.pi * x)
    P[9] = -0.011 / (cs * math.sqrt(prob.psi * pg))     # dP = -0.011 in the rescaled variable
    return prob, P, x


def fitted_rate(T, A, t0=0.5):
    T, A = np.asarray(T), np.abs(np.asarray(A))
    m = T > t0
    return np.polyfit(T[m], np.log(A[m]), 1)[0]


def amplitude(P, x):
    return 2.0 * np.mean(P[3, 0, 0] * np.sin(2 * np.pi * x))


def test_firehose_growth_oracle(orc):
    n = 48
    prob, P, x = firehose(n)
    dt = 0.5 / n
    T, A = [], []
    for s in range(int(2.5 / dt) + 1):
        T.append(s * dt)
        A.append(amplitude(P, x))
        P, _, st, _ = orc.step(prob, P, dt)
        assert st.max() == 0
    assert abs(fitted_rate(T, A) / GAMMA_LINEAR - 1) < 0.02


@pytest.mark.gpu
def test_firehose_growth_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_01106_b300.grim import Grim
    dev = torch.device("cuda:0")
    errs = []
    for n in (64, 128):
        prob, P, x = firehose(n)
        dt = 0.5 / n
        g = Grim(prob)
        a = torch.from_numpy(P).to(dev)
        T, A = [], []
        for s in range(int(3.0 / dt) + 1):
            T.append(s * dt)
            A.append(amplitude(a.cpu().numpy(), x))
            g.step(a, a, dt)
        assert g.stats()["failed"] == 0
        g.close()
        errs.append(abs(fitted_rate(T, A) / GAMMA_LINEAR - 1))
    assert errs[1] < 0.005 and errs[1] < errs[0], errs
