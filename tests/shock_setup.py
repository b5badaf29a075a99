"""The steady ideal-MHD shock of Table 2 (Section 8.1.2) as a 1-D run: left
and right states on [-1, 1] with the jump at x = 0, outflow boundaries,
conduction, viscosity and higher-order terms off, gamma = 4/3."""
import numpy as np

from paper_1702_01106_b300 import inputs
from tests.oracle_helpers import read_golden


def shock_problem(n, tol=1e-12):
    return inputs.Problem(dim=2, n=(n, 1, 1), x_start=(-1.0, 0.0, 0.0), x_end=(1.0, 1.0, 1.0),
                          bc=((inputs.BC_OUTFLOW, inputs.BC_OUTFLOW), (inputs.BC_PERIODIC, inputs.BC_PERIODIC),
                              (inputs.BC_PERIODIC, inputs.BC_PERIODIC)),
                          gamma=4.0 / 3.0, conduction=False, viscosity=False, higher_order=False, tol=tol)


def shock_states():
    rows = {r[0]: (float(r[1]), float(r[2])) for r in read_golden("table2_shock_states.txt")}
    names = ["rho", "u", "u1", "u2", "u3", "B1", "B2", "B3"]
    L = np.zeros(10)
    R = np.zeros(10)
    for a, nm in enumerate(names):
        L[a], R[a] = rows[nm]
    return L, R


def shock_state(prob):
    L, R = shock_states()
    n = prob.n[0]
    x = prob.x_start[0] + (np.arange(n) + 0.5) * prob.dx[0]
    return np.where(x[None, :] < 0, L[:, None], R[:, None]).reshape(10, 1, 1, n), x


def shock_position(rho, x, L, R):
    """Where rho crosses the mean of the two states (linear interpolation)."""
    mid = 0.5 * (L[0] + R[0])
    k = int(np.argmax(rho > mid))
    return x[k - 1] + (mid - rho[k - 1]) / (rho[k] - rho[k - 1]) * (x[k] - x[k - 1])
