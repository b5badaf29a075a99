"""Shared helpers for the oracle tests: zone-constant vectors and golden files."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def minkowski_derived(P, gamma):
    """Theta, u^t and u_mu of a primitive vector in Minkowski space (test setup)."""
    v = np.asarray(P[2:5])
    ut = math.sqrt(1.0 + float(v @ v))
    theta = (gamma - 1.0) * P[1] / P[0]
    ucov = np.array([-ut, v[0], v[1], v[2]])
    return theta, ut, ucov


def zone_vector(orc, prob, Pn, PE, dts, divF=None, dTh=None, du=None, divu=0.0):
    """Pack the 80-double zone-constant vector used by the single-zone oracle calls."""
    U, _, _ = orc.point(prob, Pn)
    th, ut, ucov = minkowski_derived(Pn, prob.gamma)
    zc = []
    zc += list(U)
    zc += list(np.zeros(10) if divF is None else divF)
    zc += [0.0] * 10
    zc += list(np.zeros(4) if dTh is None else dTh)
    zc += list(np.zeros(16) if du is None else np.ravel(du))
    zc += [divu, th, ut] + list(ucov) + [Pn[8], Pn[9]]
    zc += list(dts / (np.abs(U) + abs(U[0])))
    zc += [dts] + list(PE)
    zc = np.array(zc, dtype=np.float64)
    assert zc.size == 80
    return zc


def random_zone_state(rng, with_field=True, dissipative=True):
    P = np.zeros(10)
    P[0] = rng.uniform(0.5, 2.0)
    P[1] = rng.uniform(0.5, 3.0)
    P[2:5] = rng.normal(0.0, 0.3, 3)
    if with_field:
        P[5:8] = rng.normal(0.0, 0.3, 3)
    if dissipative:
        P[8:10] = rng.normal(0.0, 0.1, 2)
    return P
