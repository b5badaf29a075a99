"""Write tests/golden/flop_counts.txt: algorithmic flops per unit of work,
counted by the oracle's flop-counting scalar (one flop per +, -, *, /, sqrt;
a*b + c is two; operations on zone constants are hoisted and not counted;
multiplying by a constant 0 or +-1 is not counted).  Run from the repo root:
    python tests/golden/make_flop_counts.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1702_01106_b300 import inputs  # noqa: E402
from tests.oracle_helpers import zone_vector  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flop_counts.txt")


def counts():
    prob = inputs.turbulent_box_problem(64)
    P = inputs.turbulent_box_state(prob).reshape(10, -1)
    rng = np.random.default_rng(0)
    Pn = P[:, 1000].copy()
    Pn[8:10] = 1e-3 * rng.standard_normal(2)       # a zone with heat flux and anisotropy
    zc = zone_vector(oracle, prob, Pn, Pn, 0.25 / 1024, divu=0.01)
    res, lu, book, lu7 = oracle.flop_counts(prob, zc, Pn * 1.001)
    line = np.stack([P[:, 1000 + t] for t in range(-4, 4)])
    line[:, 8:10] = 1e-3
    face, zone = oracle.explicit_flops(prob, line, Pn)
    # bookkeeping with the 7 non-magnetic Jacobian columns: 7 perturbations,
    # 7 divisor differences, 70 residual differences and 70 divisions, the
    # 10 step updates (2 each) and the two norms (20 each)
    book7 = 7 + 7 + 70 + 70 + 20 + 40
    return {"residual": int(res), "lu_solve": int(lu), "newton_update_bookkeeping": int(book),
            "face_flux": int(face), "zone_explicit_remainder_2d": int(zone), "lu_solve_7x7": int(lu7),
            "newton_update_bookkeeping_7x7": book7}


def main():
    c = counts()
    with open(OUT, "w") as f:
        f.write("# Algorithmic flops per unit of work, Minkowski space, conduction, viscosity and\n")
        f.write("# higher-order terms on, MC reconstruction; written by make_flop_counts.py\n")
        f.write("# (oracle flop-counting scalar).  unit flops\n")
        for k, v in c.items():
            f.write(f"{k} {v}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
