"""Write tests/golden/flop_count.json: operations per particle-step of the counted restatement
of the method (oracle/flop_count.py) by Gauss-Legendre order Q of Eq. 18, on the sample particles
of tests/test_flop_count.py.  Calls only oracle/ code.

    python tests/golden/make_flop_count.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from oracle import flop_count as FC  # noqa: E402
from test_flop_count import _setup  # noqa: E402


def main():
    n, m, a, d, b, pts, rng = _setup()
    fields = list(d) + list(b)
    out = {}
    for Q in (1, 2, 3):
        run = FC.Run((n, n, n), m, a, 1.0, 0.4, Q)
        counts = []
        for x in pts:
            u = O.solve_u4(x - (n - 1) / 2.0, m, a, 1.0, rng.normal(0, 0.3, 3), 2)
            counts.append(FC.count_step(run, fields, np.r_[x, 0.0], u, -1.0, 0.01)[0])
        out[str(Q)] = int(round(float(np.mean(counts))))
    with open(os.path.join(HERE, "flop_count.json"), "w") as fh:
        json.dump({"ops_per_particle_step": out,
                   "convention": "add, subtract, multiply, divide, square root = 1 each (FMA = 2); "
                                 "per particle-step of the push + deposit at Q x Q Gauss-Legendre (Eq. 18)",
                   "source": "oracle/flop_count.py via tests/golden/make_flop_count.py"}, fh, indent=1)
        fh.write("\n")
    print(out)


if __name__ == "__main__":
    main()
