"""Writes tests/golden/oracle_tiny_step.npz: a whole-cycle regression snapshot of the oracle on
a hand-sized case (10^3 grid, Kerr m=1, a=0.5, three particles, two steps).  Calls only oracle/.

Run from the repository root:  python tests/golden/make_oracle_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle as O  # noqa: E402


def tiny_case(threads=1):
    N = 10
    o = O.Oracle(N, N, N, 1.0, 0.5, 1.0, 0.4, quad_order=2, threads=threads)
    o.init_uniform_field(E=(0.0, 0.01, 0.0), B=(0.0, 0.0, 0.1))
    x4 = np.array([[6.3, 3.2, 7.0], [4.1, 5.9, 2.6], [2.7, 6.4, 5.5], [0.0, 0.0, 0.0]])
    usp = np.array([[0.1, -0.2, 0.05], [0.3, 0.0, -0.1], [-0.05, 0.15, 0.2]])
    o.load_particles(0, -1.0, -0.02, x4, usp, np.array([3, 1, 2]), umode=1)
    o.load_particles(1, 0.05, 0.02, x4[:, ::-1].copy(), usp[:, ::-1].copy(), np.array([10, 11, 12]), umode=1)
    return o


def run():
    o = tiny_case()
    o.step(2)
    d, b, J = o.get_fields()
    out = dict(d=d, b=b, J=J)
    for s in (0, 1):
        x, u, ids = o.get_particles(s)
        out[f"x{s}"], out[f"u{s}"], out[f"id{s}"] = x, u, ids
    return out


if __name__ == "__main__":
    np.savez(os.path.join(HERE, "oracle_tiny_step.npz"), **run())
