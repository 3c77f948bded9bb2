"""Writes the stored expected values under tests/golden/ from the oracle only.

config1_oracle.csv: the first workload (unit-sphere icosphere level 3,
g = x^2 - y^2 + 0.5 z at the vertices with linear interpolation, 256 query
points uniform in the ball of radius 0.9 with seed 1, 64 walks per point,
path length 4, Philox seed 0) through the oracle's double-layer walks
(Sec. 4.1, Table 1): per query the point, the mean and unbiased variance
of the 64 walk values, written with 17 significant digits, the number of
walks with a near-degenerate line, and the exact harmonic solution
x^2 - y^2 + 0.5 z of the smooth problem.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2305_04403_gb300 import inputs as I  # noqa: E402


def config1():
    v, f = I.icosphere(3)
    vd = I.poly_eval(I.POLY_CONFIG1, v).astype(np.float32)
    q = I.ball_queries(256, 0.9, 1)
    r = O.dl_walks(v, f, q, 64, 4, seed=0, mode=O.DATA_VERTEX_P1, vertex_data=vd)
    est, var = O.reduce(r["per_walk"])
    return q, est, var, r["flag"].sum(axis=1), I.poly_eval(I.POLY_CONFIG1, q)


def main():
    q, est, var, flagged, exact = config1()
    path = os.path.join(HERE, "config1_oracle.csv")
    with open(path, "w") as fh:
        fh.write("# oracle double-layer walks, first workload (see make_golden.py)\n")
        fh.write("x,y,z,est,var,flagged,exact\n")
        for i in range(len(q)):
            fh.write(",".join(f"{float(c):.17g}" for c in (*q[i], est[i], var[i])) +
                     f",{int(flagged[i])}," + f"{float(exact[i]):.17g}" + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
