"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

    python tests/golden/write_golden.py

feeder13_b8.json: the 13-bus, 8-scenario wye workload (seed 101), solved by
the oracle with tol 1e-8 and max_iter 50 (maximum-step stop rule).
grid14_b4.json: a 14-bus synthetic transmission grid (seed 1), 4 scenarios,
solved by the Newton-Raphson oracle with tol 1e-10 and max_iter 20.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import nr_oracle as NO                # noqa: E402
from oracle import zbus_oracle as O               # noqa: E402
from paper_2605_14103_gb300 import feeders as F   # noqa: E402
from paper_2605_14103_gb300 import grids as G     # noqa: E402


def main():
    f, Sw, Sd, w = F.make_workload("feeder13_b8")
    r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                    tol=w.tol, max_iter=w.max_iter)
    out = {
        "what": "oracle solution of workload feeder13_b8 (13 buses, 8 scenarios, wye loads, seed 101)",
        "tol": w.tol, "max_iter": w.max_iter, "rule": "maxabs",
        "V_re": r["V"].real.round(17).tolist(), "V_im": r["V"].imag.round(17).tolist(),
        "iters": r["iters"].tolist(), "converged": r["converged"].tolist(),
    }
    with open(os.path.join(HERE, "feeder13_b8.json"), "w") as fh:
        json.dump(out, fh, indent=0)
    g = G.make_grid(14, 1)
    P, Q = G.make_injections(g, 4)
    r = NO.solve_batch(g.N, g.Y_row, g.Y_col, g.Y_val, g.bus_type, g.v_set, P, Q, tol=1e-10,
                       max_iter=20)
    out = {
        "what": "Newton-Raphson oracle solution of the 14-bus synthetic grid (seed 1), 4 scenarios",
        "tol": 1e-10, "max_iter": 20,
        "V_re": r["V"].real.round(17).tolist(), "V_im": r["V"].imag.round(17).tolist(),
        "iters": r["iters"].tolist(), "converged": r["converged"].tolist(),
    }
    with open(os.path.join(HERE, "grid14_b4.json"), "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main()
