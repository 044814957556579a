"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

    python tests/golden/write_golden.py

feeder13_b8.json: the 13-bus, 8-scenario wye workload (seed 101), solved by
the oracle with tol 1e-8 and max_iter 50 (maximum-step stop rule).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import zbus_oracle as O               # noqa: E402
from paper_2605_14103_gb300 import feeders as F   # noqa: E402


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


if __name__ == "__main__":
    main()
