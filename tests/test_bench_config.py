"""The benchmark's two arms describe the same workload.

The reference arm (the FP64 oracle on the host cores) must print the same
`config` as the solver's line, so that the two lines compare like with like.
Both build it with bench.feeder_config; this runs the reference arm on a
small workload (CPU only) and checks its line against that function's
result for the solver's default batch.
"""
import argparse
import contextlib
import io
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench                                             # noqa: E402
from paper_2605_14103_gb300 import feeders as F          # noqa: E402


def test_reference_arm_prints_the_solver_config(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    args = argparse.Namespace(impl="reference", workload="feeder13_b8", precision="fp16_scaled",
                              steps=1, warmup=0)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    f, Sw, _, wl = F.make_workload("feeder13_b8")
    expect = bench.feeder_config("feeder13_b8", wl, Sw.shape[1], wl.B, "fp16_scaled", 1)
    assert line["impl"] == "reference"
    assert line["config"] == expect
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
