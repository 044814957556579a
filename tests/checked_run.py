"""Child process of tests/test_gpu_checked.py: runs small and odd sizes of
every form through the library the environment names (ZBUS_LIB, the checked
build) and checks that no index check fired and the results match the
oracles.  Prints "checked ok" on success."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import nr_oracle as NO                       # noqa: E402
from oracle import zbus_oracle as O                      # noqa: E402
from paper_2605_14103_gb300 import feeders as F          # noqa: E402
from paper_2605_14103_gb300 import grids as Gr           # noqa: E402
from paper_2605_14103_gb300 import zbus                  # noqa: E402


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def main():
    flag, word = zbus.zbus_checked_status()
    assert flag == 1, "not the checked build"
    assert word == 0, hex(word)
    # Z-bus forms: one bus (n = 3), 13 and 60 buses; odd batches
    for N, seed in ((2, 1), (13, 101), (60, 7)):
        f = F.make_feeder(N, seed, delta_frac=0.4)
        net = zbus.Network.from_feeder(f)
        for B in (1, 7, 129):
            Sw, Sd = F.make_scenarios(f, B, 0.8, 1.2, seed=seed + B)
            ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw,
                              Sd)
            for form in ("fp64", "fp16_scaled", "bf16x2", "tree"):
                V, it, cv = net.solve(dev(Sw), dev(Sd), precision=form)
                torch.cuda.synchronize()
                assert np.array_equal(cv.cpu().numpy(), ref["converged"]), (N, B, form)
                m = ref["converged"] == 1
                assert np.abs(V.cpu().numpy()[m] - ref["V"][m]).max() <= 1e-6, (N, B, form)
            mm = net.power_mismatch(V, dev(Sw), dev(Sd)).cpu().numpy()
            assert mm[m].max(initial=0.0) <= 1e-6
        # load gradient, both forms
        Sw, Sd = F.make_scenarios(f, 7, 0.8, 1.2)
        r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                        tol=1e-14, max_iter=300)
        G = np.random.default_rng(N).normal(size=Sw.shape) * (1 - 0.5j)
        Hw, Hd = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G)
        for form in ("fp64", "tree"):
            dw, dd, ait, acv = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd),
                                                 tol=1e-13, precision=form)
            assert acv.cpu().numpy().all()
            assert np.abs(dw.cpu().numpy() - Hw).max() <= 1e-9 * np.abs(Hw).max(), form
            assert np.abs(dd.cpu().numpy() - Hd).max() <= 1e-9 * np.abs(Hd).max(), form
        net.close()
    # partial-phase feeder, every form
    f = F.make_partial_feeder(30, 5, lateral_frac=0.8, delta_frac=0.5)
    Sw, Sd = F.make_partial_scenarios(f, 9, 0.8, 1.2)
    ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                      bus_phase=f.bus_phase)
    net = zbus.Network.from_feeder(f)
    for form in ("fp64", "fp16_scaled", "bf16x2", "tree"):
        V, it, cv = net.solve(dev(Sw), dev(Sd), precision=form)
        torch.cuda.synchronize()
        assert np.array_equal(cv.cpu().numpy(), ref["converged"]), form
        assert np.abs(V.cpu().numpy() - ref["V"]).max() <= 1e-6, form
    # two feeders in one batched solve
    fa, fb = F.make_feeder(20, 3, delta_frac=0.3), F.make_feeder(45, 4, delta_frac=0.3)
    loads = [tuple(dev(x) for x in F.make_scenarios(fx, B, 0.8, 1.2)) for fx, B in ((fa, 33),
                                                                                      (fb, 5))]
    outs = zbus.solve_batched([zbus.Network.from_feeder(fa), zbus.Network.from_feeder(fb)],
                              loads, precision="fp16_scaled")
    for (V, it, cv) in outs:
        assert cv.cpu().numpy().all()
    # Newton-Raphson, both arithmetic forms, odd batches
    g = Gr.make_grid(30, 2)
    nnet = zbus.NrNetwork.from_grid(g)
    for B in (1, 7):
        P, Q = Gr.make_injections(g, B, seed=B)
        ref = NO.solve_batch(g.N, g.Y_row, g.Y_col, g.Y_val, g.bus_type, g.v_set, P, Q)
        for prec in ("fp64", "mixed"):
            V, it, cv, gm = nnet.solve(dev(P), dev(Q), precision=prec)
            torch.cuda.synchronize()
            assert np.array_equal(cv.cpu().numpy(), ref["converged"]), prec
            assert np.abs(V.cpu().numpy() - ref["V"]).max() <= 1e-8, prec
    flag, word = zbus.zbus_checked_status()
    assert word == 0, f"an index check fired: {word:#x}"
    print("checked ok")


if __name__ == "__main__":
    main()
