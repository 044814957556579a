"""Child process of tests/test_gpu_checked.py: makes the tensor-core pipeline
give up without a fault, through the library the environment names
(ZBUS_LIB, the checked build, whose wait limit zbus_checked_set_wait can
lower), and checks that the failure is reported and that the same process
then solves normally.

With the limit at 0 a pipeline wait that is not complete at its first test
gives up (the epilogue's first wait for an accumulator always is not): the
kernel records the code, waits for the MMAs and TMA loads it already issued,
frees its tensor memory and the sweep loop ends.  Prints "giveup ok" on
success."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import zbus_oracle as O                      # noqa: E402
from paper_2605_14103_gb300 import feeders as F          # noqa: E402
from paper_2605_14103_gb300 import zbus                  # noqa: E402

ZBUS_ERR_TIMEOUT = 5


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def solve_and_check(net, f, Sw, Sd, ref, form):
    V, it, cv = net.solve(dev(Sw), dev(Sd), precision=form)
    torch.cuda.synchronize()
    assert net.device_status() == 0, form
    assert np.array_equal(cv.cpu().numpy(), ref["converged"]), form
    m = ref["converged"] == 1
    assert np.abs(V.cpu().numpy()[m] - ref["V"][m]).max() <= 1e-6, form


def main():
    flag, word = zbus.zbus_checked_status()
    assert flag == 1, "not the checked build"
    f = F.make_feeder(128, 202, delta_frac=0.3, mult_hi=1.5)
    Sw, Sd = F.make_scenarios(f, 300, 0.5, 1.5, seed=9)
    ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd)
    net = zbus.Network.from_feeder(f)
    for form in ("fp16_scaled", "bf16x2"):
        solve_and_check(net, f, Sw, Sd, ref, form)
        zbus._check(zbus.lib().zbus_checked_set_wait(0))
        try:
            net.solve(dev(Sw), dev(Sd), precision=form)
            torch.cuda.synchronize()
            st = net.device_status()
        finally:
            zbus._check(zbus.lib().zbus_checked_set_wait(2000000000))
        assert st == ZBUS_ERR_TIMEOUT, (form, st)
        # the context is usable and the next ordinary solve is right
        solve_and_check(net, f, Sw, Sd, ref, form)
    flag, word = zbus.zbus_checked_status()
    assert word == 0, hex(word)
    net.close()
    print("giveup ok")


if __name__ == "__main__":
    main()
