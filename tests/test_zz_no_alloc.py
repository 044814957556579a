"""The allocation-free solve entry point against the regular one.

zbus_solve_noalloc serves callers that cannot allocate device memory while
they solve (their device memory belongs to another allocator, or their loop
forbids allocation after start-up): it keeps its scratch in a static device
array instead.  Its results must equal those of zbus_solve (FP64) within the
parity tolerance of the other tests, on two calls in a row (the second one
reusing the array the first one left behind), and a batch too large for the
array must be refused before anything is launched.

This file is collected last, so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_14103_gb300 import feeders as F   # noqa: E402
from paper_2605_14103_gb300 import zbus           # noqa: E402

pytestmark = pytest.mark.gpu

TOL_V = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    B.build()
    zbus.lib()


def _outs(B, n):
    return (torch.empty((B, n), dtype=torch.complex128, device="cuda"),
            torch.empty((B,), dtype=torch.int32, device="cuda"),
            torch.empty((B,), dtype=torch.uint8, device="cuda"))


def test_noalloc_matches_solve_on_two_calls_in_a_row():
    f = F.make_feeder(128, 202, delta_frac=0.3, mult_hi=1.5)
    net = zbus.Network.from_feeder(f)
    for call, (B, seed) in enumerate([(700, 1), (333, 2)]):
        Sw_h, Sd_h = F.make_scenarios(f, B, 0.5, 1.5, seed=seed)
        Sw = torch.from_numpy(Sw_h).cuda()
        Sd = torch.from_numpy(Sd_h).cuda()
        V, it, cv = net.solve(Sw, Sd, tol=1e-8, max_iter=50)
        V2, it2, cv2 = _outs(B, f.n)
        zbus.zbus_solve_noalloc(net.handle, Sw, Sd, None, 1e-8, 50, "maxabs", V2, it2, cv2)
        torch.cuda.synchronize()
        assert torch.equal(cv2, cv), call
        assert torch.equal(it2, it), call
        assert cv2.all()
        err = (V2 - V).abs().max().item()
        assert err <= TOL_V, (call, err)


def test_noalloc_refuses_a_batch_beyond_the_array():
    f = F.make_feeder(128, 202, delta_frac=0.3)
    net = zbus.Network.from_feeder(f)
    B = 4096                               # needs ~37 MiB of scratch at n = 381
    z = torch.zeros((B, f.n), dtype=torch.complex128, device="cuda")
    V, it, cv = _outs(B, f.n)
    V.fill_(7.0)
    with pytest.raises(zbus.ZbusError) as ei:
        zbus.zbus_solve_noalloc(net.handle, z, z, None, 1e-8, 50, "maxabs", V, it, cv)
    assert ei.value.status == 1
    assert "static scratch" in str(ei.value)
    torch.cuda.synchronize()
    assert (V == 7.0).all()               # nothing was launched
