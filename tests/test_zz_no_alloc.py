"""The allocation-free solve entry point against the regular one.

zbus_solve_noalloc serves callers that cannot allocate device memory while
they solve (their device memory belongs to another allocator, or their loop
forbids allocation after start-up): it keeps its scratch in a static device
array instead.  It launches the same FP64 kernels as zbus_solve, so its
results must equal those of zbus_solve (FP64) bit for bit, on two calls in a
row (the second one reusing the array the first one left behind), over both
stop rules, warm and cold starts, with and without delta loads; one case is
also checked against the FP64 oracle.  The first call must not change the
device's free memory (the array was loaded when the network was created).  A
batch too large for the array, a host array and a partial-phase network must
be refused before anything is launched.

This file is collected last, so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_14103_gb300 import feeders as F   # noqa: E402
from paper_2605_14103_gb300 import zbus           # noqa: E402

pytestmark = pytest.mark.gpu

TOL_V = 1e-6      # parity bar against the FP64 oracle (pu)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    B.build()
    zbus.lib()


@pytest.fixture(scope="module")
def feeder():
    return F.make_feeder(128, 202, delta_frac=0.3, mult_hi=1.5)


def _outs(B, n):
    return (torch.empty((B, n), dtype=torch.complex128, device="cuda"),
            torch.empty((B,), dtype=torch.int32, device="cuda"),
            torch.empty((B,), dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("rule", ["maxabs", "summag"])
@pytest.mark.parametrize("warm", [False, True])
@pytest.mark.parametrize("delta", [True, False])
def test_noalloc_equals_solve_on_two_calls_in_a_row(feeder, rule, warm, delta):
    f = feeder
    net = zbus.Network.from_feeder(f)
    for call, (B, seed) in enumerate([(700, 1), (333, 2)]):
        Sw_h, Sd_h = F.make_scenarios(f, B, 0.5, 1.5, seed=seed)
        Sw = torch.from_numpy(Sw_h).cuda()
        Sd = torch.from_numpy(Sd_h).cuda() if delta else None
        V0 = None
        if warm:   # a warm start near the solution: the no-load voltages scaled down
            _, w = net.get_z()
            V0 = (0.97 * w).expand(B, -1).contiguous()
        V, it, cv = net.solve(Sw, Sd, V_init=V0, tol=1e-8, max_iter=50, rule=rule)
        V2, it2, cv2 = _outs(B, f.n)
        V2.fill_(float("nan"))
        zbus.zbus_solve_noalloc(net.handle, Sw, Sd, V0, 1e-8, 50, rule, V2, it2, cv2)
        torch.cuda.synchronize()
        assert cv2.all(), call
        assert torch.equal(cv2, cv), call
        assert torch.equal(it2, it), call
        assert torch.equal(V2, V), (call, (V2 - V).abs().max().item())
    net.close()


def test_noalloc_matches_the_oracle(feeder):
    from oracle import zbus_oracle as O
    f = feeder
    B = 48
    Sw_h, Sd_h = F.make_scenarios(f, B, 0.5, 1.5, seed=3)
    ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw_h, Sd_h,
                      tol=1e-8, max_iter=50)
    net = zbus.Network.from_feeder(f)
    V, it, cv = _outs(B, f.n)
    zbus.zbus_solve_noalloc(net.handle, torch.from_numpy(Sw_h).cuda(),
                            torch.from_numpy(Sd_h).cuda(), None, 1e-8, 50, "maxabs", V, it, cv)
    torch.cuda.synchronize()
    assert np.array_equal(cv.cpu().numpy(), ref["converged"])
    assert np.array_equal(it.cpu().numpy(), ref["iters"])
    assert float(np.abs(V.cpu().numpy() - ref["V"]).max()) <= TOL_V
    net.close()


def test_noalloc_first_call_changes_no_device_memory(feeder):
    """The static array is loaded by zbus_network_create, not by the call."""
    f = feeder
    net = zbus.Network.from_feeder(f)
    B = 256
    Sw_h, Sd_h = F.make_scenarios(f, B, 0.5, 1.5, seed=4)
    Sw, Sd = torch.from_numpy(Sw_h).cuda(), torch.from_numpy(Sd_h).cuda()
    net.solve(Sw, Sd)           # loads the FP64 kernels both calls launch
    V, it, cv = _outs(B, f.n)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    zbus.zbus_solve_noalloc(net.handle, Sw, Sd, None, 1e-8, 50, "maxabs", V, it, cv)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert cv.all()
    net.close()


def test_noalloc_clears_an_earlier_device_status(feeder):
    """After a mixed solve, the status reported is the FP64 solve's own (OK)."""
    f = feeder
    net = zbus.Network.from_feeder(f)
    B = 128
    Sw_h, Sd_h = F.make_scenarios(f, B, 0.5, 1.5, seed=5)
    Sw, Sd = torch.from_numpy(Sw_h).cuda(), torch.from_numpy(Sd_h).cuda()
    net.solve(Sw, Sd, precision="fp16_scaled")
    torch.cuda.synchronize()
    assert net.device_status() == 0
    V, it, cv = _outs(B, f.n)
    zbus.zbus_solve_noalloc(net.handle, Sw, Sd, None, 1e-8, 50, "maxabs", V, it, cv)
    torch.cuda.synchronize()
    assert net.device_status() == 0
    net.close()


def test_noalloc_refuses_a_batch_beyond_the_array(feeder):
    f = feeder
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
    net.close()


def test_noalloc_refuses_host_arrays(feeder):
    """A host load array through the C ABI: ZBUS_ERR_ARG, nothing launched."""
    f = feeder
    net = zbus.Network.from_feeder(f)
    B = 16
    Sw_host = torch.zeros((B, f.n), dtype=torch.complex128).pin_memory()
    V, it, cv = _outs(B, f.n)
    V.fill_(7.0)
    st = zbus.lib().zbus_solve_noalloc(
        C.c_void_p(net.handle), B, C.c_void_p(Sw_host.data_ptr()), None, None, 1e-8, 50, 0,
        C.c_void_p(V.data_ptr()), C.c_void_p(it.data_ptr()), C.c_void_p(cv.data_ptr()), None)
    assert st == 1
    torch.cuda.synchronize()
    assert (V == 7.0).all()
    net.close()


def test_noalloc_refuses_a_partial_phase_network():
    f = F.make_partial_feeder(30, 11)
    net = zbus.Network.from_feeder(f)
    B = 4
    n = net.n
    z = torch.zeros((B, n), dtype=torch.complex128, device="cuda")
    V, it, cv = _outs(B, n)
    with pytest.raises(zbus.ZbusError) as ei:
        zbus.zbus_solve_noalloc(net.handle, z, None, None, 1e-8, 50, "maxabs", V, it, cv)
    assert ei.value.status == 7            # ZBUS_ERR_UNSUPPORTED
    net.close()
