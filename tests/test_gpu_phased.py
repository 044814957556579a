"""Partial-phase feeders on the GPU (single- and two-phase laterals): every
form against the oracle's direct phased solve (flags equal, max |dV| <= 1e-6
pu, iterations within one, FP64 mismatch <= 1e-6), Z and w on the present
phases, host buffers, ignored delta entries, and the calls that refuse such
networks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import zbus_oracle as O                      # noqa: E402
from paper_2605_14103_gb300 import feeders as F          # noqa: E402
from paper_2605_14103_gb300 import zbus                  # noqa: E402

pytestmark = pytest.mark.gpu
FORMS = ["fp64", "fp16_scaled", "bf16x2", "tree"]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    B.build()
    zbus.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def oracle(f, Sw, Sd, **kw):
    return O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                       bus_phase=f.bus_phase, **kw)


@pytest.mark.parametrize("mode", FORMS)
@pytest.mark.parametrize("N,B,lat,delta,seed", [(12, 5, 1.0, 0.5, 3), (60, 70, 0.5, 0.4, 77),
                                                (128, 200, 0.3, 0.3, 202),
                                                (400, 33, 0.4, 0.3, 9)])
def test_parity_against_the_phased_oracle(mode, N, B, lat, delta, seed):
    f = F.make_partial_feeder(N, seed, lateral_frac=lat, delta_frac=delta, mult_hi=1.5)
    Sw, Sd = F.make_partial_scenarios(f, B, 0.5, 1.5)
    ref = oracle(f, Sw, Sd)
    net = zbus.Network.from_feeder(f)
    assert net.n == f.n
    V, it, cv = net.solve(dev(Sw), dev(Sd), precision=mode)
    V, it, cv = V.cpu().numpy(), it.cpu().numpy(), cv.cpu().numpy()
    np.testing.assert_array_equal(cv, ref["converged"])
    m = ref["converged"] == 1
    assert np.abs(V[m] - ref["V"][m]).max() <= 1e-6
    assert np.abs(it[m] - ref["iters"][m]).max() <= 1
    mm = net.power_mismatch(dev(V), dev(Sw), dev(Sd)).cpu().numpy()
    assert mm[m].max() <= 1e-6
    mo = O.power_mismatch(ref["Y_LL"], ref["Y_Ls"], f.v_slack, V, Sw, Sd, ref["bus_phase"])
    np.testing.assert_allclose(mm, mo, rtol=1e-6, atol=1e-12)
    assert net.device_status() == 0


def test_reduced_impedance_on_the_present_phases():
    f = F.make_partial_feeder(50, 13, lateral_frac=0.6)
    ref = oracle(f, np.zeros((1, f.n)), np.zeros((1, f.n)))
    net = zbus.Network.from_feeder(f)
    Z, w = net.get_z()
    np.testing.assert_allclose(Z.cpu().numpy(), ref["Z"], rtol=0,
                               atol=1e-10 * np.abs(ref["Z"]).max())
    np.testing.assert_allclose(w.cpu().numpy(), ref["w"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("mode", ["fp64", "tree"])
def test_host_buffers(mode):
    f = F.make_partial_feeder(128, 202, lateral_frac=0.3, delta_frac=0.3)
    Sw, Sd = F.make_partial_scenarios(f, 3000, 0.8, 1.2)
    net = zbus.Network.from_feeder(f)
    Vd, itd, cvd = net.solve(dev(Sw), dev(Sd), precision=mode)
    Vh, ith, cvh = net.solve(torch.from_numpy(Sw).pin_memory(), torch.from_numpy(Sd).pin_memory(),
                             precision=mode)
    torch.cuda.synchronize()
    assert torch.equal(Vh, Vd.cpu()) and torch.equal(ith, itd.cpu())


def test_delta_entries_without_a_second_phase_are_ignored():
    f = F.make_partial_feeder(80, 21, lateral_frac=0.6, delta_frac=0.4)
    Sw, Sd = F.make_partial_scenarios(f, 8, 0.8, 1.2)
    # the delta slots of partial-phase buses, whose branch lacks its second phase
    bp = f.bus_phase[3:]
    present = set(int(g) for g in f.bus_phase)
    bad = [j for j, g in enumerate(bp) if (3 * (g // 3) + (g % 3 + 1) % 3) not in present]
    assert bad
    junk = Sd.copy()
    junk[:, bad] = 0.7 + 0.2j
    net = zbus.Network.from_feeder(f)
    for mode in ("fp64", "fp16_scaled"):
        a = net.solve(dev(Sw), dev(Sd), precision=mode)[0]
        b = net.solve(dev(Sw), dev(junk), precision=mode)[0]
        assert torch.equal(a, b)


def test_calls_that_take_three_phase_networks_refuse_it():
    f = F.make_partial_feeder(30, 5, lateral_frac=0.5)
    Sw, Sd = F.make_partial_scenarios(f, 4, 0.8, 1.2)
    net = zbus.Network.from_feeder(f)
    with pytest.raises(zbus.ZbusError):
        zbus.solve_batched([net], [(dev(Sw), dev(Sd))], precision="fp16_scaled")
    with pytest.raises(zbus.ZbusError):
        zbus.serve([net], [{"feeder": 0, "S_wye": dev(Sw), "S_delta": dev(Sd), "arrival": 0.0}])


@pytest.mark.parametrize("mode", FORMS)
def test_benchmark_workload_full_batch_sampled(mode):
    """The partial-phase benchmark workload (1024 buses with laterals, 16384
    scenarios) in the launch configuration the bench times: every scenario
    converged with its FP64 mismatch <= 1e-6 pu; 96 sampled scenarios
    against the oracle (flags, |dV| <= 1e-6 pu, iterations within one)."""
    f, Sw, Sd, w = F.make_workload("partial1024_b16384")
    net = zbus.Network.from_feeder(f)
    sw, sd = dev(Sw), dev(Sd)
    V, it, cv = net.solve(sw, sd, tol=w.tol, max_iter=w.max_iter, precision=mode)
    mm = net.power_mismatch(V, sw, sd)
    assert bool((cv == 1).all()) and mm.max().item() <= 1e-6
    pick = np.sort(np.random.default_rng(11).choice(Sw.shape[0], 96, replace=False))
    ref = oracle(f, Sw[pick], Sd[pick], tol=w.tol, max_iter=w.max_iter)
    Vs, its, cvs = V.cpu().numpy()[pick], it.cpu().numpy()[pick], cv.cpu().numpy()[pick]
    np.testing.assert_array_equal(cvs, ref["converged"])
    assert np.abs(Vs - ref["V"]).max() <= 1e-6
    assert np.abs(its - ref["iters"]).max() <= 1
    net.close()
