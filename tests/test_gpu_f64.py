"""GPU parity of the plain FP64 path against the FP64 oracle, through the C ABI.

Bar (per scenario): converged flags identical, iteration counts identical,
max |V_gpu - V_oracle| <= 1e-6 pu on converged scenarios, and FP64 power
mismatch <= 1e-6 pu.  Both sides compute in FP64 with different summation
orders, so the expected difference is ~1e-13; a tighter 1e-10 check catches
subtle errors well below the stated bar.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import zbus_oracle as O                      # noqa: E402
from paper_2605_14103_gb300 import feeders as F          # noqa: E402
from paper_2605_14103_gb300 import zbus                  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_V = 1e-6
TOL_TIGHT = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    B.build()
    zbus.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def oracle(f, Sw, Sd, tol=1e-8, max_iter=50, rule="maxabs", V0=None):
    return O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                       tol=tol, max_iter=max_iter, rule=rule, V0=V0)


def compare(V, it, cv, ref, tight=True):
    V, it, cv = V.cpu().numpy(), it.cpu().numpy(), cv.cpu().numpy()
    np.testing.assert_array_equal(cv, ref["converged"])
    np.testing.assert_array_equal(it, ref["iters"])
    m = ref["converged"] == 1
    err = np.abs(V[m] - ref["V"][m]).max() if m.any() else 0.0
    assert err <= TOL_V
    if tight:
        assert err <= TOL_TIGHT, err
    return err


@pytest.mark.parametrize("N,seed", [(2, 5), (13, 101), (128, 202)])
def test_device_Z_matches_oracle(N, seed):
    f = F.make_feeder(N, seed, delta_frac=0.3)
    net = zbus.Network.from_feeder(f)
    Z, w = net.get_z()
    ref = oracle(f, *F.make_scenarios(f, 1, 0.8, 1.2))
    Zr = ref["Z"]
    np.testing.assert_allclose(Z.cpu().numpy(), Zr, rtol=0, atol=1e-11 * np.abs(Zr).max())
    # series-only feeder: w equals the slack voltage on every bus
    np.testing.assert_allclose(w.cpu().numpy(), np.tile(f.v_slack, N - 1), atol=1e-10)


def test_device_Z_lca_closed_form():
    from tests.test_oracle_pins import lca_impedance
    f = F.make_feeder(30, 9)
    net = zbus.Network.from_feeder(f)
    Z, _ = net.get_z()
    Zl = lca_impedance(f)
    np.testing.assert_allclose(Z.cpu().numpy(), Zl, rtol=0, atol=1e-11 * np.abs(Zl).max())


def test_golden_feeder13():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "feeder13_b8.json")))
    f, Sw, Sd, w = F.make_workload("feeder13_b8")
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=g["tol"], max_iter=g["max_iter"])
    ref = dict(V=np.array(g["V_re"]) + 1j * np.array(g["V_im"]), iters=np.array(g["iters"]),
               converged=np.array(g["converged"]))
    compare(V, it, cv, ref)


@pytest.mark.parametrize("N,B,delta,seed", [(13, 8, 0.4, 101), (17, 1, 0.5, 3),
                                             (40, 7, 0.3, 4), (128, 129, 0.3, 202),
                                             (128, 512, 0.3, 202), (65, 33, 1.0, 8)])
def test_solve_parity(N, B, delta, seed):
    f = F.make_feeder(N, seed, delta_frac=delta, mult_hi=1.5)
    Sw, Sd = F.make_scenarios(f, B, 0.5, 1.5)
    ref = oracle(f, Sw, Sd)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=1e-8, max_iter=50)
    compare(V, it, cv, ref)
    mm = net.power_mismatch(V, dev(Sw), dev(Sd)).cpu().numpy()
    assert mm.max() <= 1e-6


def test_summag_rule_parity():
    f = F.make_feeder(60, 12, delta_frac=0.3)
    Sw, Sd = F.make_scenarios(f, 40, 0.8, 1.2)
    ref = oracle(f, Sw, Sd, tol=1e-9, rule="summag")
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=1e-9, rule="summag")
    compare(V, it, cv, ref)


def test_wye_only_and_delta_only_pointers():
    f = F.make_feeder(20, 13, delta_frac=0.5)
    Sw, Sd = F.make_scenarios(f, 6, 0.8, 1.2)
    net = zbus.Network.from_feeder(f)
    z = np.zeros_like(Sw)
    for a, b in ((Sw, None), (None, Sd)):
        ref = oracle(f, a if a is not None else z, b if b is not None else z)
        V, it, cv = net.solve(dev(a) if a is not None else None, dev(b) if b is not None else None)
        compare(V, it, cv, ref)


def test_warm_start_and_aliasing():
    f = F.make_feeder(50, 14, delta_frac=0.3)
    Sw, Sd = F.make_scenarios(f, 16, 0.8, 1.2)
    V0 = oracle(f, Sw * 0.9, Sd * 0.9)["V"]
    ref = oracle(f, Sw, Sd, V0=V0)
    net = zbus.Network.from_feeder(f)
    Vt = dev(V0)
    it = torch.empty(16, dtype=torch.int32, device="cuda")
    cv = torch.empty(16, dtype=torch.uint8, device="cuda")
    net.solve(dev(Sw), dev(Sd), V_init=Vt, out=(Vt, it, cv))   # V_out aliases V_init
    compare(Vt, it, cv, ref)


def test_zero_load_gives_no_load_voltage():
    f = F.make_feeder(30, 15, delta_frac=0.3)
    z = np.zeros((5, f.n), dtype=np.complex128)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(z), dev(z))
    _, w = net.get_z()
    assert (it.cpu().numpy() == 1).all() and (cv.cpu().numpy() == 1).all()
    assert torch.equal(V, w.expand(5, -1))


def test_divergence_flags_and_cap():
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=6)
    Sw = Sw * 60.0
    Sd = Sd * 60.0
    Sw[0] /= 60.0
    Sd[0] /= 60.0
    ref = oracle(f, Sw, Sd, max_iter=40)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), max_iter=40)
    np.testing.assert_array_equal(cv.cpu().numpy(), ref["converged"])
    np.testing.assert_array_equal(it.cpu().numpy(), ref["iters"])
    assert cv.cpu().numpy()[0] == 1 and not cv.cpu().numpy()[1:].any()


def test_scenario_results_do_not_depend_on_the_batch():
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=300)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd))
    perm = np.random.default_rng(0).permutation(300)[:77]
    V2, it2, cv2 = net.solve(dev(Sw[perm]), dev(Sd[perm]))
    assert torch.equal(V2, V[torch.from_numpy(perm).cuda()])          # bitwise
    assert torch.equal(it2, it[torch.from_numpy(perm).cuda()])


def test_repeat_calls_and_batch_growth():
    f = F.make_feeder(30, 16, delta_frac=0.3)
    net = zbus.Network.from_feeder(f)
    for B in (3, 64, 5, 200, 64):
        Sw, Sd = F.make_scenarios(f, B, 0.8, 1.2, seed=B)
        V, it, cv = net.solve(dev(Sw), dev(Sd))
        compare(V, it, cv, oracle(f, Sw, Sd))


def test_max_iter_one_and_zero_batch():
    f = F.make_feeder(20, 17, delta_frac=0.3)
    Sw, Sd = F.make_scenarios(f, 4, 0.8, 1.2)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), max_iter=1)
    compare(V, it, cv, oracle(f, Sw, Sd, max_iter=1))
    e = torch.empty((0, f.n), dtype=torch.complex128, device="cuda")
    net.solve(e, e)


def test_singular_network_is_reported():
    # bus 2 is connected to nothing: Y_LL has an all-zero block
    f = F.make_feeder(3, 18)
    keep = (f.Y_row < 6) & (f.Y_col < 6)
    row = np.concatenate([f.Y_row[keep], [6]])
    col = np.concatenate([f.Y_col[keep], [6]])
    val = np.concatenate([f.Y_val[keep], [1.0 + 0j]])
    with pytest.raises(zbus.ZbusError) as ei:
        zbus.Network(f.n_total, row, col, val, f.slack_idx, f.v_slack)
    assert ei.value.status == 2


def test_power_mismatch_matches_oracle():
    f = F.make_feeder(40, 19, delta_frac=0.5)
    Sw, Sd = F.make_scenarios(f, 10, 0.8, 1.2)
    ref = oracle(f, Sw, Sd, tol=1e-3)           # loosely converged: mismatch well above 0
    net = zbus.Network.from_feeder(f)
    got = net.power_mismatch(dev(ref["V"]), dev(Sw), dev(Sd)).cpu().numpy()
    want = O.power_mismatch(ref["Y_LL"], ref["Y_Ls"], f.v_slack, ref["V"], Sw, Sd)
    # r = Y v + ys - i(v) cancels terms of size ~1e3 down to ~1e-5, so both sides
    # carry ~1e-16 * 1e3 absolute rounding in r: compare with that scale
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-12)


def test_full_size_128bus_4096_scenarios_sampled():
    """The benchmark's workload in its launch configuration; the oracle checks a sample."""
    f, Sw, Sd, w = F.make_workload("feeder128_b4096")
    net = zbus.Network.from_feeder(f)
    net.reserve(w.B)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=w.tol, max_iter=w.max_iter)
    mm = net.power_mismatch(V, dev(Sw), dev(Sd)).cpu().numpy()
    assert cv.cpu().numpy().all()
    assert mm.max() <= 1e-6
    idx = np.random.default_rng(1).choice(w.B, 96, replace=False)
    ref = oracle(f, Sw[idx], Sd[idx], tol=w.tol, max_iter=w.max_iter)
    compare(V[torch.from_numpy(idx).cuda()], it[torch.from_numpy(idx).cuda()],
            cv[torch.from_numpy(idx).cuda()], ref)


def test_1024bus_small_batch():
    f, Sw, Sd, w = F.make_workload("feeder1024_b16384", B=24)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=w.tol, max_iter=w.max_iter)
    ref = oracle(f, Sw, Sd, tol=w.tol, max_iter=w.max_iter)
    compare(V, it, cv, ref, tight=False)
    assert np.abs(V.cpu().numpy() - ref["V"]).max() <= 1e-9


def _bits(V):
    """Bit patterns of a complex128 tensor (NaNs compare equal by their bits)."""
    return V.view(torch.float64).view(torch.int64)


@pytest.mark.parametrize("N,B,delta,seed", [(2, 1, 0.0, 5), (13, 8, 0.4, 101), (25, 32, 0.5, 7),
                                             (33, 17, 1.0, 9)])
def test_one_launch_solve_equals_the_sweep_per_launch_path(N, B, delta, seed):
    """Feeders of at most 96 padded unknowns with at most 32 scenarios solve in
    one launch (a block per scenario runs every sweep); the profile mode
    launches the sweep kernels one by one.  Both give the same bits
    (voltages, counts, flags) under both stop rules, cold and warm, with
    scenarios that diverge and with the iteration cap reached; the one-launch
    results also match the oracle."""
    f = F.make_feeder(N, seed, delta_frac=delta, mult_hi=1.5)
    Sw, Sd = F.make_scenarios(f, B, 0.5, 1.5)
    if B > 2:   # one scenario far beyond what the feeder can carry
        Sw[1] *= 500.0
        Sd[1] *= 500.0
    net = zbus.Network.from_feeder(f)
    for rule in ("maxabs", "summag"):
        for tol, max_iter in ((1e-8, 50), (1e-13, 3)):
            kw = dict(tol=tol, max_iter=max_iter, rule=rule)
            V1, it1, cv1 = net.solve(dev(Sw), dev(Sd), **kw)
            V2, it2, cv2 = net.solve(dev(Sw), dev(Sd), profile=True, **kw)
            assert torch.equal(_bits(V1), _bits(V2))
            assert torch.equal(it1, it2) and torch.equal(cv1, cv2)
            if max_iter == 50:
                compare(V1, it1, cv1, oracle(f, Sw, Sd, tol=tol, rule=rule), tight=False)
            # warm start from a perturbed solution, the output aliasing the start
            V0 = V1 * (1.0 - 1e-3)
            Va = V0.clone()
            ita = torch.empty_like(it1)
            cva = torch.empty_like(cv1)
            net.solve(dev(Sw), dev(Sd), V_init=Va, out=(Va, ita, cva), **kw)
            Vb, itb, cvb = net.solve(dev(Sw), dev(Sd), V_init=V0, profile=True, **kw)
            assert torch.equal(_bits(Va), _bits(Vb))
            assert torch.equal(ita, itb) and torch.equal(cva, cvb)
    # wye-only and delta-only pointers
    for a, b in ((Sw, None), (None, Sd)):
        args = (dev(a) if a is not None else None, dev(b) if b is not None else None)
        V1, it1, cv1 = net.solve(*args)
        V2, it2, cv2 = net.solve(*args, profile=True)
        assert torch.equal(_bits(V1), _bits(V2))
        assert torch.equal(it1, it2) and torch.equal(cv1, cv2)
