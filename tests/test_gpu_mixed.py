"""GPU parity of the defect forms against the FP64 oracle: the mixed-precision
tcgen05 contraction (FP16 row-scaled, BF16 hi+lo) and the tree sweep.

Bar (per scenario): identical converged flags, max |V_gpu - V_oracle| <= 1e-6 pu
on converged scenarios, FP64 power mismatch <= 1e-6 pu, iteration counts
within one of the oracle's.  A single sweep from a warm start isolates the
residual, the tensor-core contraction and the epilogue: its step must match
the FP64 step Z r(v) to the precision of the operands (FP16 row-scaled:
relative 2^-10 of the step size; BF16 hi+lo with BF16 residual: 2^-7; tree
sweep with FP16 branch impedances: 2^-9).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import zbus_oracle as O                      # noqa: E402
from paper_2605_14103_gb300 import feeders as F          # noqa: E402
from paper_2605_14103_gb300 import zbus                  # noqa: E402

pytestmark = pytest.mark.gpu

MODES = ["fp16_scaled", "bf16x2", "tree"]
# the tree sweep applies Z exactly up to its FP16 branch impedances
STEP_RTOL = {"fp16_scaled": 2.0 ** -10, "bf16x2": 2.0 ** -7, "tree": 2.0 ** -9}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    B.build()
    zbus.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def oracle(f, Sw, Sd, tol=1e-8, max_iter=50, V0=None):
    return O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                       tol=tol, max_iter=max_iter, V0=V0)


def check(net, f, Sw, Sd, ref, V, it, cv):
    V, it, cv = V.cpu().numpy(), it.cpu().numpy(), cv.cpu().numpy()
    np.testing.assert_array_equal(cv, ref["converged"])
    m = ref["converged"] == 1
    if m.any():
        err = np.abs(V[m] - ref["V"][m]).max()
        assert err <= 1e-6, err
        assert np.abs(it[m] - ref["iters"][m]).max() <= 1
    mm = net.power_mismatch(dev(V), dev(Sw), dev(Sd)).cpu().numpy()
    assert mm[m].max(initial=0.0) <= 1e-6


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("N,B,seed", [(13, 8, 101), (128, 200, 202), (700, 130, 7)])
def test_one_defect_step_matches_fp64_step(mode, N, B, seed):
    f = F.make_feeder(N, seed, delta_frac=0.3)
    Sw, Sd = F.make_scenarios(f, B, 0.8, 1.2)
    V0 = oracle(f, 0.7 * Sw, 0.7 * Sd)["V"]           # a warm start away from the solution
    ref1 = oracle(f, Sw, Sd, tol=0.0, max_iter=1, V0=V0)["V"]   # v + Z r(v) = Z i(v) + w
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), V_init=dev(V0), tol=0.0, max_iter=1, precision=mode)
    V = V.cpu().numpy()
    step = np.abs(ref1 - V0).max(axis=1, keepdims=True)
    err = np.abs(V - ref1) / step
    assert err.max() <= STEP_RTOL[mode], err.max()
    assert (it.cpu().numpy() == 1).all()


@pytest.mark.parametrize("mode", ["fp16_scaled", "bf16x2"])
@pytest.mark.parametrize("N,B,seed", [(128, 300, 202), (300, 130, 9)])
def test_every_contraction_variant(mode, N, B, seed):
    """Each compiled (N-tile, stages) variant of the tensor-core contraction,
    forced through zbus_tune_set: one defect step against the FP64 step and a
    full solve against the oracle (ragged batches: 300 = 2 x 128 + 44 slots;
    n = 381 and 897 give 12 / 6 / 3 and 28 / 14 / 7 N-tiles of 64 / 128 / 256
    columns)."""
    f = F.make_feeder(N, seed, delta_frac=0.3)
    Sw, Sd = F.make_scenarios(f, B, 0.8, 1.2)
    V0 = oracle(f, 0.7 * Sw, 0.7 * Sd)["V"]
    ref1 = oracle(f, Sw, Sd, tol=0.0, max_iter=1, V0=V0)["V"]
    ref = oracle(f, Sw, Sd)
    net = zbus.Network.from_feeder(f)
    variants = zbus.zbus_tune_variants(mode)
    assert (64, 8 if mode == "fp16_scaled" else 6) in variants and len(variants) >= 4
    step = np.abs(ref1 - V0).max(axis=1, keepdims=True)
    try:
        for bn, st in variants:
            zbus.zbus_tune_set(mode, net.n, B, bn, st)
            V, it, cv = net.solve(dev(Sw), dev(Sd), V_init=dev(V0), tol=0.0, max_iter=1,
                                  precision=mode)
            err = np.abs(V.cpu().numpy() - ref1) / step
            assert err.max() <= STEP_RTOL[mode], (bn, st, err.max())
            V, it, cv = net.solve(dev(Sw), dev(Sd), precision=mode)
            check(net, f, Sw, Sd, ref, V, it, cv)
    finally:
        zbus.zbus_tune_set(mode, net.n, B, 0, 0)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("N,B,delta,seed", [(13, 8, 0.4, 101), (17, 1, 0.5, 3),
                                             (40, 7, 0.3, 4), (128, 129, 0.3, 202),
                                             (128, 512, 0.3, 202), (65, 33, 1.0, 8),
                                             (300, 260, 0.4, 9)])
def test_mixed_solve_parity(mode, N, B, delta, seed):
    f = F.make_feeder(N, seed, delta_frac=delta, mult_hi=1.5)
    Sw, Sd = F.make_scenarios(f, B, 0.5, 1.5)
    ref = oracle(f, Sw, Sd)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=1e-8, max_iter=50, precision=mode)
    check(net, f, Sw, Sd, ref, V, it, cv)


@pytest.mark.parametrize("mode", MODES)
def test_mixed_1024bus(mode):
    f, Sw, Sd, w = F.make_workload("feeder1024_b16384", B=40)
    ref = oracle(f, Sw, Sd)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), precision=mode)
    check(net, f, Sw, Sd, ref, V, it, cv)


@pytest.fixture(scope="module")
def full1024():
    """The 1024-bus workload at its full 16384 scenarios (host arrays) and its
    network; built once for the three forms."""
    f, Sw, Sd, w = F.make_workload("feeder1024_b16384")
    net = zbus.Network.from_feeder(f)
    idx = np.random.default_rng(3).choice(w.B, 256, replace=False)
    ref = oracle(f, Sw[idx], Sd[idx])
    Swd, Sdd = dev(Sw), dev(Sd)
    # the plain FP64 method on every scenario (itself oracle-checked on the sample)
    V64, it64, cv64 = net.solve(Swd, Sdd, tol=w.tol, max_iter=w.max_iter, precision="fp64")
    check(net, f, Sw[idx], Sd[idx], ref, V64[torch.from_numpy(idx).cuda()].contiguous(),
          it64[torch.from_numpy(idx).cuda()].contiguous(),
          cv64[torch.from_numpy(idx).cuda()].contiguous())
    return f, Sw, Sd, w, net, Swd, Sdd, idx, ref, V64


@pytest.mark.parametrize("mode", MODES)
def test_mixed_full_size_1024bus_sampled(mode, full1024):
    """1024 buses x 16384 scenarios in the launch configuration the benchmark
    times: every scenario converged with FP64 mismatch <= 1e-6 and within
    1e-6 pu of the plain FP64 method, and the oracle checks a sample of 256
    scenarios one by one."""
    f, Sw, Sd, w, net, Swd, Sdd, idx, ref, V64 = full1024
    net.reserve(w.B, mode)
    V, it, cv = net.solve(Swd, Sdd, tol=w.tol, max_iter=w.max_iter, precision=mode)
    assert cv.cpu().numpy().all()
    mm = net.power_mismatch(V, Swd, Sdd).cpu().numpy()
    assert mm.max() <= 1e-6
    assert (V - V64).abs().max().item() <= 1e-6
    ti = torch.from_numpy(idx).cuda()
    check(net, f, Sw[idx], Sd[idx], ref, V[ti].contiguous(), it[ti].contiguous(),
          cv[ti].contiguous())


@pytest.mark.parametrize("mode", MODES)
def test_mixed_full_size_128bus_sampled(mode):
    f, Sw, Sd, w = F.make_workload("feeder128_b4096")
    net = zbus.Network.from_feeder(f)
    net.reserve(w.B, mode)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=w.tol, max_iter=w.max_iter, precision=mode)
    assert cv.cpu().numpy().all()
    mm = net.power_mismatch(V, dev(Sw), dev(Sd)).cpu().numpy()
    assert mm.max() <= 1e-6
    idx = np.random.default_rng(2).choice(w.B, 96, replace=False)
    ref = oracle(f, Sw[idx], Sd[idx])
    ti = torch.from_numpy(idx).cuda()
    check(net, f, Sw[idx], Sd[idx], ref, V[ti].contiguous(), it[ti].contiguous(),
          cv[ti].contiguous())


@pytest.mark.parametrize("mode", MODES)
def test_mixed_results_do_not_depend_on_the_batch(mode):
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=300)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), precision=mode)
    perm = np.random.default_rng(0).permutation(300)[:77]
    V2, it2, cv2 = net.solve(dev(Sw[perm]), dev(Sd[perm]), precision=mode)
    ti = torch.from_numpy(perm).cuda()
    assert torch.equal(V2, V[ti])
    assert torch.equal(it2, it[ti])


@pytest.mark.parametrize("mode", MODES)
def test_mixed_zero_load_and_divergence(mode):
    f = F.make_feeder(30, 15, delta_frac=0.3)
    z = np.zeros((5, f.n), dtype=np.complex128)
    net = zbus.Network.from_feeder(f)
    _, w = net.get_z()
    # one sweep in double-float; with the FP32 start sweeps the first sweep
    # cannot stop a scenario, so the second one (double-float) does
    for fp32_start, n_it in ((False, 1), (True, 2)):
        V, it, cv = net.solve(dev(z), dev(z), precision=mode, fp32_start=fp32_start)
        assert (cv.cpu().numpy() == 1).all() and (it.cpu().numpy() == n_it).all()
        # the FP64 residual of w is rounding noise, not exactly zero: V = w + O(1e-15)
        assert (V - w.expand(5, -1)).abs().max().item() <= 1e-12
    f, Sw, Sd, _ = F.make_workload("feeder128_b4096", B=6)
    Sw, Sd = Sw * 60.0, Sd * 60.0
    Sw[0] /= 60.0
    Sd[0] /= 60.0
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), max_iter=40, precision=mode)
    c = cv.cpu().numpy()
    assert c[0] == 1 and not c[1:].any()
    assert (it.cpu().numpy() <= 40).all()


def test_modes_agree_with_each_other_and_fp64():
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=256)
    net = zbus.Network.from_feeder(f)
    outs = {m: net.solve(dev(Sw), dev(Sd), precision=m)[0].cpu().numpy()
            for m in ["fp64", "fp16_scaled", "bf16x2", "tree"]}
    for m in ("fp16_scaled", "bf16x2", "tree"):
        assert np.abs(outs[m] - outs["fp64"]).max() <= 1e-6


@pytest.mark.parametrize("mode", MODES)
def test_final_mismatch_test_agrees_with_oracle(mode):
    """The FP64 mismatch test of the mixed path decides like the oracle's mismatch.

    Solve once, compute the oracle's power mismatch of the returned voltages,
    then solve again with the threshold between the smallest and the largest
    of those values: exactly the scenarios the oracle puts above it lose their
    flag (the voltages are the same, the solve being deterministic).
    """
    f = F.make_feeder(90, 31, delta_frac=0.5)
    Sw, Sd = F.make_scenarios(f, 64, 0.8, 1.2)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=1e-7, precision=mode)
    assert cv.cpu().numpy().all()
    ref = oracle(f, Sw[:1], Sd[:1])
    mm = O.power_mismatch(ref["Y_LL"], ref["Y_Ls"], f.v_slack, V.cpu().numpy(), Sw, Sd)
    thr = float(np.sqrt(mm.min() * mm.max()))
    assert mm.min() < thr < mm.max()
    V2, it2, cv2 = net.solve(dev(Sw), dev(Sd), tol=1e-7, precision=mode, mismatch_tol=thr,
                             max_correction=0)
    assert torch.equal(V2, V)
    want = (mm <= thr).astype(np.uint8)
    # both sides sum in FP64 in different orders: leave out near-ties
    clear = np.abs(mm / thr - 1.0) > 1e-3
    np.testing.assert_array_equal(cv2.cpu().numpy()[clear], want[clear])


@pytest.mark.parametrize("mode", ["fp16_scaled", "bf16x2"])
def test_final_mismatch_test_without_identical_mirror_blocks(mode):
    """The FP64 test on a network whose line blocks are not all mirrored
    (Y_ab != Y_ba for one line, as with a non-reciprocal element): each block
    product is formed at its own bus (the line-once form needs identical
    mirrors), and the test still decides like the oracle's mismatch."""
    f = F.make_feeder(90, 31, delta_frac=0.5)
    r0, c0 = next((r, c) for r, c in zip(f.Y_row, f.Y_col)
                  if r // 3 != c // 3 and min(r, c) >= 3)
    row = np.append(f.Y_row, r0).astype(np.int32)
    col = np.append(f.Y_col, c0).astype(np.int32)
    val = np.append(f.Y_val, 0.5 + 0.25j)
    Sw, Sd = F.make_scenarios(f, 64, 0.8, 1.2)
    net = zbus.Network(f.n_total, row, col, val, f.slack_idx, f.v_slack)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=1e-7, precision=mode, mismatch_tol=1.0,
                          max_correction=0)
    ref = O.solve_coo(f.n_total, row, col, val, f.slack_idx, f.v_slack, Sw, Sd, tol=1e-12,
                      max_iter=100)
    assert ref["converged"].all() and cv.cpu().numpy().all()
    assert np.abs(V.cpu().numpy() - ref["V"]).max() <= 1e-6
    mm = O.power_mismatch(ref["Y_LL"], ref["Y_Ls"], f.v_slack, V.cpu().numpy(), Sw, Sd)
    thr = float(np.sqrt(mm.min() * mm.max()))
    V2, it2, cv2 = net.solve(dev(Sw), dev(Sd), tol=1e-7, precision=mode, mismatch_tol=thr,
                             max_correction=0)
    assert torch.equal(V2, V)
    clear = np.abs(mm / thr - 1.0) > 1e-3
    np.testing.assert_array_equal(cv2.cpu().numpy()[clear], (mm <= thr).astype(np.uint8)[clear])


@pytest.mark.parametrize("mode", MODES)
def test_fp64_correction_sweeps(mode):
    """The final FP64 correction of the mixed forms.

    A loose stop tolerance (1e-5) leaves every scenario with an FP64 power
    mismatch of about 5e-7 .. 1e-6.  With the gate between the smallest and
    the largest of the oracle's mismatches of those voltages:
      * max_correction = 0: exactly the scenarios the oracle puts above the
        gate lose their flag, voltages unchanged;
      * max_correction = 8: every scenario keeps its flag; those below the
        gate are untouched (voltages bitwise, same iteration counts), those
        above took one or more FP64 correction sweeps (counted as
        iterations), and now pass the gate by the oracle's mismatch and lie
        within 1e-6 pu of the oracle's tight solution;
      * an unreachable gate: every flag is cleared after the allowed sweeps.
    """
    f = F.make_feeder(90, 31, delta_frac=0.5)
    Sw, Sd = F.make_scenarios(f, 64, 0.8, 1.2)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=1e-5, precision=mode, mismatch_tol=1.0,
                          max_correction=0)
    assert cv.cpu().numpy().all()
    ref = oracle(f, Sw, Sd, tol=1e-12, max_iter=100)
    mm = O.power_mismatch(ref["Y_LL"], ref["Y_Ls"], f.v_slack, V.cpu().numpy(), Sw, Sd)
    thr = float(np.sqrt(mm.min() * mm.max()))
    assert mm.min() < thr < mm.max()
    clear = np.abs(mm / thr - 1.0) > 1e-3   # FP64 sums in different orders: no near-ties
    above = (mm > thr) & clear
    below = (mm <= thr) & clear
    assert above.any() and below.any()

    V0, it0, cv0 = net.solve(dev(Sw), dev(Sd), tol=1e-5, precision=mode, mismatch_tol=thr,
                             max_correction=0)
    assert torch.equal(V0, V) and torch.equal(it0, it)
    np.testing.assert_array_equal(cv0.cpu().numpy()[clear], below[clear].astype(np.uint8))

    V8, it8, cv8 = net.solve(dev(Sw), dev(Sd), tol=1e-5, precision=mode, mismatch_tol=thr,
                             max_correction=8)
    V8h, it8h, ith = V8.cpu().numpy(), it8.cpu().numpy(), it.cpu().numpy()
    assert cv8.cpu().numpy().all()
    np.testing.assert_array_equal(V8h[below], V.cpu().numpy()[below])
    np.testing.assert_array_equal(it8h[below], ith[below])
    assert (it8h[above] > ith[above]).all() and (it8h[above] <= ith[above] + 8).all()
    mm8 = O.power_mismatch(ref["Y_LL"], ref["Y_Ls"], f.v_slack, V8h, Sw, Sd)
    assert mm8[above].max() <= thr * (1 + 1e-3)
    assert np.abs(V8h - ref["V"]).max() <= 1e-6
    err_before = np.abs(V.cpu().numpy() - ref["V"]).max(axis=1)
    err_after = np.abs(V8h - ref["V"]).max(axis=1)
    assert (err_after[above] < err_before[above]).all()

    Vx, itx, cvx = net.solve(dev(Sw), dev(Sd), tol=1e-5, precision=mode, mismatch_tol=1e-300,
                             max_correction=2)
    assert not cvx.cpu().numpy().any()
    np.testing.assert_array_equal(itx.cpu().numpy(), ith + 2)


def test_device_status_is_clean_after_solves():
    """No bounded device wait gives up in ordinary solves of every form."""
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=200)
    net = zbus.Network.from_feeder(f)
    for mode in ("fp64", "fp16_scaled", "bf16x2", "tree"):
        V, it, cv = net.solve(dev(Sw), dev(Sd), precision=mode)
        assert net.device_status() == 0, mode
        assert cv.cpu().numpy().all()


@pytest.mark.parametrize("mode", MODES)
def test_paper_stop_rule_sum_of_magnitudes(mode):
    """The paper's stop rule (the change of the sum of voltage magnitudes,
    Sec. II-B) in the defect forms: flags equal to the oracle's under the
    same rule, voltages within 1e-6 pu, sweep counts within one."""
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=96)
    ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                      tol=w.tol, max_iter=w.max_iter, rule="summag")
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), tol=w.tol, max_iter=w.max_iter, precision=mode,
                          rule="summag")
    check(net, f, Sw, Sd, ref, V, it, cv)


@pytest.mark.parametrize("mode", MODES)
def test_fp32_start_sweeps(mode):
    """Cold starts of the mixed forms begin with FP32 residual sweeps.

    Against double-float from the first sweep (fp32_start=False): the same
    flags, both within the parity bar of the oracle, iteration counts within
    one; warm starts never take the FP32 path (bitwise equal); no scenario
    stops on an FP32 sweep (a tolerance every step meets: one sweep without
    the FP32 start, two with it); the results of a scenario do not depend on
    the batch around it (lanes of a warp on different paths)."""
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=256)
    net = zbus.Network.from_feeder(f)
    ref = oracle(f, Sw, Sd)
    V1, it1, cv1 = net.solve(dev(Sw), dev(Sd), precision=mode)
    V0, it0, cv0 = net.solve(dev(Sw), dev(Sd), precision=mode, fp32_start=False)
    check(net, f, Sw, Sd, ref, V1, it1, cv1)
    check(net, f, Sw, Sd, ref, V0, it0, cv0)
    assert torch.equal(cv1, cv0)
    d_it = (it1 - it0).cpu().numpy()
    assert d_it.min() >= -1 and d_it.max() <= 1
    assert (V1 - V0).abs().max().item() <= 1e-8

    Vw = dev(ref["V"] * 0.999)
    Va, ita, cva = net.solve(dev(Sw), dev(Sd), V_init=Vw, precision=mode)
    Vb, itb, cvb = net.solve(dev(Sw), dev(Sd), V_init=Vw, precision=mode, fp32_start=False)
    assert torch.equal(Va, Vb) and torch.equal(ita, itb) and torch.equal(cva, cvb)

    # (the FP64 test passes whatever the mismatch, so no correction sweep adds
    # iterations)
    loose = dict(tol=10.0, precision=mode, mismatch_tol=1e9, max_correction=0)
    _, ita, cva = net.solve(dev(Sw[:40]), dev(Sd[:40]), fp32_start=False, **loose)
    assert (ita.cpu().numpy() == 1).all() and cva.cpu().numpy().all()
    _, ita, cva = net.solve(dev(Sw[:40]), dev(Sd[:40]), **loose)
    assert (ita.cpu().numpy() == 2).all() and cva.cpu().numpy().all()

    # a batch in which scenarios leave the FP32 path at different sweeps
    # (loads scaled per scenario), solved whole and as a subset
    scale = np.linspace(0.05, 1.6, 256)[:, None]
    Sws, Sds = Sw * scale, Sd * scale
    V, it, cv = net.solve(dev(Sws), dev(Sds), precision=mode)
    perm = np.random.default_rng(5).permutation(256)[:61]
    V2, it2, cv2 = net.solve(dev(Sws[perm]), dev(Sds[perm]), precision=mode)
    ti = torch.from_numpy(perm).cuda()
    assert torch.equal(V2, V[ti]) and torch.equal(it2, it[ti]) and torch.equal(cv2, cv[ti])
    assert len(np.unique(it.cpu().numpy())) > 1

