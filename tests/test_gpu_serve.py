"""Serving loop: continuous batching over a pool of feeders.

A request's result must be the same served alone and in a mix of requests
that overlap on the GPU (bitwise: the per-scenario arithmetic does not depend
on slot position or neighbours), match the FP64 oracle within 1e-6 pu with
identical flags, honour warm starts, and report requests that cannot fit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import zbus_oracle as O                      # noqa: E402
from paper_2605_14103_gb300 import feeders as F          # noqa: E402
from paper_2605_14103_gb300 import zbus                  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    B.build()
    zbus.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def pool():
    specs = [(40, 1), (90, 2), (200, 3)]
    feeders = [F.make_feeder(N, 600 + s, delta_frac=0.4) for N, s in specs]
    nets = [zbus.Network.from_feeder(f) for f in feeders]
    return feeders, nets


def make_requests(feeders, sizes, seed=0):
    rng = np.random.default_rng(seed)
    reqs, host = [], []
    for i, B in enumerate(sizes):
        k = int(rng.integers(0, len(feeders)))
        Sw, Sd = F.make_scenarios(feeders[k], B, 0.8, 1.2, seed=1000 + i)
        reqs.append({"feeder": k, "S_wye": dev(Sw), "S_delta": dev(Sd), "arrival": 0.0})
        host.append((k, Sw, Sd))
    return reqs, host


@pytest.mark.parametrize("mode", ["fp16_scaled", "bf16x2", "tree"])
def test_same_alone_and_in_the_mix(pool, mode):
    feeders, nets = pool
    reqs, host = make_requests(feeders, [1, 5, 33, 130, 200, 7, 64, 129], seed=3)
    mixed = zbus.serve(nets, reqs, precision=mode, max_slots=512)
    for i, q in enumerate(reqs):
        alone = zbus.serve(nets, [q], precision=mode, max_slots=512)[0]
        m = mixed[i]
        assert m["status"] == 0 and alone["status"] == 0
        assert torch.equal(m["V"], alone["V"])
        assert torch.equal(m["iters"], alone["iters"])
        assert torch.equal(m["converged"], alone["converged"])
        k, Sw, Sd = host[i]
        f = feeders[k]
        ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd)
        np.testing.assert_array_equal(m["converged"].cpu().numpy(), ref["converged"])
        mk = ref["converged"] == 1
        assert np.abs(m["V"].cpu().numpy()[mk] - ref["V"][mk]).max() <= 1e-6
        assert m["n_converged"] == int(ref["converged"].sum())
        assert m["t_done"] >= m["t_admit"] >= 0.0


def test_staggered_arrivals_overlap(pool):
    feeders, nets = pool
    reqs, host = make_requests(feeders, [300, 20, 20, 20, 20, 20], seed=5)
    for i, q in enumerate(reqs):
        q["arrival"] = 0.0 if i == 0 else 1e-4 * i
    res = zbus.serve(nets, reqs, max_slots=512)
    assert all(r["status"] == 0 for r in res)
    # later small requests are admitted while the first one is still running
    assert any(r["t_admit"] < res[0]["t_done"] for r in res[1:])
    for r, (k, Sw, Sd) in zip(res, host):
        assert r["n_converged"] == r["B"]


def test_warm_start_from_the_last_converged_voltage(pool):
    feeders, nets = pool
    f = feeders[2]
    Sw, Sd = F.make_scenarios(f, 8, 0.8, 1.2, seed=77)
    first = {"feeder": 2, "S_wye": dev(Sw), "S_delta": dev(Sd), "arrival": 0.0}
    second = {"feeder": 2, "S_wye": dev(Sw), "S_delta": dev(Sd), "arrival": 0.05,
              "warm_start": True}
    res = zbus.serve(nets, [first, second], max_slots=256)
    assert res[1]["max_iters"] < res[0]["max_iters"]
    ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd)
    assert np.abs(res[1]["V"].cpu().numpy() - ref["V"]).max() <= 1e-6


def test_oversized_request_is_reported_and_others_served(pool):
    feeders, nets = pool
    reqs, host = make_requests(feeders, [10, 300, 10], seed=9)
    res = zbus.serve(nets, reqs, max_slots=128)
    assert res[1]["status"] == 1
    assert res[0]["status"] == 0 and res[2]["status"] == 0


def test_budget_too_small_is_refused(pool):
    feeders, nets = pool
    reqs, _ = make_requests(feeders, [4], seed=1)
    with pytest.raises(zbus.ZbusError) as ei:
        zbus.serve(nets, reqs, hbm_budget_bytes=1 << 20)
    assert ei.value.status == 3


@pytest.mark.parametrize("mode", ["fp16_scaled", "tree"])
def test_operand_cache_under_a_budget_below_the_pool(mode):
    """The pool's operands exceed the budget: the serving loop keeps an
    operand cache, evicts idle feeders (least recently used first) and forms
    a feeder's operands on demand.  Every request completes, each equal,
    bitwise, to its result alone and within 1e-6 pu of the oracle; operands
    are formed more often than there are feeders; a network the loop released
    still solves (its Z formed again, bitwise the same)."""
    feeders = [F.make_feeder(N, 700 + N, delta_frac=0.4) for N in (200, 220, 60)]
    nets = [zbus.Network.from_feeder(f) for f in feeders]
    Z0, w0 = nets[1].get_z()
    Z0, w0 = Z0.clone(), w0.clone()
    fp = [zbus.zbus_serve_footprint(n.handle, mode) for n in nets]
    slots = 128
    peak = max(a + b for a, b, _ in fp)
    budget = sum(c for _, _, c in fp) * slots + peak   # room for one large feeder at a time
    assert fp[0][0] + fp[1][0] > peak                  # the two large ones never fit together
    # requests far enough apart that each finds the previous one's feeder idle:
    # the two large feeders keep evicting each other (and the small one)
    order = [0, 1, 0, 2, 1, 1, 0, 2]
    reqs, host = [], []
    for i, k in enumerate(order):
        Sw, Sd = F.make_scenarios(feeders[k], 16 + 7 * i, 0.8, 1.2, seed=50 + i)
        reqs.append({"feeder": k, "S_wye": dev(Sw), "S_delta": dev(Sd), "arrival": 0.08 * i})
        host.append((k, Sw, Sd))
    mixed = zbus.serve(nets, reqs, precision=mode, max_slots=slots, hbm_budget_bytes=budget)
    assert all(r["status"] == 0 for r in mixed)
    assert sum(r["operands_formed"] for r in mixed) >= 4
    for i, q in enumerate(reqs):
        alone = zbus.serve(nets, [dict(q, arrival=0.0)], precision=mode, max_slots=slots,
                           hbm_budget_bytes=budget)[0]
        m = mixed[i]
        assert torch.equal(m["V"], alone["V"]), i
        assert torch.equal(m["iters"], alone["iters"]), i
        assert torch.equal(m["converged"], alone["converged"]), i
        k, Sw, Sd = host[i]
        f = feeders[k]
        ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd)
        np.testing.assert_array_equal(m["converged"].cpu().numpy(), ref["converged"])
        assert np.abs(m["V"].cpu().numpy() - ref["V"]).max() <= 1e-6
    # the networks the loop released form their operands again on demand
    Z1, w1 = nets[1].get_z()
    assert torch.equal(Z1, Z0) and torch.equal(w1, w0)
    for k, net in enumerate(nets):
        Sw, Sd = F.make_scenarios(feeders[k], 9, 0.8, 1.2, seed=99)
        V, it, cv = net.solve(dev(Sw), dev(Sd), precision="fp64")
        f = feeders[k]
        ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd)
        assert np.abs(V.cpu().numpy() - ref["V"]).max() <= 1e-6
