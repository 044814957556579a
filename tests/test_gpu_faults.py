"""Failures made on the host, none of which faults, traps or hangs the GPU:
non-finite loads in one scenario, a delta branch whose two phase voltages are
equal in a warm start (its current divides by zero), a serving request with
non-finite loads, and a request source that fails in the middle of serving.
In every case the other scenarios and requests are untouched and the call
returns."""
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
    return O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd, **kw)


@pytest.mark.parametrize("form", FORMS)
def test_non_finite_loads_stop_only_their_scenario(form):
    f = F.make_feeder(50, 21, delta_frac=0.4)
    Sw, Sd = F.make_scenarios(f, 9, 0.8, 1.2)
    Sw[2, 5] = np.nan
    Sd[6, 9] = complex(np.inf, 0.0) if Sd[6, 9] != 0 else Sd[6, 9]
    Sw[6, 9] = np.inf
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), precision=form)
    cv = cv.cpu().numpy()
    assert cv[2] == 0 and cv[6] == 0
    ok = [b for b in range(9) if b not in (2, 6)]
    ref = oracle(f, Sw[ok], Sd[ok])
    np.testing.assert_array_equal(cv[ok], ref["converged"])
    assert np.abs(V.cpu().numpy()[ok] - ref["V"]).max() <= 1e-6
    assert net.device_status() == 0


@pytest.mark.parametrize("form", FORMS)
def test_equal_phase_voltages_on_a_delta_branch(form):
    """A warm start with v_a = v_b at a bus with a delta load: the first
    current is a division by zero.  The scenario either stops unconverged or
    recovers to the oracle's solution; the others are untouched."""
    f = F.make_feeder(40, 22, delta_frac=1.0)
    Sw, Sd = F.make_scenarios(f, 5, 0.8, 1.2)
    ref = oracle(f, Sw, Sd)
    V0 = np.broadcast_to(ref["V"][0], Sw.shape).copy()
    bus = 7
    V0[3, 3 * bus + 1] = V0[3, 3 * bus + 0]
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), V_init=dev(V0), precision=form)
    V, cv = V.cpu().numpy(), cv.cpu().numpy()
    ok = [0, 1, 2, 4]
    np.testing.assert_array_equal(cv[ok], ref["converged"][ok])
    assert np.abs(V[ok] - ref["V"][ok]).max() <= 1e-6
    if cv[3]:
        assert np.abs(V[3] - ref["V"][3]).max() <= 1e-6
    assert net.device_status() == 0


@pytest.fixture(scope="module")
def pool():
    feeders = [F.make_feeder(N, 700 + s, delta_frac=0.4) for N, s in ((30, 1), (70, 2))]
    return feeders, [zbus.Network.from_feeder(f) for f in feeders]


def test_serving_request_with_non_finite_loads(pool):
    feeders, nets = pool
    reqs = []
    for i, (k, B) in enumerate(((0, 5), (1, 9), (0, 3))):
        Sw, Sd = F.make_scenarios(feeders[k], B, 0.8, 1.2, seed=50 + i)
        if i == 1:
            Sw[4, 0] = np.nan
        reqs.append({"feeder": k, "S_wye": dev(Sw), "S_delta": dev(Sd), "arrival": 0.0})
    res = zbus.serve(nets, reqs, max_slots=256)
    assert all(r["status"] == 0 for r in res)
    assert res[0]["n_converged"] == 5 and res[2]["n_converged"] == 3
    assert res[1]["n_converged"] == 8
    assert res[1]["converged"].cpu().numpy()[4] == 0


def test_failing_request_source(pool):
    """The source delivers two requests and then raises: the loop stops taking
    requests, serves the two, returns ZBUS_ERR_SOURCE, and the binding raises
    the source's own exception."""
    feeders, nets = pool
    keep, done = [], []
    reqs = []
    for i, (k, B) in enumerate(((0, 4), (1, 6))):
        Sw, Sd = F.make_scenarios(feeders[k], B, 0.8, 1.2, seed=80 + i)
        Swd, Sdd = dev(Sw), dev(Sd)
        V = torch.empty((B, nets[k].n), dtype=torch.complex128, device="cuda")
        it = torch.empty((B,), dtype=torch.int32, device="cuda")
        cv = torch.empty((B,), dtype=torch.uint8, device="cuda")
        keep.append((Swd, Sdd, V, it, cv))
        r = zbus.zbus_request()
        r.feeder, r.B = k, B
        r.S_wye, r.S_delta = Swd.data_ptr(), Sdd.data_ptr()
        r.V_out, r.iters, r.converged = V.data_ptr(), it.data_ptr(), cv.data_ptr()
        r.tag = i
        reqs.append(r)
    calls = [0]

    def source(now):
        calls[0] += 1
        if calls[0] <= 2:
            return reqs[calls[0] - 1]
        raise RuntimeError("request feed lost")

    def sink(req, res):
        done.append((req.tag, res.status, res.n_converged))

    cfg = zbus.zbus_serve_config()
    cfg.hbm_budget_bytes = 8 << 30
    cfg.max_slots = 256
    cfg.precision = zbus.PRECISION["fp16_scaled"]
    cfg.conv_rule = 0
    cfg.max_iter = 50
    cfg.tol = 1e-8
    cfg.mismatch_tol = 1e-6
    with pytest.raises(RuntimeError, match="request feed lost"):
        zbus.zbus_serve(cfg, [n.handle for n in nets], source, sink)
    assert sorted(done) == [(0, 0, 4), (1, 0, 6)]
    # a source that ends normally gives ZBUS_OK; the status of a failed one
    # is ZBUS_ERR_SOURCE through the raw call
    assert zbus.zbus_status_string(8) == "ZBUS_ERR_SOURCE"
