"""GPU parity of the load gradient (zbus_solve_adjoint) against the oracle.

Both sides receive the oracle's converged voltages and the same seeded loss
gradient G; the oracle solves the adjoint system directly (dense real solve),
the library iterates it in FP64 to a relative tolerance of 1e-13.  Bar: per
scenario max |H_gpu - H_oracle| <= 1e-9 max |H_oracle| (the iteration's
truncation is ~1e-13 of the gradient's size and FP64 rounding far below), the
adjoint converged on every scenario.  Also: the autograd wrapper against
central differences of the GPU forward solve, batch independence (bitwise),
host-driven and graph loops equal, zero G, a scenario with non-finite
voltages, partial-phase feeders and the bench's 128-bus workload at full
batch (sampled).  Both forms of the adjoint are checked: the dense FP64 Z^T
sweeps and the tree form (defect iteration with the exact Y^T residual and
the transposed tree sweep, radial networks), also with shunts, and the tree
form's refusal of a meshed network.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import zbus_oracle as O                      # noqa: E402
from paper_2605_14103_gb300 import feeders as F          # noqa: E402
from paper_2605_14103_gb300 import zbus                  # noqa: E402

pytestmark = pytest.mark.gpu
REL = 1e-9
FORMS = ["fp64", "tree"]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    B.build()
    zbus.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def forward_oracle(f, Sw, Sd, bus_phase=None):
    r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                    tol=1e-14, max_iter=300, bus_phase=bus_phase)
    assert r["converged"].all()
    return r


def loss_grad(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def assert_close(H, Href):
    for b in range(Href.shape[0]):
        scale = max(np.abs(Href[b]).max(), 1e-300)
        err = np.abs(H[b] - Href[b]).max()
        assert err <= REL * scale, (b, err, scale)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("N,B,delta,seed", [(13, 5, 0.0, 101), (40, 33, 0.4, 7),
                                            (128, 17, 0.3, 202), (200, 3, 0.3, 9)])
def test_parity_against_the_oracle(N, B, delta, seed, form):
    f = F.make_feeder(N, seed, delta_frac=delta, mult_hi=1.5)
    Sw, Sd = F.make_scenarios(f, B, 0.5, 1.5)
    r = forward_oracle(f, Sw, Sd)
    G = loss_grad(Sw.shape, seed)
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G)
    net = zbus.Network.from_feeder(f)
    dw, dd, it, cv = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd), tol=1e-13,
                                       precision=form)
    assert cv.cpu().numpy().all()
    assert it.cpu().numpy().max() < 200
    assert_close(dw.cpu().numpy(), Hw)
    assert_close(dd.cpu().numpy(), Hd)
    net.close()


def test_wye_only_and_one_output():
    f = F.make_feeder(60, 31, delta_frac=0.0)
    Sw, Sd = F.make_scenarios(f, 9, 0.8, 1.2)
    r = forward_oracle(f, Sw, Sd)
    G = loss_grad(Sw.shape, 3)
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"], Sw, 0 * Sw, G)
    net = zbus.Network.from_feeder(f)
    dw, dd, it, cv = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), None, tol=1e-13,
                                       delta=False)
    assert dd is None and cv.cpu().numpy().all()
    assert_close(dw.cpu().numpy(), Hw)
    _, dd2, _, _ = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), None, tol=1e-13, wye=False)
    assert_close(dd2.cpu().numpy(), Hd)


@pytest.mark.parametrize("form", FORMS)
def test_autograd_against_finite_differences_of_the_gpu_solve(form):
    f = F.make_feeder(20, 44, delta_frac=0.5)
    Sw, Sd = F.make_scenarios(f, 4, 0.8, 1.2)
    net = zbus.Network.from_feeder(f)
    G = dev(loss_grad(Sw.shape, 5))
    sw = dev(Sw).requires_grad_(True)
    sd = dev(Sd).requires_grad_(True)
    V, it, cv = zbus.solve_differentiable(net, sw, sd, tol=1e-13, max_iter=300,
                                          adj_precision=form)
    assert cv.all()
    L = (torch.conj(G) * V).real.sum()
    L.backward()
    ait, acv = net.last_adjoint
    assert acv.all()

    def Lof(a, b):
        V, _, c = net.solve(a, b, tol=1e-13, max_iter=300)
        assert c.all()
        return float((torch.conj(G) * V).real.sum())

    rng = np.random.default_rng(9)
    h = 1e-4
    for grad, wye in ((sw.grad, True), (sd.grad, False)):
        d = dev((rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)) * 0.05)
        base_w, base_d = dev(Sw), dev(Sd)
        if wye:
            fd = (Lof(base_w + h * d, base_d) - Lof(base_w - h * d, base_d)) / (2 * h)
        else:
            fd = (Lof(base_w, base_d + h * d) - Lof(base_w, base_d - h * d)) / (2 * h)
        ad = float((torch.conj(grad) * d).real.sum())
        assert abs(ad - fd) <= 1e-5 * max(1.0, abs(fd)), (wye, ad, fd)


@pytest.mark.parametrize("form", FORMS)
def test_batch_independence_and_loop_forms(monkeypatch, form):
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=100)
    r = forward_oracle(f, Sw, Sd)
    G = loss_grad(Sw.shape, 11)
    net = zbus.Network.from_feeder(f)
    dw, dd, it, cv = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd), precision=form)
    perm = np.random.default_rng(0).permutation(100)[:37]
    dw2, dd2, it2, cv2 = net.solve_adjoint(dev(r["V"][perm]), dev(G[perm]), dev(Sw[perm]),
                                           dev(Sd[perm]), precision=form)
    idx = torch.from_numpy(perm).cuda()
    assert torch.equal(dw2, dw[idx]) and torch.equal(dd2, dd[idx])     # bitwise
    assert torch.equal(it2, it[idx])
    if form == "tree":
        return   # one launch, no sweep loop on the host side
    monkeypatch.setenv("ZBUS_NO_GRAPH", "1")
    dw3, dd3, it3, cv3 = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd))
    assert torch.equal(dw3, dw) and torch.equal(dd3, dd) and torch.equal(it3, it)


@pytest.mark.parametrize("form", FORMS)
def test_zero_gradient_and_non_finite_voltages(form):
    f = F.make_feeder(30, 12, delta_frac=0.3)
    Sw, Sd = F.make_scenarios(f, 6, 0.8, 1.2)
    r = forward_oracle(f, Sw, Sd)
    net = zbus.Network.from_feeder(f)
    G = loss_grad(Sw.shape, 4)
    G[2] = 0
    V = r["V"].copy()
    V[4, 7] = np.nan
    dw, dd, it, cv = net.solve_adjoint(dev(V), dev(G), dev(Sw), dev(Sd), tol=1e-13,
                                       precision=form)
    cv, it = cv.cpu().numpy(), it.cpu().numpy()
    assert cv[2] == 1 and it[2] == 1
    assert not np.any(dw.cpu().numpy()[2]) and not np.any(dd.cpu().numpy()[2])
    assert cv[4] == 0
    ok = [0, 1, 3, 5]
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"][ok], Sw[ok], Sd[ok], G[ok])
    assert cv[ok].all()
    assert_close(dw.cpu().numpy()[ok], Hw)
    assert_close(dd.cpu().numpy()[ok], Hd)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("N,B,seed", [(12, 4, 3), (90, 20, 77)])
def test_partial_phase_feeders(N, B, seed, form):
    f = F.make_partial_feeder(N, seed, lateral_frac=0.8, delta_frac=0.5, mult_hi=1.5)
    Sw, Sd = F.make_partial_scenarios(f, B, 0.5, 1.5)
    r = forward_oracle(f, Sw, Sd, f.bus_phase)
    G = loss_grad(Sw.shape, seed)
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G, bus_phase=r["bus_phase"])
    net = zbus.Network.from_feeder(f)
    dw, dd, it, cv = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd), tol=1e-13,
                                       precision=form)
    assert cv.cpu().numpy().all()
    assert_close(dw.cpu().numpy(), Hw)
    assert_close(dd.cpu().numpy(), Hd)


@pytest.mark.parametrize("form", FORMS)
def test_bench_workload_full_batch_sampled(form):
    """The 128-bus workload at its full 4096 scenarios, in the launch
    configuration the benchmark times; the oracle checks a sample."""
    f, Sw, Sd, w = F.make_workload("feeder128_b4096")
    r = forward_oracle(f, Sw, Sd)
    G = loss_grad(Sw.shape, 2024)
    net = zbus.Network.from_feeder(f)
    dw, dd, it, cv = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd), tol=1e-12,
                                       precision=form)
    assert cv.cpu().numpy().all()
    pick = np.random.default_rng(1).choice(Sw.shape[0], 6, replace=False)
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"][pick], Sw[pick], Sd[pick], G[pick])
    assert_close(dw.cpu().numpy()[pick], Hw)
    assert_close(dd.cpu().numpy()[pick], Hd)


def with_extra(f, extra):
    row = list(f.Y_row) + [r for r, c in extra]
    col = list(f.Y_col) + [c for r, c in extra]
    val = list(f.Y_val) + list(extra.values())
    return (np.asarray(row, np.int32), np.asarray(col, np.int32),
            np.asarray(val, np.complex128))


def test_tree_form_with_shunts_and_refusal_of_a_meshed_network():
    # capacitive shunts: the transposed sweep inverts only the series part,
    # the exact Y^T residual keeps them
    f = F.make_feeder(90, 12, delta_frac=0.4)
    extra = {(3 * bus + p, 3 * bus + p): 0.02j for bus in (3, 9, 20, 33, 71) for p in range(3)}
    row, col, val = with_extra(f, extra)
    Sw, Sd = F.make_scenarios(f, 20, 0.8, 1.2, seed=4)
    r = O.solve_coo(f.n_total, row, col, val, f.slack_idx, f.v_slack, Sw, Sd, tol=1e-14,
                    max_iter=300)
    assert r["converged"].all()
    G = loss_grad(Sw.shape, 8)
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G)
    net = zbus.Network(f.n_total, row, col, val, f.slack_idx, f.v_slack)
    dw, dd, it, cv = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd), tol=1e-13,
                                       precision="tree")
    assert cv.cpu().numpy().all()
    assert_close(dw.cpu().numpy(), Hw)
    assert_close(dd.cpu().numpy(), Hd)
    # a loop: the tree form refuses, the dense form still answers
    a, b = 5, 17
    y = np.linalg.inv(f.z_line[4])
    mesh = {}
    for p in range(3):
        for q in range(3):
            mesh[(3 * a + p, 3 * a + q)] = y[p, q]
            mesh[(3 * b + p, 3 * b + q)] = y[p, q]
            mesh[(3 * a + p, 3 * b + q)] = -y[p, q]
            mesh[(3 * b + p, 3 * a + q)] = -y[p, q]
    row, col, val = with_extra(f, mesh)
    netm = zbus.Network(f.n_total, row, col, val, f.slack_idx, f.v_slack)
    rm = O.solve_coo(f.n_total, row, col, val, f.slack_idx, f.v_slack, Sw[:3], Sd[:3],
                     tol=1e-14, max_iter=300)
    with pytest.raises(zbus.ZbusError) as e:
        netm.solve_adjoint(dev(rm["V"]), dev(G[:3]), dev(Sw[:3]), dev(Sd[:3]), precision="tree")
    assert e.value.status == 7
    dw, dd, it, cv = netm.solve_adjoint(dev(rm["V"]), dev(G[:3]), dev(Sw[:3]), dev(Sd[:3]),
                                        tol=1e-13)
    Hw, Hd = O.solve_adjoint(rm["Z"], rm["V"], Sw[:3], Sd[:3], G[:3])
    assert_close(dw.cpu().numpy(), Hw)
    with pytest.raises(zbus.ZbusError):
        net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd), precision="fp16_scaled")


def test_argument_errors():
    f = F.make_feeder(10, 1)
    Sw, Sd = F.make_scenarios(f, 2, 0.8, 1.2)
    net = zbus.Network.from_feeder(f)
    V = dev(Sw)
    with pytest.raises(zbus.ZbusError):
        zbus.zbus_solve_adjoint(net.handle, None, None, V, V, -1.0, 10, None, None, None,
                                torch.empty(2, dtype=torch.int32, device="cuda"),
                                torch.empty(2, dtype=torch.uint8, device="cuda"))
    with pytest.raises(zbus.ZbusError):
        zbus.zbus_solve_adjoint(net.handle, None, None, V, V, 1e-10, 0, None, None, None,
                                torch.empty(2, dtype=torch.int32, device="cuda"),
                                torch.empty(2, dtype=torch.uint8, device="cuda"))
    assert os.environ.get("ZBUS_NO_GRAPH") != "1"


def test_dense_form_on_a_non_reciprocal_network():
    """Feeder matrices are symmetric (Z^T = Z), so a transposition mistake in
    the device's Z^T would pass every other case.  A phase-shifting element
    on one line (Y_ab != Y_ba) makes Y and Z non-symmetric; the dense form
    must still match the oracle, and the tree form must refuse."""
    f = F.make_feeder(25, 61, delta_frac=0.4)
    a = 9
    p = int(f.parent[a])
    y = np.linalg.inv(f.z_line[a])
    extra = {}
    for i in range(3):
        for j in range(3):
            extra[(3 * a + i, 3 * p + j)] = 0.08j * y[i, j]
            extra[(3 * p + i, 3 * a + j)] = -0.08j * y[i, j]
    row, col, val = with_extra(f, extra)
    Y = O.dense_from_coo(f.n_total, row, col, val)
    assert np.abs(Y - Y.T).max() > 1.0
    Sw, Sd = F.make_scenarios(f, 9, 0.8, 1.2)
    r = O.solve_coo(f.n_total, row, col, val, f.slack_idx, f.v_slack, Sw, Sd, tol=1e-14,
                    max_iter=300)
    assert r["converged"].all()
    assert np.abs(r["Z"] - r["Z"].T).max() > 1e-4
    G = loss_grad(Sw.shape, 17)
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G)
    net = zbus.Network(f.n_total, row, col, val, f.slack_idx, f.v_slack)
    dw, dd, it, cv = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd), tol=1e-13)
    assert cv.cpu().numpy().all()
    assert_close(dw.cpu().numpy(), Hw)
    assert_close(dd.cpu().numpy(), Hd)
    with pytest.raises(zbus.ZbusError) as e:
        net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd), precision="tree")
    assert e.value.status == 7


@pytest.mark.parametrize("form", FORMS)
def test_iteration_cap(form):
    """With one sweep allowed the adjoint cannot meet a tight tolerance: the
    flags say so and the call returns (the partial gradient is not used)."""
    f = F.make_feeder(30, 14, delta_frac=0.4)
    Sw, Sd = F.make_scenarios(f, 5, 0.8, 1.2)
    r = forward_oracle(f, Sw, Sd)
    net = zbus.Network.from_feeder(f)
    G = loss_grad(Sw.shape, 6)
    dw, dd, it, cv = net.solve_adjoint(dev(r["V"]), dev(G), dev(Sw), dev(Sd), tol=1e-13,
                                       max_iter=1, precision=form)
    assert not cv.cpu().numpy().any()
    assert (it.cpu().numpy() == 1).all()
