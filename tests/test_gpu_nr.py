"""GPU parity of the batched Newton-Raphson power flow (zbus_nr_solve) against
the FP64 Newton-Raphson oracle, through the C ABI.

Both arithmetic forms of the Newton direction are checked (FP64, and FP32
GMRES under the FP64 mismatch).  Bar (per scenario): converged flags
identical; on converged scenarios
max |V_gpu - V_oracle| <= 1e-6 pu (checked tighter, 1e-8: both sides stop
at max |F| <= 1e-10 and the solution moves by about |J^-1| times that),
Newton step counts within one of the oracle's (GMRES solves each Newton
system to a relative 1e-6, the oracle exactly), and the mismatch of the GPU
voltages, recomputed on the CPU with the admittance matrix, <= 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nr_oracle as O                        # noqa: E402
from paper_2605_14103_gb300 import grids as G            # noqa: E402
from paper_2605_14103_gb300 import zbus                  # noqa: E402

pytestmark = pytest.mark.gpu
TOL_V = 1e-6
TOL_TIGHT = 1e-8


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    B.build()
    zbus.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def cpu_mismatch(g, V, P, Q):
    Y = O.dense_Y(g.N, g.Y_row, g.Y_col, g.Y_val)
    th, q = O.index_sets(g.bus_type)
    return np.array([np.abs(O.mismatch(Y, V[b], P[b], Q[b], th, q)).max()
                     for b in range(V.shape[0])])


def compare(g, P, Q, V, it, cv, ref, idx=None):
    V, it, cv = V.cpu().numpy(), it.cpu().numpy(), cv.cpu().numpy()
    if idx is not None:
        V, it, cv, P, Q = V[idx], it[idx], cv[idx], P[idx], Q[idx]
    np.testing.assert_array_equal(cv, ref["converged"])
    m = ref["converged"] == 1
    assert m.any()
    err = np.abs(V[m] - ref["V"][m]).max()
    assert err <= TOL_V and err <= TOL_TIGHT, err
    assert np.abs(it[m] - ref["iters"][m]).max() <= 1
    assert cpu_mismatch(g, V[m], P[m], Q[m]).max() <= 1e-9


PRECISIONS = ["fp64", "mixed"]


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("N,B,seed", [(14, 7, 1), (30, 33, 2), (118, 64, 611), (300, 5, 9)])
def test_parity_against_the_oracle(N, B, seed, prec):
    g = G.make_grid(N, seed)
    P, Q = G.make_injections(g, B)
    ref = O.solve_batch(g.N, g.Y_row, g.Y_col, g.Y_val, g.bus_type, g.v_set, P, Q)
    net = zbus.NrNetwork.from_grid(g)
    V, it, cv, gm = net.solve(dev(P), dev(Q), precision=prec)
    compare(g, P, Q, V, it, cv, ref)
    gm = gm.cpu().numpy()
    assert (gm >= it.cpu().numpy()).all() and gm.max() < 40 * 20
    nt, nq, fnnz, flev = net.info()
    assert nt == N - 1 and nq == int((g.bus_type == G.PQ).sum())
    net.close()


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("name,sample", [("grid1354_b1000", 2), ("grid2224_b1000", 2)])
def test_large_grids_full_batch_sampled(name, sample, prec):
    """The benchmark's grids at their full 1000 scenarios; the oracle checks a
    sample, the CPU mismatch every scenario."""
    g, P, Q, w = G.make_grid_workload(name)
    net = zbus.NrNetwork.from_grid(g)
    V, it, cv, gm = net.solve(dev(P), dev(Q), tol=w.tol, max_iter=w.max_iter, precision=prec)
    assert cv.cpu().numpy().all()
    pick = np.random.default_rng(5).choice(P.shape[0], sample, replace=False)
    ref = O.solve_batch(g.N, g.Y_row, g.Y_col, g.Y_val, g.bus_type, g.v_set, P[pick], Q[pick])
    compare(g, P, Q, V, it, cv, ref, idx=pick)
    import scipy.sparse as sp
    Y = sp.csr_matrix((g.Y_val, (g.Y_row, g.Y_col)), shape=(g.N, g.N))
    Vn = V.cpu().numpy()
    S = Vn * np.conj((Y @ Vn.T).T)
    th, q = O.index_sets(g.bus_type)
    F = np.concatenate([S.real[:, th] - P[:, th], S.imag[:, q] - Q[:, q]], axis=1)
    assert np.abs(F).max() <= 1e-9


def test_two_bus_closed_form_and_pv_only_grid():
    z, S = 0.02 + 0.1j, 1.2 + 0.4j
    y = 1.0 / z
    row, col, val = [0, 1, 0, 1], [0, 1, 1, 0], [y, y, -y, -y]
    net = zbus.NrNetwork(2, row, col, val, [2, 0], [1.0, 1.0])
    P = dev(np.array([[0.0, -S.real]]))
    Q = dev(np.array([[0.0, -S.imag]]))
    V, it, cv, gm = net.solve(P, Q, tol=1e-13)
    c = 2.0 * (np.conj(z) * S).real - 1.0
    u = 0.5 * (-c + np.sqrt(c * c - 4.0 * abs(z) ** 2 * abs(S) ** 2))
    assert cv.item() == 1
    assert abs(V.cpu().numpy()[0, 1] - (u + np.conj(z) * S)) < 1e-12
    # slack + two PV buses: no magnitude unknowns (an empty B'')
    g = G.make_grid(3, 4)
    bt = np.array([2, 1, 1], dtype=np.int32)
    vs = np.array([1.0, 1.01, 0.99])
    P3 = np.array([[0.0, 0.3, -0.4]])
    Q3 = np.zeros((1, 3))
    net3 = zbus.NrNetwork(3, g.Y_row, g.Y_col, g.Y_val, bt, vs)
    V3, it3, cv3, _ = net3.solve(dev(P3), dev(Q3))
    Vo, ito, cvo = O.newton(O.dense_Y(3, g.Y_row, g.Y_col, g.Y_val), bt, vs, P3[0], Q3[0])
    assert cv3.item() == 1 and cvo == 1
    assert np.abs(V3.cpu().numpy()[0] - Vo).max() <= TOL_TIGHT


@pytest.mark.parametrize("prec", PRECISIONS)
def test_batch_independence_and_short_gmres_cycles(prec):
    g = G.make_grid(90, 17)
    P, Q = G.make_injections(g, 40)
    net = zbus.NrNetwork.from_grid(g)
    V, it, cv, gm = net.solve(dev(P), dev(Q), precision=prec)
    perm = np.random.default_rng(2).permutation(40)[:13]
    V2, it2, cv2, gm2 = net.solve(dev(P[perm]), dev(Q[perm]), precision=prec)
    idx = torch.from_numpy(perm).cuda()
    assert torch.equal(V2, V[idx]) and torch.equal(it2, it[idx]) and torch.equal(gm2, gm[idx])
    # two Krylov vectors per cycle: restarts do the work, same solution
    V3, it3, cv3, gm3 = net.solve(dev(P), dev(Q), gmres_restart=2, gmres_max_restarts=40,
                                  precision=prec)
    assert cv3.cpu().numpy().all()
    assert (V3 - V).abs().max().item() <= TOL_TIGHT


def test_divergence_and_iteration_cap():
    g = G.make_grid(40, 8)
    P, Q = G.make_injections(g, 3)
    net = zbus.NrNetwork.from_grid(g)
    P2, Q2 = P.copy(), Q.copy()
    P2[1] *= 400
    Q2[1] *= 400
    V, it, cv, gm = net.solve(dev(P2), dev(Q2), max_iter=15)
    cv = cv.cpu().numpy()
    assert cv[0] == 1 and cv[1] == 0 and cv[2] == 1
    assert it.cpu().numpy()[1] <= 15
    V0, it0, cv0, _ = net.solve(dev(P), dev(Q), max_iter=0)
    assert not cv0.cpu().numpy().any() and not it0.cpu().numpy().any()
    e = torch.empty((0, g.N), dtype=torch.float64, device="cuda")
    net.solve(e, e)


def test_argument_errors():
    g = G.make_grid(10, 1)
    bt = g.bus_type.copy()
    bt[3] = 2
    with pytest.raises(zbus.ZbusError):
        zbus.NrNetwork(g.N, g.Y_row, g.Y_col, g.Y_val, bt, g.v_set)
    net = zbus.NrNetwork.from_grid(g)
    P, Q = G.make_injections(g, 2)
    with pytest.raises(zbus.ZbusError):
        net.solve(dev(P), dev(Q), gmres_restart=0)
    with pytest.raises(zbus.ZbusError):
        net.solve(dev(P), dev(Q), gmres_tol=2.0)
    o = zbus.zbus_nr_opts_default()
    o.precision = 7
    B = P.shape[0]
    outs = (torch.empty((B, g.N), dtype=torch.complex128, device="cuda"),
            torch.empty((B,), dtype=torch.int32, device="cuda"),
            torch.empty((B,), dtype=torch.uint8, device="cuda"))
    with pytest.raises(zbus.ZbusError):
        zbus.zbus_nr_solve(net.handle, g.N, dev(P), dev(Q), 1e-10, 20, o, *outs)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_phase_shifter_makes_y_non_symmetric(prec):
    """A phase-shifting transformer (complex tap) between two PQ buses: Y,
    B' and G_Q,Theta are no longer symmetric; both forms still match the
    oracle."""
    g = G.make_grid(60, 13)
    br = next(k for k in range(g.n_branch)
              if g.bus_type[g.from_bus[k]] == G.PQ and g.bus_type[g.to_bus[k]] == G.PQ)
    f, t = int(g.from_bus[br]), int(g.to_bus[br])
    y = 1.0 / (g.r[br] + 1j * g.x[br])
    tap = np.exp(1j * 0.15)
    row = np.concatenate([g.Y_row, [f, t]]).astype(np.int32)
    col = np.concatenate([g.Y_col, [t, f]]).astype(np.int32)
    val = np.concatenate([g.Y_val, [y - y / np.conj(tap), y - y / tap]])
    Y = O.dense_Y(g.N, row, col, val)
    assert np.abs(Y - Y.T).max() > 1.0
    P, Q = G.make_injections(g, 6)
    ref = O.solve_batch(g.N, row, col, val, g.bus_type, g.v_set, P, Q)
    assert ref["converged"].all()
    net = zbus.NrNetwork(g.N, row, col, val, g.bus_type, g.v_set)
    V, it, cv, gm = net.solve(dev(P), dev(Q), precision=prec)
    np.testing.assert_array_equal(cv.cpu().numpy(), ref["converged"])
    assert np.abs(V.cpu().numpy() - ref["V"]).max() <= TOL_TIGHT
    assert np.abs(it.cpu().numpy() - ref["iters"]).max() <= 1


def test_golden_grid14():
    """The GPU against the stored Newton-Raphson oracle solution."""
    import json
    import os
    gd = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "grid14_b4.json")))
    g = G.make_grid(14, 1)
    P, Q = G.make_injections(g, 4)
    net = zbus.NrNetwork.from_grid(g)
    V, it, cv, gm = net.solve(dev(P), dev(Q), tol=gd["tol"], max_iter=gd["max_iter"])
    Vg = np.asarray(gd["V_re"]) + 1j * np.asarray(gd["V_im"])
    np.testing.assert_array_equal(cv.cpu().numpy(), gd["converged"])
    assert np.abs(V.cpu().numpy() - Vg).max() <= TOL_TIGHT
