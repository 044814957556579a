"""Pins of the Newton-Raphson oracle (transmission power flow, Sec. II-A).

None of these retypes the oracle: closed forms of two-bus cases (a PQ bus
and a lossless PV bus), central differences of the mismatch map against the
analytic Jacobian, quadratic convergence, an independent root finder on the
rectangular formulation, the Z-bus oracle on the positive-sequence network
of a balanced feeder, and power-balance invariants at the solution.
"""
import numpy as np
import pytest

from oracle import nr_oracle as O
from oracle import zbus_oracle as ZO
from paper_2605_14103_gb300 import feeders as F
from paper_2605_14103_gb300 import grids as G


def two_bus_Y(z, b=0.0):
    y = 1.0 / z
    sh = 0.5j * b
    return np.array([[y + sh, -y], [-y, y + sh]])


@pytest.mark.parametrize("seed", range(5))
def test_two_bus_pq_closed_form(seed):
    """Load S at bus 1 fed from a 1.0 pu slack over z: v = 1 - z conj(S / v);
    with u = |v|^2, conj(v) = u + z conj(S) and u^2 + (2 Re(conj(z) S) - 1) u
    + |z|^2 |S|^2 = 0 (high-voltage root)."""
    rng = np.random.default_rng(seed)
    z = complex(rng.uniform(0.005, 0.05), rng.uniform(0.02, 0.2))
    S = complex(rng.uniform(0.2, 2.0), rng.uniform(0.0, 0.8))
    c = 2.0 * (np.conj(z) * S).real - 1.0
    u = 0.5 * (-c + np.sqrt(c * c - 4.0 * abs(z) ** 2 * abs(S) ** 2))
    v_ref = u + np.conj(z) * S
    Y = two_bus_Y(z)
    bt = np.array([O.SLACK, O.PQ])
    V, it, cv = O.newton(Y, bt, np.array([1.0, 1.0]), np.array([0.0, -S.real]),
                         np.array([0.0, -S.imag]), tol=1e-13)
    assert cv == 1
    assert abs(V[1] - v_ref) < 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_two_bus_lossless_pv_closed_form(seed):
    """Lossless line x, PV bus with |V2| = a and injection P: P = a v1 sin(t2) / x."""
    rng = np.random.default_rng(10 + seed)
    x = rng.uniform(0.05, 0.3)
    v1, a = rng.uniform(0.98, 1.05), rng.uniform(0.98, 1.05)
    P = rng.uniform(-1.5, 1.5)
    Y = two_bus_Y(1j * x)
    bt = np.array([O.SLACK, O.PV])
    V, it, cv = O.newton(Y, bt, np.array([v1, a]), np.array([0.0, P]), np.zeros(2), tol=1e-13)
    assert cv == 1
    assert abs(abs(V[1]) - a) < 1e-14
    assert abs(np.angle(V[1]) - np.arcsin(P * x / (a * v1))) < 1e-12


@pytest.mark.parametrize("N,seed", [(6, 1), (14, 2), (40, 3)])
def test_jacobian_against_central_differences(N, seed):
    g = G.make_grid(N, seed)
    Y = O.dense_Y(N, g.Y_row, g.Y_col, g.Y_val)
    th, q = O.index_sets(g.bus_type)
    rng = np.random.default_rng(seed)
    vm = np.where(g.bus_type == O.PQ, rng.uniform(0.95, 1.05, N), g.v_set)
    va = np.where(g.bus_type == O.SLACK, 0.0, rng.uniform(-0.3, 0.3, N))
    P, Q = G.make_injections(g, 1)

    def F(x):
        a, m = va.copy(), vm.copy()
        a[th] = x[:th.size]
        m[q] = x[th.size:]
        return O.mismatch(Y, m * np.exp(1j * a), P[0], Q[0], th, q)

    x0 = np.concatenate([va[th], vm[q]])
    J = O.jacobian(Y, vm * np.exp(1j * va), th, q)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for k in range(x0.size):
        e = np.zeros_like(x0)
        e[k] = h
        Jfd[:, k] = (F(x0 + e) - F(x0 - e)) / (2 * h)
    np.testing.assert_allclose(J, Jfd, rtol=0, atol=1e-7 * np.abs(J).max())


def test_quadratic_convergence():
    g = G.make_grid(60, 7)
    P, Q = G.make_injections(g, 1)
    Y = O.dense_Y(g.N, g.Y_row, g.Y_col, g.Y_val)
    h = []
    V, it, cv = O.newton(Y, g.bus_type, g.v_set, P[0], Q[0], tol=1e-12, history=h)
    assert cv == 1 and it >= 3
    # once in the basin, |F_{k+1}| <= C |F_k|^2 with a moderate C
    # (steps that end at the rounding floor, |F| < 1e-10, say nothing)
    ratios = [h[k + 1] / h[k] ** 2 for k in range(len(h) - 1) if h[k] < 1e-1 and h[k + 1] > 1e-10]
    assert ratios and max(ratios) < 50.0


@pytest.mark.parametrize("N,seed", [(5, 21), (9, 22), (14, 23)])
def test_against_an_independent_root_finder(N, seed):
    """scipy's MINPACK hybrid solver on the rectangular formulation (e, f per
    non-slack bus; P and Q at PQ buses, P and |V|^2 at PV buses)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    g = G.make_grid(N, seed)
    P, Q = G.make_injections(g, 1)
    P, Q = P[0], Q[0]
    Y = O.dense_Y(N, g.Y_row, g.Y_col, g.Y_val)
    ns = np.arange(1, N)
    vs = g.v_set[0]

    def eqs(z):
        V = np.concatenate([[vs], z[:N - 1] + 1j * z[N - 1:]])
        I = Y @ V
        S = V * np.conj(I)
        out = []
        for i in ns:
            out.append(S[i].real - P[i])
            if g.bus_type[i] == G.PQ:
                out.append(S[i].imag - Q[i])
            else:
                out.append(abs(V[i]) ** 2 - g.v_set[i] ** 2)
        return np.array(out)

    z0 = np.concatenate([np.where(g.bus_type[1:] == G.PQ, 1.0, g.v_set[1:]), np.zeros(N - 1)])
    sol = scipy_opt.root(eqs, z0, method="hybr", tol=1e-14)
    assert sol.success and np.abs(eqs(sol.x)).max() < 1e-11
    V_ref = np.concatenate([[vs], sol.x[:N - 1] + 1j * sol.x[N - 1:]])
    V, it, cv = O.newton(Y, g.bus_type, g.v_set, P, Q, tol=1e-12)
    assert cv == 1
    np.testing.assert_allclose(V, V_ref, rtol=0, atol=1e-10)


def test_positive_sequence_of_a_balanced_feeder_matches_the_zbus_oracle():
    """A radial three-phase feeder with balanced wye loads runs balanced: its
    phase-a voltages are those of the single-phase network with the
    positive-sequence impedance z_self - z_mut and the per-phase loads, every
    bus PQ.  The Z-bus fixed point (another method, another oracle) and
    Newton-Raphson must agree."""
    f = F.make_feeder(25, 31, delta_frac=0.0)
    s = f.base_S[:, 0]                                   # per-phase load of each bus
    Sw = np.repeat(s, 3)[None, :].astype(np.complex128)
    r = ZO.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw,
                     np.zeros_like(Sw), tol=1e-14, max_iter=500)
    assert r["converged"][0] == 1
    va = r["V"][0, 0::3]                                 # phase a of buses 1..N-1
    N = f.N
    rows, cols, vals = [], [], []
    for k in range(1, N):
        z1 = f.z_line[k][0, 0] - f.z_line[k][0, 1]
        y = 1.0 / z1
        p = int(f.parent[k])
        rows += [p, k, p, k]
        cols += [p, k, k, p]
        vals += [y, y, -y, -y]
    Y = O.dense_Y(N, rows, cols, vals)
    bt = np.full(N, O.PQ)
    bt[0] = O.SLACK
    P = np.concatenate([[0.0], -s.real])
    Q = np.concatenate([[0.0], -s.imag])
    V, it, cv = O.newton(Y, bt, np.ones(N), P, Q, tol=1e-13)
    assert cv == 1
    np.testing.assert_allclose(V[1:], va, rtol=0, atol=1e-11)


def test_power_balance_at_the_solution():
    g = G.make_grid(80, 9)
    P, Q = G.make_injections(g, 2)
    r = O.solve_batch(g.N, g.Y_row, g.Y_col, g.Y_val, g.bus_type, g.v_set, P, Q)
    assert r["converged"].all()
    for b in range(2):
        V = r["V"][b]
        S = O.power_injection(r["Y"], V)
        pv = g.bus_type == G.PV
        pq = g.bus_type == G.PQ
        np.testing.assert_allclose(S.real[~(g.bus_type == G.SLACK)],
                                   P[b][~(g.bus_type == G.SLACK)], atol=1e-10)
        np.testing.assert_allclose(S.imag[pq], Q[b][pq], atol=1e-10)
        np.testing.assert_allclose(np.abs(V[pv | (g.bus_type == G.SLACK)]),
                                   g.v_set[pv | (g.bus_type == G.SLACK)], atol=1e-14)
        # losses from the branches equal the sum of the injections
        f, t = g.from_bus, g.to_bus
        ys = 1.0 / (g.r + 1j * g.x)
        Iser = ys * (V[f] - V[t])
        loss_p = float((g.r * np.abs(Iser) ** 2).sum())
        assert abs(S.real.sum() - loss_p) < 1e-9


def test_flat_network_and_divergence():
    g = G.make_grid(20, 4)
    Y = O.dense_Y(g.N, g.Y_row, g.Y_col, g.Y_val)
    # no charging, no injections, all set-points 1: the flat start is the solution
    ch = np.zeros(g.N)
    np.add.at(ch, g.from_bus, 0.5 * g.b)
    np.add.at(ch, g.to_bus, 0.5 * g.b)
    Y0 = Y - np.diag(1j * ch)
    V, it, cv = O.newton(Y0, g.bus_type, np.ones(g.N), np.zeros(g.N), np.zeros(g.N))
    assert cv == 1 and it == 0 and np.allclose(V, 1.0)
    P, Q = G.make_injections(g, 1)
    V, it, cv = O.newton(Y, g.bus_type, g.v_set, 400 * P[0], 400 * Q[0], max_iter=15)
    assert cv == 0


def test_jacobian_and_solution_with_a_phase_shifter():
    """A phase-shifting transformer (complex tap t = e^{j phi}) makes Y
    non-symmetric: Y_ft = -y / conj(t), Y_tf = -y / t.  Grid matrices are
    otherwise symmetric, so a transposed Y in the Jacobian would go unnoticed."""
    g = G.make_grid(30, 12)
    Y = O.dense_Y(g.N, g.Y_row, g.Y_col, g.Y_val)
    # a branch between two PQ buses (rows and columns of both in the Jacobian)
    br = next(k for k in range(g.n_branch)
              if g.bus_type[g.from_bus[k]] == O.PQ and g.bus_type[g.to_bus[k]] == O.PQ)
    f, t = int(g.from_bus[br]), int(g.to_bus[br])
    y = 1.0 / (g.r[br] + 1j * g.x[br])
    tap = np.exp(1j * 0.2)
    Y[f, t] += y - y / np.conj(tap)
    Y[t, f] += y - y / tap
    assert np.abs(Y - Y.T).max() > 1.0
    th, q = O.index_sets(g.bus_type)
    rng = np.random.default_rng(3)
    vm = np.where(g.bus_type == O.PQ, rng.uniform(0.95, 1.05, g.N), g.v_set)
    va = np.where(g.bus_type == O.SLACK, 0.0, rng.uniform(-0.3, 0.3, g.N))
    P, Q = G.make_injections(g, 1)

    def F(x):
        a, m = va.copy(), vm.copy()
        a[th] = x[:th.size]
        m[q] = x[th.size:]
        return O.mismatch(Y, m * np.exp(1j * a), P[0], Q[0], th, q)

    x0 = np.concatenate([va[th], vm[q]])
    J = O.jacobian(Y, vm * np.exp(1j * va), th, q)
    h = 1e-6
    Jfd = np.stack([(F(x0 + h * e) - F(x0 - h * e)) / (2 * h) for e in np.eye(x0.size)], axis=1)
    np.testing.assert_allclose(J, Jfd, rtol=0, atol=1e-7 * np.abs(J).max())
    V, it, cv = O.newton(Y, g.bus_type, g.v_set, P[0], Q[0], tol=1e-12)
    assert cv == 1 and it <= 8


@pytest.mark.parametrize("N,seed", [(118, 611), (1354, 612)])
def test_grid_generator_structure(N, seed):
    g = G.make_grid(N, seed)
    # connected: a search from the slack reaches every bus
    adj = [[] for _ in range(N)]
    for f, t in zip(g.from_bus, g.to_bus):
        adj[f].append(t)
        adj[t].append(f)
    seen, stack = {0}, [0]
    while stack:
        a = stack.pop()
        for b in adj[a]:
            if b not in seen:
                seen.add(b)
                stack.append(b)
    assert len(seen) == N
    assert 1.3 <= g.n_branch / N <= 1.7
    assert (g.bus_type == G.SLACK).sum() == 1 and g.bus_type[0] == G.SLACK
    assert abs((g.bus_type == G.PV).sum() - round(0.15 * N)) <= 1
    Y = O.dense_Y(N, g.Y_row, g.Y_col, g.Y_val)
    np.testing.assert_allclose(Y, Y.T, rtol=0, atol=1e-9)
    assert (g.x > 0).all() and (g.r > 0).all() and (g.b >= 0).all()
    # scenarios: loads within +-20 %, generation scaled with the total load
    P, Q = G.make_injections(g, 50)
    mult = np.divide(-Q, g.Q_load[None, :], out=np.ones_like(Q), where=g.Q_load[None, :] > 0)
    assert mult.min() >= 0.8 - 1e-12 and mult.max() <= 1.2 + 1e-12
    pl = mult * g.P_load[None, :]
    gen_total = (P + pl).sum(axis=1)
    np.testing.assert_allclose(gen_total, pl.sum(axis=1) * g.P_gen.sum() / g.P_load.sum(),
                               rtol=1e-12)


def test_golden_grid14_regression():
    """The stored Newton-Raphson oracle solution (tests/golden/write_golden.py) still holds."""
    import json
    import os
    gd = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "grid14_b4.json")))
    g = G.make_grid(14, 1)
    P, Q = G.make_injections(g, 4)
    r = O.solve_batch(g.N, g.Y_row, g.Y_col, g.Y_val, g.bus_type, g.v_set, P, Q,
                      tol=gd["tol"], max_iter=gd["max_iter"])
    V = np.asarray(gd["V_re"]) + 1j * np.asarray(gd["V_im"])
    np.testing.assert_allclose(r["V"], V, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(r["iters"], gd["iters"])
    np.testing.assert_array_equal(r["converged"], gd["converged"])
