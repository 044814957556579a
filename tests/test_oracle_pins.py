"""Pins of the FP64 oracle against facts fixed by physics and mathematics.

None of these tests retypes the oracle's formulas: each compares it with a
closed form, a conservation law, a structural identity or an independent
solver (brute-force Newton-Raphson).
"""
import numpy as np
import pytest

from oracle import zbus_oracle as O
from paper_2605_14103_gb300 import feeders as F
from tests import ref_newton

A = np.exp(2j * np.pi / 3)
ROT = np.array([1.0, A.conjugate(), A])


def two_bus(zs, zm, S, rule="maxabs", tol=1e-12, max_iter=200, delta=False):
    z = np.full((3, 3), zm, dtype=np.complex128)
    np.fill_diagonal(z, zs)
    y = np.linalg.inv(z)
    Y = np.block([[y, -y], [-y, y]])
    Y_LL, Y_Ls, _ = O.partition(Y, [0, 1, 2])
    Zr, w = O.reduced_impedance(Y_LL, Y_Ls, ROT)
    Sv = np.full((1, 3), S, dtype=np.complex128)
    zero = np.zeros((1, 3), dtype=np.complex128)
    if delta:
        out = O.fixed_point(Zr, w, zero, Sv, tol, max_iter, rule=rule)
    else:
        out = O.fixed_point(Zr, w, Sv, zero, tol, max_iter, rule=rule)
    return out, Zr, w


def closed_form_two_bus(zs, zm, S):
    """High-voltage root of v = 1 - z1 conj(S / v), z1 = zs - zm (balanced operation).

    Conjugating and writing u = |v|^2 gives v = u + conj(z1) S and
    u^2 + (2 Re(conj(z1) S) - 1) u + |z1|^2 |S|^2 = 0.
    """
    z1 = zs - zm
    b = 1.0 - 2.0 * (z1.conjugate() * S).real
    u = 0.5 * (b + np.sqrt(b * b - 4.0 * abs(z1) ** 2 * abs(S) ** 2))
    va = u + z1.conjugate() * S
    return va * ROT


@pytest.mark.parametrize("seed", range(6))
def test_two_bus_closed_form(seed):
    rng = np.random.default_rng(seed)
    zs = complex(rng.uniform(0.01, 0.05), rng.uniform(0.02, 0.1))
    zm = complex(rng.uniform(0.0, 0.4), rng.uniform(0.0, 0.4)) * zs
    S = complex(rng.uniform(0.5, 2.0), rng.uniform(0.1, 0.8))
    (V, it, cv), _, _ = two_bus(zs, zm, S)
    assert cv[0] == 1
    np.testing.assert_allclose(V[0], closed_form_two_bus(zs, zm, S), rtol=0, atol=1e-12)


def test_two_bus_delta_closed_form():
    # a balanced delta of S per branch draws the same phase currents as a
    # balanced wye of S per phase, so the same closed form holds
    zs, zm, S = 0.03 + 0.07j, 0.01 + 0.02j, 1.3 + 0.5j
    (V, it, cv), _, _ = two_bus(zs, zm, S, delta=True)
    assert cv[0] == 1
    np.testing.assert_allclose(V[0], closed_form_two_bus(zs, zm, S), rtol=0, atol=1e-12)


@pytest.mark.parametrize("rule", ["maxabs", "summag"])
@pytest.mark.parametrize("tol", [1e-3, 1e-6, 1e-9, 1e-12])
def test_two_bus_iteration_count(rule, tol):
    """Iteration count and stop rule against the scalar recursion of phase a."""
    zs, zm, S = 0.04 + 0.08j, 0.01 + 0.03j, 1.5 + 0.6j
    z1 = zs - zm
    u = [1.0 + 0j]
    for _ in range(200):
        u.append(1.0 - z1 * np.conj(S / u[-1]))
    u = np.array(u)
    if rule == "maxabs":
        d = np.abs(np.diff(u))
    else:
        d = 3.0 * np.abs(np.diff(np.abs(u)))
    assert np.min(np.abs(d / tol - 1.0)) > 1e-3, "tol too close to an increment"
    expect = int(np.argmax(d <= tol)) + 1
    (V, it, cv), _, _ = two_bus(zs, zm, S, rule=rule, tol=tol)
    assert cv[0] == 1
    assert it[0] == expect
    np.testing.assert_allclose(V[0, 0], u[expect], atol=1e-14)


def test_two_bus_contraction_rate():
    """Increments shrink geometrically at |z1||S|/|v|^2, the derivative of the map."""
    zs, zm, S = 0.04 + 0.08j, 0.01 + 0.03j, 1.5 + 0.6j
    z1 = zs - zm
    va = closed_form_two_bus(zs, zm, S)[0]
    rate = abs(z1) * abs(S) / abs(va) ** 2
    z = np.full((3, 3), zm, dtype=np.complex128)
    np.fill_diagonal(z, zs)
    y = np.linalg.inv(z)
    Y = np.block([[y, -y], [-y, y]])
    Y_LL, Y_Ls, _ = O.partition(Y, [0, 1, 2])
    Zr, w = O.reduced_impedance(Y_LL, Y_Ls, ROT)
    V = w[None, :].copy()
    Sv = np.full((1, 3), S)
    zero = np.zeros((1, 3), dtype=np.complex128)
    incs = []
    for _ in range(12):
        Vn, _, _ = O.fixed_point(Zr, w, Sv, zero, 0.0, 1, V0=V)
        incs.append(np.abs(Vn - V).max())
        V = Vn
    ratios = np.array(incs[5:]) / np.array(incs[4:-1])
    np.testing.assert_allclose(ratios, rate, rtol=1e-3)


def test_balanced_delta_current_equals_wye():
    rng = np.random.default_rng(7)
    B, nb = 4, 5
    va = (rng.uniform(0.9, 1.05, (B, nb)) * np.exp(1j * rng.uniform(-0.2, 0.2, (B, nb))))
    V = (va[..., None] * ROT).reshape(B, 3 * nb)
    s = rng.uniform(0.1, 1, (B, nb)) + 1j * rng.uniform(0, 0.5, (B, nb))
    S = np.repeat(s, 3, axis=1)
    zero = np.zeros_like(S)
    np.testing.assert_allclose(O.load_currents(V, zero, S), O.load_currents(V, S, zero),
                               rtol=0, atol=1e-14)


@pytest.mark.parametrize("branch", [0, 1, 2])
def test_single_delta_branch_physics(branch):
    """A lone branch xy draws I from phase x, returns it at phase y, consumes S_xy."""
    rng = np.random.default_rng(11 + branch)
    V = (rng.uniform(0.8, 1.1, (3, 6)) * np.exp(1j * rng.uniform(-3, 3, (3, 6))))
    S = np.zeros((3, 6), dtype=np.complex128)
    s = rng.uniform(0.2, 1.0, 3) + 1j * rng.uniform(-0.5, 0.5, 3)
    S[:, 3 + branch] = s                      # bus 1 of 2
    drawn = -O.load_currents(V, np.zeros_like(S), S)
    x, y = branch, (branch + 1) % 3
    other = (branch + 2) % 3
    assert np.all(drawn[:, :3] == 0)
    np.testing.assert_allclose(drawn[:, 3 + other], 0, atol=1e-15)
    np.testing.assert_allclose(drawn[:, 3 + x], -drawn[:, 3 + y], atol=1e-15)
    vxy = V[:, 3 + x] - V[:, 3 + y]
    np.testing.assert_allclose(vxy * np.conj(drawn[:, 3 + x]), s, rtol=1e-13)


def test_delta_bus_power_balance():
    """Sum over phases of v_p conj(drawn_p) equals the bus's total delta power."""
    rng = np.random.default_rng(3)
    V = rng.uniform(0.8, 1.1, (5, 12)) * np.exp(1j * rng.uniform(-3, 3, (5, 12)))
    S = rng.uniform(0.1, 1, (5, 12)) + 1j * rng.uniform(-0.3, 0.6, (5, 12))
    drawn = -O.load_currents(V, np.zeros_like(S), S)
    p = (V * np.conj(drawn)).reshape(5, 4, 3).sum(-1)
    np.testing.assert_allclose(p, S.reshape(5, 4, 3).sum(-1), rtol=1e-12)


def test_wye_power():
    rng = np.random.default_rng(4)
    V = rng.uniform(0.8, 1.1, (5, 9)) * np.exp(1j * rng.uniform(-3, 3, (5, 9)))
    S = rng.uniform(0.1, 1, (5, 9)) + 1j * rng.uniform(-0.3, 0.6, (5, 9))
    S[0, 4] = 0
    drawn = -O.load_currents(V, S, np.zeros_like(S))
    np.testing.assert_allclose(V * np.conj(drawn), S, rtol=1e-13, atol=0)
    assert drawn[0, 4] == 0


@pytest.mark.parametrize("N,seed", [(13, 101), (128, 202)])
def test_no_load_voltage_is_slack(N, seed):
    """Series-only lines: every row of Y sums to zero, so w = v_s on every bus."""
    f = F.make_feeder(N, seed, delta_frac=0.3)
    Y = O.dense_from_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val)
    Y_LL, Y_Ls, _ = O.partition(Y, f.slack_idx)
    _, w = O.reduced_impedance(Y_LL, Y_Ls, f.v_slack)
    np.testing.assert_allclose(w, np.tile(f.v_slack, N - 1), atol=1e-11)


def lca_impedance(f):
    """Z[(i,p),(j,q)] = sum of z_e[p,q] over lines e shared by the paths slack->i and slack->j."""
    paths = [set()]
    for k in range(1, f.N):
        paths.append(paths[f.parent[k]] | {k})
    n = f.n
    Z = np.zeros((n, n), dtype=np.complex128)
    for i in range(1, f.N):
        for j in range(1, f.N):
            common = paths[i] & paths[j]
            if common:
                blk = sum(f.z_line[e] for e in common)
                Z[3 * (i - 1):3 * i, 3 * (j - 1):3 * j] = blk
    return Z


@pytest.mark.parametrize("N,seed", [(2, 1), (9, 2), (40, 3)])
def test_reduced_impedance_lca(N, seed):
    f = F.make_feeder(N, seed)
    Y = O.dense_from_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val)
    Y_LL, Y_Ls, _ = O.partition(Y, f.slack_idx)
    Z, _ = O.reduced_impedance(Y_LL, Y_Ls, f.v_slack)
    Zl = lca_impedance(f)
    np.testing.assert_allclose(Z, Zl, rtol=0, atol=1e-12 * np.abs(Zl).max())


@pytest.mark.parametrize("N,seed,kappa", [(2, 21, 40.0), (3, 22, 25.0), (4, 23, 20.0), (6, 24, 12.0)])
def test_against_bruteforce_newton(N, seed, kappa):
    f = F.make_feeder(N, seed, delta_frac=0.5, kappa=kappa)
    S_wye, S_del = F.make_scenarios(f, 3, 0.8, 1.2)
    r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack,
                    S_wye, S_del, tol=1e-14, max_iter=2000)
    assert r["converged"].all()
    assert np.abs(r["V"]).min() < 0.97          # the loads are not negligible
    for b in range(3):
        v, res = ref_newton.newton_solve(r["Y_LL"], r["Y_Ls"], f.v_slack, S_wye[b], S_del[b],
                                         r["w"])
        assert res < 1e-11
        np.testing.assert_allclose(r["V"][b], v, rtol=0, atol=1e-10)


@pytest.mark.parametrize("name,B", [("feeder13_b8", 8), ("feeder128_b4096", 256)])
def test_power_mismatch_invariant(name, B):
    f, Sw, Sd, w = F.make_workload(name, B=B)
    r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                    tol=w.tol, max_iter=w.max_iter)
    assert r["converged"].all()
    mm = O.power_mismatch(r["Y_LL"], r["Y_Ls"], f.v_slack, r["V"], Sw, Sd)
    assert mm.max() <= 1e-6
    # and the mismatch of the start (no-load voltage) is large: the check bites
    V0 = np.broadcast_to(r["w"], Sw.shape)
    assert O.power_mismatch(r["Y_LL"], r["Y_Ls"], f.v_slack, V0, Sw, Sd).min() > 1e-3


def test_zero_load():
    f, Sw, Sd, w = F.make_workload("feeder13_b8")
    z = np.zeros_like(Sw)
    r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, z, z)
    assert (r["iters"] == 1).all() and r["converged"].all()
    np.testing.assert_array_equal(r["V"], np.broadcast_to(r["w"], Sw.shape))


def test_divergence_is_flagged():
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=6)
    Sw = Sw * 60.0
    Sd = Sd * 60.0
    Sw[0] /= 60.0
    Sd[0] /= 60.0
    r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                    tol=1e-8, max_iter=40)
    assert r["converged"][0] == 1
    assert not r["converged"][1:].any()
    assert (r["iters"] <= 40).all()


def test_scenario_independence():
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=64)
    full = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd)
    idx = np.array([5, 17, 40, 63])
    part = O.fixed_point(full["Z"], full["w"], Sw[idx], Sd[idx], 1e-8, 50)
    np.testing.assert_allclose(part[0], full["V"][idx], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(part[1], full["iters"][idx])


def test_summag_rule_reaches_same_solution():
    f, Sw, Sd, w = F.make_workload("feeder13_b8")
    a = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                    tol=1e-12, rule="maxabs")
    b = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                    tol=1e-12, rule="summag")
    assert a["converged"].all() and b["converged"].all()
    np.testing.assert_allclose(a["V"], b["V"], atol=1e-10)


def test_coo_duplicates_are_summed():
    row = np.array([0, 0, 1, 1, 0])
    col = np.array([0, 1, 0, 1, 0])
    val = np.array([1 + 1j, 2, 3, 4, 5j])
    Y = O.dense_from_coo(2, row, col, val)
    np.testing.assert_array_equal(Y, np.array([[1 + 6j, 2], [3, 4]]))


def test_nonsymmetric_admittance_against_newton():
    """A non-reciprocal network (Y != Y^T, as with a phase-shifting element).

    Feeder matrices are symmetric, so a transposed Z would go unnoticed there;
    here the fixed point must still agree with Newton-Raphson on Y itself.
    """
    rng = np.random.default_rng(5)
    n = 9
    Y_LL = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) * 2.0
    Y_LL += np.diag(40.0 - 60.0j + rng.normal(size=n))
    T = np.tile(np.eye(3), (n // 3, 1))                  # bus-phase j -> slack phase j % 3
    Y_Ls = -Y_LL @ T + (rng.normal(size=(n, 3)) + 1j * rng.normal(size=(n, 3))) * 0.3
    assert np.abs(Y_LL - Y_LL.T).max() > 1.0
    Z, w = O.reduced_impedance(Y_LL, Y_Ls, ROT)
    S_wye = (rng.uniform(0.5, 2.0, (2, n)) + 1j * rng.uniform(0.1, 0.6, (2, n))) * 0.4
    S_del = np.zeros_like(S_wye)
    S_del[:, 3:6] = S_wye[:, 3:6]
    S_wye[:, 3:6] = 0
    V, it, cv = O.fixed_point(Z, w, S_wye, S_del, 1e-14, 500)
    assert cv.all()
    for b in range(2):
        v, res = ref_newton.newton_solve(Y_LL, Y_Ls, ROT, S_wye[b], S_del[b], w)
        assert res < 1e-11
        np.testing.assert_allclose(V[b], v, rtol=0, atol=1e-10)
    assert O.power_mismatch(Y_LL, Y_Ls, ROT, V, S_wye, S_del).max() < 1e-10


def test_golden_feeder13_regression():
    """The stored oracle solution (written by tests/golden/write_golden.py) still holds."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "feeder13_b8.json")))
    f, Sw, Sd, w = F.make_workload("feeder13_b8")
    r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                    tol=g["tol"], max_iter=g["max_iter"])
    V = np.array(g["V_re"]) + 1j * np.array(g["V_im"])
    np.testing.assert_allclose(r["V"], V, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(r["iters"], g["iters"])
    np.testing.assert_array_equal(r["converged"], g["converged"])
