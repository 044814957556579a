"""Pins of the oracle on partial-phase feeders (single- and two-phase laterals).

As for three-phase feeders, none of these retypes the oracle: a closed form
for a single-phase line, an independent brute-force Newton-Raphson with its
own load model, the power-mismatch invariant, and the reading the CUDA
library uses (every bus padded to three phase slots, absent phases isolated
with a unit self-admittance) against the oracle's direct phased solve.
"""
import numpy as np
import pytest

from oracle import zbus_oracle as O
from paper_2605_14103_gb300 import feeders as F
from tests import ref_newton
from tests.test_oracle_pins import closed_form_two_bus


def solve(f, Sw, Sd, **kw):
    return O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                       bus_phase=f.bus_phase, **kw)


@pytest.mark.parametrize("seed", range(4))
def test_single_phase_line_closed_form(seed):
    # slack (three phases, compact 0..2) and one load bus on phase a only
    rng = np.random.default_rng(seed)
    z = complex(rng.uniform(0.01, 0.05), rng.uniform(0.02, 0.1))
    S = complex(rng.uniform(0.5, 2.0), rng.uniform(0.1, 0.8))
    y = 1.0 / z
    row = [0, 3, 0, 3]
    col = [0, 3, 3, 0]
    val = [y, y, -y, -y]
    bp = np.array([0, 1, 2, 3], dtype=np.int32)
    r = O.solve_coo(4, row, col, val, [0, 1, 2], F.V_SLACK, np.array([[S]]),
                    np.zeros((1, 1)), tol=1e-13, max_iter=300, bus_phase=bp)
    assert r["converged"][0] == 1
    ref = closed_form_two_bus(z, 0.0, S)[0]          # v = 1 - z conj(S / v)
    np.testing.assert_allclose(r["V"][0, 0], ref, rtol=0, atol=1e-12)


def test_three_phase_map_equals_triples():
    f = F.make_feeder(40, 8, delta_frac=0.4)
    Sw, Sd = F.make_scenarios(f, 5, 0.8, 1.2)
    bp = np.arange(f.n_total, dtype=np.int32)
    a = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd)
    b = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                    bus_phase=bp)
    np.testing.assert_allclose(b["V"], a["V"], rtol=0, atol=1e-14)
    np.testing.assert_array_equal(b["iters"], a["iters"])


def test_generator_structure():
    f = F.make_partial_feeder(200, 31, lateral_frac=0.5, delta_frac=0.4)
    for k in range(1, f.N):
        assert not (f.phases[k] & ~f.phases[f.parent[k]]).any()   # laterals narrow only
        assert f.phases[k].any()
    Y = O.dense_from_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val)
    np.testing.assert_allclose(Y, Y.T, rtol=0, atol=1e-9)
    assert (f.phases.sum(axis=1) < 3).sum() > 10
    Sw, Sd = F.make_partial_scenarios(f, 3, 0.8, 1.2)
    assert Sw.shape == (3, f.n) and Sd.shape == (3, f.n)
    # delta loads only where all three phases are present
    bp = f.bus_phase[3:]
    for j in np.nonzero(Sd[0])[0]:
        assert f.phases[bp[j] // 3].all()


def test_partial_benchmark_workload_is_the_three_phase_feeder_with_laterals():
    """partial1024_b16384: the tree, impedances and loads of feeder1024_b16384
    (same seed and multipliers) with laterals; three-phase buses keep their
    wye or delta loads, lateral buses carry their loads as wye on the
    present phases."""
    f, Sw, Sd, w = F.make_workload("partial1024_b16384", B=5)
    g, Sw3, Sd3, w3 = F.make_workload("feeder1024_b16384", B=5)
    assert isinstance(f, F.PhasedFeeder) and (w.N, w.B, w.seed) == (w3.N, w3.B, w3.seed)
    np.testing.assert_array_equal(f.parent, g.parent)
    assert f.n < g.n and Sw.shape == (5, f.n) and Sd.shape == (5, f.n)
    bp = f.bus_phase[3:]
    j3 = 3 * (bp // 3 - 1) + bp % 3            # the same (bus, phase) in the three-phase feeder
    three = f.phases[bp // 3].all(axis=1)
    np.testing.assert_array_equal(Sw[:, three], Sw3[:, j3[three]])
    np.testing.assert_array_equal(Sd[:, three], Sd3[:, j3[three]])
    np.testing.assert_array_equal(Sw[:, ~three], (Sw3 + Sd3)[:, j3[~three]])
    assert not Sd[:, ~three].any()


@pytest.mark.parametrize("N,seed,kappa", [(3, 41, 25.0), (5, 42, 15.0), (7, 43, 10.0)])
def test_against_bruteforce_newton(N, seed, kappa):
    base = F.make_partial_feeder(N, seed, lateral_frac=1.0, delta_frac=0.6)
    f = base
    scale = kappa / base.kappa
    f.base_S = base.base_S * scale
    Sw, Sd = F.make_partial_scenarios(f, 3, 0.8, 1.2)
    assert (f.phases.sum(axis=1) < 3).any()
    r = solve(f, Sw, Sd, tol=1e-14, max_iter=3000)
    assert r["converged"].all()
    assert np.abs(r["V"]).min() < 0.98
    for b in range(3):
        v, res = ref_newton.newton_solve(r["Y_LL"], r["Y_Ls"], f.v_slack, Sw[b], Sd[b], r["w"],
                                         bus_phase=f.bus_phase[3:])
        assert res < 1e-11
        np.testing.assert_allclose(r["V"][b], v, rtol=0, atol=1e-10)


def test_power_mismatch_invariant():
    f = F.make_partial_feeder(128, 202, lateral_frac=0.3, delta_frac=0.3, mult_hi=1.5)
    Sw, Sd = F.make_partial_scenarios(f, 32, 0.5, 1.5)
    r = solve(f, Sw, Sd)
    assert r["converged"].all()
    mm = O.power_mismatch(r["Y_LL"], r["Y_Ls"], f.v_slack, r["V"], Sw, Sd, r["bus_phase"])
    assert mm.max() <= 1e-6
    V0 = np.broadcast_to(r["w"], Sw.shape)
    assert O.power_mismatch(r["Y_LL"], r["Y_Ls"], f.v_slack, V0, Sw, Sd,
                            r["bus_phase"]).min() > 1e-3


def pad(f, Sw, Sd):
    """Every bus padded to three phase slots; absent phases isolated (unit self-admittance)."""
    n3 = 3 * f.N
    row = [int(f.bus_phase[r]) for r in f.Y_row]
    col = [int(f.bus_phase[c]) for c in f.Y_col]
    val = list(f.Y_val)
    present = np.zeros(n3, dtype=bool)
    present[f.bus_phase] = True
    for g in np.nonzero(~present)[0]:
        row.append(int(g))
        col.append(int(g))
        val.append(1.0)
    B = Sw.shape[0]
    Pw = np.zeros((B, n3 - 3), dtype=np.complex128)
    Pd = np.zeros((B, n3 - 3), dtype=np.complex128)
    Pw[:, f.bus_phase[3:] - 3] = Sw
    Pd[:, f.bus_phase[3:] - 3] = Sd
    return n3, row, col, val, Pw, Pd


def test_padded_three_phase_network_gives_the_same_solution():
    f = F.make_partial_feeder(60, 77, lateral_frac=0.5, delta_frac=0.4)
    Sw, Sd = F.make_partial_scenarios(f, 6, 0.8, 1.2)
    r = solve(f, Sw, Sd, tol=1e-13, max_iter=200)
    n3, row, col, val, Pw, Pd = pad(f, Sw, Sd)
    q = O.solve_coo(n3, row, col, val, [0, 1, 2], f.v_slack, Pw, Pd, tol=1e-13, max_iter=200)
    assert r["converged"].all() and q["converged"].all()
    real = f.bus_phase[3:] - 3
    np.testing.assert_allclose(q["V"][:, real], r["V"], rtol=0, atol=1e-12)
    virtual = np.setdiff1d(np.arange(n3 - 3), real)
    assert np.abs(q["V"][:, virtual]).max() == 0.0
    np.testing.assert_array_equal(q["iters"], r["iters"])


def test_delta_on_a_missing_branch_is_refused():
    V = np.ones((1, 2), dtype=np.complex128)
    bp = np.array([3, 4])                     # bus 1, phases a and b: branch ab only
    Sd = np.array([[0.0, 0.5 + 0.1j]])        # the bc entry: phase c is absent
    with pytest.raises(ValueError):
        O.load_currents(V, np.zeros((1, 2)), Sd, bp)
