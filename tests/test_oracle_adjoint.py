"""Pins of the oracle's load gradient (solve_adjoint) on the CPU.

The gradient of a real loss L(v*(S)) with respect to the loads is checked
against quantities computed without it: central finite differences of the
forward fixed point (along random complex directions, and entry by entry on
a tiny feeder), the derivative of the two-bus closed-form solution, and on
partial-phase feeders.  Convention: grad = dL/dRe + j dL/dIm, so
dL = Re(sum conj(grad) dS).
"""
import numpy as np
import pytest

from oracle import zbus_oracle as O
from paper_2605_14103_gb300 import feeders as F
from tests.test_oracle_pins import ROT, closed_form_two_bus


def forward(f, Sw, Sd, bus_phase=None):
    r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd,
                    tol=1e-15, max_iter=400, bus_phase=bus_phase)
    assert r["converged"].all() or np.isfinite(r["V"]).all()
    return r


def loss(V, G):
    return float(np.real(np.sum(np.conj(G) * V)))


def fd_directional(f, Sw, Sd, G, dW, dD, h, bus_phase=None):
    lp = loss(forward(f, Sw + h * dW, Sd + h * dD, bus_phase)["V"], G)
    lm = loss(forward(f, Sw - h * dW, Sd - h * dD, bus_phase)["V"], G)
    return (lp - lm) / (2 * h)


@pytest.mark.parametrize("N,seed,delta", [(5, 11, 0.0), (9, 12, 0.5), (13, 13, 0.4)])
def test_directional_derivative_matches_finite_differences(N, seed, delta):
    f = F.make_feeder(N, seed, delta_frac=delta)
    Sw, Sd = F.make_scenarios(f, 2, 0.8, 1.2)
    r = forward(f, Sw, Sd)
    assert r["converged"].all()
    rng = np.random.default_rng(seed)
    G = rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G)
    scale = np.abs(Sw + Sd).max()
    for which in ("wye", "delta"):
        d = (rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)) * scale
        # delta directions also apply where no delta load sits (delta = 0)
        dW, dD = (d, 0 * d) if which == "wye" else (0 * d, d)
        fd = fd_directional(f, Sw, Sd, G, dW, dD, 1e-5)
        H = Hw if which == "wye" else Hd
        ad = float(np.real(np.sum(np.conj(H) * d)))
        assert abs(ad - fd) <= 1e-7 * max(1.0, abs(fd)), (which, ad, fd)


def test_every_entry_on_a_three_bus_feeder():
    f = F.make_feeder(3, 5, delta_frac=0.0)
    Sw, Sd = F.make_scenarios(f, 1, 0.8, 1.2)
    Sd = Sw.copy() * 0.7          # delta loads on every bus as well
    r = forward(f, Sw, Sd)
    rng = np.random.default_rng(0)
    G = rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G)
    h = 1e-6
    for H, wye in ((Hw, True), (Hd, False)):
        for j in range(f.n):
            for unit in (1.0, 1j):
                d = np.zeros_like(Sw)
                d[0, j] = unit
                fd = fd_directional(f, Sw, Sd, G, d if wye else 0 * d, 0 * d if wye else d, h)
                ad = float(np.real(np.conj(H[0, j]) * unit))
                assert abs(ad - fd) <= 1e-6 * max(1.0, abs(fd)), (wye, j, unit, ad, fd)


@pytest.mark.parametrize("seed", range(4))
def test_two_bus_closed_form_derivative(seed):
    """Balanced wye load S on the three phases of a one-line feeder: the
    closed-form voltage v_a(S) differentiated by central differences (no
    fixed point, no Z) against the adjoint's gradient summed over the phases."""
    rng = np.random.default_rng(100 + seed)
    zs = complex(rng.uniform(0.01, 0.05), rng.uniform(0.02, 0.1))
    zm = complex(rng.uniform(0.0, 0.4), rng.uniform(0.0, 0.4)) * zs
    S = complex(rng.uniform(0.5, 2.0), rng.uniform(0.1, 0.8))
    z = np.full((3, 3), zm, dtype=np.complex128)
    np.fill_diagonal(z, zs)
    y = np.linalg.inv(z)
    Y = np.block([[y, -y], [-y, y]])
    Y_LL, Y_Ls, _ = O.partition(Y, [0, 1, 2])
    Z, w = O.reduced_impedance(Y_LL, Y_Ls, closed_form_two_bus(zs, zm, 0.0))
    V = closed_form_two_bus(zs, zm, S)[None, :]
    g = complex(rng.normal(), rng.normal())
    G = np.array([[g, 0, 0]], dtype=np.complex128)       # L = Re(conj(g) v_a)
    Sw = np.full((1, 3), S)
    Hw, _ = O.solve_adjoint(Z, V, Sw, 0 * Sw, G)
    Hs = Hw[0].sum()                                        # balanced direction
    h = 1e-6

    def L(s):
        return float(np.real(np.conj(g) * closed_form_two_bus(zs, zm, s)[0]))

    dP = (L(S + h) - L(S - h)) / (2 * h)
    dQ = (L(S + 1j * h) - L(S - 1j * h)) / (2 * h)
    np.testing.assert_allclose([Hs.real, Hs.imag], [dP, dQ], rtol=1e-7, atol=1e-9)


def test_gradient_is_real_linear_in_G():
    f = F.make_feeder(7, 3, delta_frac=0.5)
    Sw, Sd = F.make_scenarios(f, 2, 0.8, 1.2)
    r = forward(f, Sw, Sd)
    rng = np.random.default_rng(1)
    G1 = rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)
    G2 = rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)
    a = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G1)
    b = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G2)
    c = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, 2.5 * G1 - 0.75 * G2)
    for x, y, z in zip(a, b, c):
        np.testing.assert_allclose(z, 2.5 * x - 0.75 * y, rtol=0, atol=1e-11)
    zero = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, 0 * G1)
    assert not np.any(zero[0]) and not np.any(zero[1])


@pytest.mark.parametrize("N,seed", [(6, 21), (12, 22)])
def test_partial_phase_feeder_directional(N, seed):
    f = F.make_partial_feeder(N, seed, lateral_frac=1.0, delta_frac=0.5)
    Sw, Sd = F.make_partial_scenarios(f, 2, 0.8, 1.2)
    assert (f.phases.sum(axis=1) < 3).any()
    r = forward(f, Sw, Sd, f.bus_phase)
    assert r["converged"].all()
    bp = r["bus_phase"]
    rng = np.random.default_rng(seed)
    G = rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)
    Hw, Hd = O.solve_adjoint(r["Z"], r["V"], Sw, Sd, G, bus_phase=bp)
    # delta directions only where the branch has both phases (else no load)
    where = {int(g): j for j, g in enumerate(bp)}
    valid = np.array([(3 * (g // 3) + (g % 3 + 1) % 3) in where for g in bp])
    assert not np.any(Hd[:, ~valid])
    scale = np.abs(Sw + Sd).max()
    for wye in (True, False):
        d = (rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)) * scale
        if not wye:
            d[:, ~valid] = 0
        fd = fd_directional(f, Sw, Sd, G, d if wye else 0 * d, 0 * d if wye else d, 1e-5, f.bus_phase)
        H = Hw if wye else Hd
        ad = float(np.real(np.sum(np.conj(H) * d)))
        assert abs(ad - fd) <= 1e-7 * max(1.0, abs(fd)), (wye, ad, fd)


def test_nonsymmetric_admittance_directional():
    """A non-reciprocal network (Y != Y^T): feeder matrices are symmetric, so a
    transposed Z in the gradient would go unnoticed on them."""
    rng = np.random.default_rng(5)
    n = 9
    rot = ROT
    Y_LL = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) * 2.0
    Y_LL += np.diag(40.0 - 60.0j + rng.normal(size=n))
    T = np.tile(np.eye(3), (n // 3, 1))
    Y_Ls = -Y_LL @ T + (rng.normal(size=(n, 3)) + 1j * rng.normal(size=(n, 3))) * 0.3
    assert np.abs(Y_LL - Y_LL.T).max() > 1.0
    Z, w = O.reduced_impedance(Y_LL, Y_Ls, rot)
    Sw = (rng.uniform(0.5, 2.0, (2, n)) + 1j * rng.uniform(0.1, 0.6, (2, n))) * 0.4
    Sd = np.zeros_like(Sw)
    Sd[:, 3:6] = Sw[:, 3:6]
    Sw[:, 3:6] = 0
    V, _, cv = O.fixed_point(Z, w, Sw, Sd, 1e-15, 500)
    assert cv.all()
    G = rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)
    Hw, Hd = O.solve_adjoint(Z, V, Sw, Sd, G)
    h = 1e-5
    for wye in (True, False):
        d = rng.normal(size=Sw.shape) + 1j * rng.normal(size=Sw.shape)
        dW, dD = (d, 0 * d) if wye else (0 * d, d)
        Lp = loss(O.fixed_point(Z, w, Sw + h * dW, Sd + h * dD, 1e-15, 500)[0], G)
        Lm = loss(O.fixed_point(Z, w, Sw - h * dW, Sd - h * dD, 1e-15, 500)[0], G)
        fd = (Lp - Lm) / (2 * h)
        H = Hw if wye else Hd
        ad = float(np.real(np.sum(np.conj(H) * d)))
        assert abs(ad - fd) <= 1e-7 * max(1.0, abs(fd)), (wye, ad, fd)
