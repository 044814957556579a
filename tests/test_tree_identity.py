"""The radial-feeder identity behind the tree-sweep form (CPU).

For a feeder whose buses form a tree hanging off the slack with series
branches only, Y_LL^{-1} r is a backward sweep (the sum of r over the subtree
of every bus) followed by a forward sweep (x_c = x_parent + z_c S_c, with z_c
the series impedance of the branch joining c to its parent and x = 0 at the
slack).  The sweep is written here from that statement, independently of the
CUDA kernels, and checked against the oracle's dense inverse.  With shunts
the sweep inverts only the series part; the defect iteration
v <- v + T r(v) then still lands on the oracle's fixed point.
"""
import numpy as np
import pytest

from oracle import zbus_oracle as O
from paper_2605_14103_gb300 import feeders as F


def blk(M, a, b):
    return M[3 * a:3 * a + 3, 3 * b:3 * b + 3]


def bus_tree(Y_LL, Y_Ls):
    """Breadth-first order, parents and parent-branch impedances of the buses."""
    nb = Y_LL.shape[0] // 3
    nbrs = [[b for b in range(nb) if b != a and np.abs(blk(Y_LL, a, b)).max() > 0]
            for a in range(nb)]
    roots = [a for a in range(nb) if np.abs(Y_Ls[3 * a:3 * a + 3]).max() > 0]
    par = {a: -1 for a in roots}
    order = list(roots)
    for a in order:
        for b in nbrs[a]:
            if b == par[a]:
                continue
            if b in par:
                raise ValueError("meshed")
            par[b] = a
            order.append(b)
    assert len(order) == nb
    z = {c: np.linalg.inv(-(blk(Y_LL, c, par[c]) if par[c] >= 0 else Y_Ls[3 * c:3 * c + 3]))
         for c in order}
    return order, par, z


def tree_apply(order, par, z, r):
    S = r.reshape(-1, 3).copy()
    for c in reversed(order):            # every descendant of c comes after c
        if par[c] >= 0:
            S[par[c]] += S[c]
    X = np.zeros_like(S)
    for c in order:                      # every ancestor of c comes before c
        X[c] = (X[par[c]] if par[c] >= 0 else 0.0) + z[c] @ S[c]
    return X.reshape(-1)


def network(f, shunt=None):
    Y = O.dense_from_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val)
    if shunt is not None:
        for bus, y in shunt.items():         # bus >= 1 (global bus index)
            Y[3 * bus:3 * bus + 3, 3 * bus:3 * bus + 3] += y * np.eye(3)
    Y_LL, Y_Ls, _ = O.partition(Y, f.slack_idx)
    return Y_LL, Y_Ls


@pytest.mark.parametrize("N,seed", [(2, 5), (13, 101), (128, 202), (300, 9)])
def test_tree_sweep_is_the_dense_inverse(N, seed):
    f = F.make_feeder(N, seed, delta_frac=0.3)
    Y_LL, Y_Ls = network(f)
    Z, w = O.reduced_impedance(Y_LL, Y_Ls, f.v_slack)
    order, par, z = bus_tree(Y_LL, Y_Ls)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        r = rng.standard_normal(f.n) + 1j * rng.standard_normal(f.n)
        ref = Z @ r
        assert np.abs(tree_apply(order, par, z, r) - ref).max() <= 1e-10 * np.abs(ref).max()
    # the no-load voltage is the same sweep applied to -Y_Ls v_s
    w_t = tree_apply(order, par, z, -(Y_Ls @ f.v_slack))
    assert np.abs(w_t - w).max() <= 1e-12


def test_tree_parents_follow_the_generator():
    f = F.make_feeder(64, 17)
    Y_LL, Y_Ls = network(f)
    order, par, z = bus_tree(Y_LL, Y_Ls)
    # buses of Y_LL are generator buses 1..N-1; the generator's parent array is
    # the ground truth of the tree
    for c in range(f.N - 1):
        assert par[c] == f.parent[c + 1] - 1
        assert np.allclose(z[c], f.z_line[c + 1], rtol=1e-12, atol=0.0)


def test_meshed_network_has_no_tree():
    f = F.make_feeder(20, 3)
    Y = O.dense_from_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val)
    a, b = 5, 17                        # a tie line between two load buses
    assert f.parent[b] != a and f.parent[a] != b
    y = np.linalg.inv(f.z_line[4])
    Y[3 * a:3 * a + 3, 3 * a:3 * a + 3] += y
    Y[3 * b:3 * b + 3, 3 * b:3 * b + 3] += y
    Y[3 * a:3 * a + 3, 3 * b:3 * b + 3] -= y
    Y[3 * b:3 * b + 3, 3 * a:3 * a + 3] -= y
    Y_LL, Y_Ls, _ = O.partition(Y, f.slack_idx)
    with pytest.raises(ValueError):
        bus_tree(Y_LL, Y_Ls)


def test_defect_iteration_with_the_series_inverse_reaches_the_fixed_point_with_shunts():
    f = F.make_feeder(40, 12, delta_frac=0.4)
    shunt = {b: 0.02j for b in (3, 9, 20, 33)}        # capacitive shunts (pu)
    Y_LL, Y_Ls = network(f, shunt)
    Z, w = O.reduced_impedance(Y_LL, Y_Ls, f.v_slack)
    order, par, z = bus_tree(Y_LL, Y_Ls)              # series part only
    rng = np.random.default_rng(1)
    r = rng.standard_normal(f.n) + 1j * rng.standard_normal(f.n)
    # T is not the inverse any more ...
    assert np.abs(tree_apply(order, par, z, r) - Z @ r).max() > 1e-6 * np.abs(Z @ r).max()
    Sw, Sd = F.make_scenarios(f, 4, 0.8, 1.2, seed=5)
    ref, it_ref, cv_ref = O.fixed_point(Z, w, Sw, Sd, 1e-12, 100)
    assert cv_ref.all()
    ys = Y_Ls @ f.v_slack
    for b in range(4):
        v = w.copy()
        for k in range(100):
            res = O.load_currents(v[None], Sw[b:b + 1], Sd[b:b + 1])[0] - Y_LL @ v - ys
            step = tree_apply(order, par, z, res)
            v = v + step
            if np.abs(step).max() <= 1e-12:
                break
        # ... but the defect form still converges to the oracle's solution
        assert np.abs(v - ref[b]).max() <= 1e-10
