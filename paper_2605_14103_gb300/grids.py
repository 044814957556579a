"""Seeded synthetic meshed transmission grids and load scenarios.

Input recipe of the batched Newton-Raphson power flow (Sec. II-A) shared by
the CUDA path, its tests and the benchmark.  It draws random numbers and
assembles the network description (bus admittance matrix in COO form from
branch pi-models, bus types, voltage set-points, injections); it holds none
of the method's arithmetic (no mismatch, no Jacobian, no Newton step).

The grids stand in for the paper's transmission cases (118-bus, 1354-bus and
the 2224-node GB network, Sec. III), which are not available here: buses at
random points of the unit square, a nearest-neighbour spanning tree plus
extra links to near neighbours (about 1.5 branches per bus, as in those
cases), line reactance growing with length, r/x of 0.1-0.3, line charging,
about 15 % of the buses generators (PV) with one slack, loads on about 70 %
of the buses.  Scenarios multiply every load by its own factor U(0.8, 1.2)
(the paper's +-20 %) and scale the generators' active power with the
scenario's total load, so that the slack takes the losses and a small share.

Per-unit on 100 MVA.  Bus 0 is the slack (angle 0).  Bus types: 0 = PQ,
1 = PV, 2 = slack.
"""
from __future__ import annotations

import dataclasses

import numpy as np

PQ, PV, SLACK = 0, 1, 2


@dataclasses.dataclass
class Grid:
    N: int
    from_bus: np.ndarray      # int32[L]
    to_bus: np.ndarray        # int32[L]
    r: np.ndarray             # float64[L] series resistance (pu)
    x: np.ndarray             # float64[L] series reactance (pu)
    b: np.ndarray             # float64[L] total line charging (pu)
    Y_row: np.ndarray         # int32[nnz] COO of the N x N bus admittance matrix
    Y_col: np.ndarray
    Y_val: np.ndarray         # complex128[nnz]
    bus_type: np.ndarray      # int32[N]
    v_set: np.ndarray         # float64[N] |V| set-point (PV, slack); 1.0 at PQ buses
    P_load: np.ndarray        # float64[N] base active load (pu)
    Q_load: np.ndarray        # float64[N] base reactive load (pu)
    P_gen: np.ndarray         # float64[N] base generation at PV buses (pu)
    seed: int

    @property
    def n_branch(self) -> int:
        return int(self.from_bus.size)


def _assemble_Y(N, fb, tb, r, x, b):
    ys = 1.0 / (r + 1j * x)
    rows, cols, vals = [], [], []
    for f, t, y, bc in zip(fb, tb, ys, b):
        sh = 0.5j * bc
        rows += [f, t, f, t]
        cols += [f, t, t, f]
        vals += [y + sh, y + sh, -y, -y]
    return (np.asarray(rows, dtype=np.int32), np.asarray(cols, dtype=np.int32),
            np.asarray(vals, dtype=np.complex128))


def make_grid(N: int, seed: int, extra_frac: float = 0.5, gen_frac: float = 0.15,
              load_frac: float = 0.7, load_pu: float = 0.25, x_scale: float = 0.08,
              x_cap: float = 0.1, gen_share: float = 1.0) -> Grid:
    """A meshed grid of N buses.

    Draw order from default_rng(seed): positions [N, 2]; extra-link draws;
    r/x ratios, charging factors; generator buses; load presence, load P,
    power factors; generator shares; voltage set-points.  Branch reactance
    x = x_scale * dist * sqrt(N) / 10 pu, clipped to [1e-3, x_cap]: the
    nearest-neighbour distance shrinks as 1 / sqrt(N), so a typical link has
    x of a few thousandths whatever N.  The generators supply gen_share of
    the total load in proportion to Dirichlet shares; the slack takes the
    rest and the losses.
    """
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 2))
    d = np.sqrt(((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1))
    edges = set()
    # spanning tree: each bus k >= 1 links to its nearest bus among 0..k-1
    for k in range(1, N):
        j = int(np.argmin(d[k, :k]))
        edges.add((min(j, k), max(j, k)))
    # extra links: a share of the buses link to their nearest bus not yet linked
    order = np.argsort(d, axis=1)
    extra = rng.random(N) < extra_frac
    for k in np.nonzero(extra)[0]:
        for j in order[k, 1:8]:
            e = (min(int(j), int(k)), max(int(j), int(k)))
            if e not in edges:
                edges.add(e)
                break
    edges = sorted(edges)
    fb = np.array([e[0] for e in edges], dtype=np.int32)
    tb = np.array([e[1] for e in edges], dtype=np.int32)
    L = fb.size
    dist = d[fb, tb]
    x = np.clip(x_scale * dist * np.sqrt(N) / 10.0, 1e-3, x_cap)
    r = x * rng.uniform(0.1, 0.3, size=L)
    b = x * rng.uniform(0.5, 1.5, size=L)
    bus_type = np.zeros(N, dtype=np.int32)
    bus_type[0] = SLACK
    n_gen = max(1, int(round(gen_frac * N)))
    gens = rng.choice(np.arange(1, N), size=min(n_gen, N - 1), replace=False)
    bus_type[gens] = PV
    has_load = rng.random(N) < load_frac
    P_load = np.where(has_load, rng.uniform(0.2, 1.8, size=N) * load_pu, 0.0)
    pf = rng.uniform(0.92, 0.99, size=N)
    Q_load = P_load * np.tan(np.arccos(pf))
    share = rng.dirichlet(np.ones(gens.size))
    P_gen = np.zeros(N)
    P_gen[gens] = gen_share * P_load.sum() * share
    v_set = np.ones(N)
    v_set[bus_type != PQ] = rng.uniform(0.99, 1.04, size=int((bus_type != PQ).sum()))
    Yr, Yc, Yv = _assemble_Y(N, fb, tb, r, x, b)
    return Grid(N=N, from_bus=fb, to_bus=tb, r=r, x=x, b=b, Y_row=Yr, Y_col=Yc, Y_val=Yv,
                bus_type=bus_type, v_set=v_set, P_load=P_load, Q_load=Q_load, P_gen=P_gen,
                seed=seed)


def make_injections(g: Grid, B: int, mult_lo: float = 0.8, mult_hi: float = 1.2,
                    seed: int | None = None):
    """(P, Q), float64[B, N] net injections (generation - load) per scenario.

    One multiplier per (scenario, bus) from default_rng(seed) (default
    g.seed + 1) on that bus's load; generator active power scaled by the
    scenario's total load over the base total.  Q at PV buses and P, Q at
    the slack are outputs of the power flow, not inputs (set here to the
    load's negative, ignored by the solvers).
    """
    if seed is None:
        seed = g.seed + 1
    rng = np.random.default_rng(seed)
    m = rng.uniform(mult_lo, mult_hi, size=(B, g.N))
    Pl = m * g.P_load[None, :]
    Ql = m * g.Q_load[None, :]
    scale = Pl.sum(axis=1, keepdims=True) / max(g.P_load.sum(), 1e-300)
    P = scale * g.P_gen[None, :] - Pl
    Q = -Ql
    return np.ascontiguousarray(P), np.ascontiguousarray(Q)


@dataclasses.dataclass
class GridWorkload:
    name: str
    N: int
    B: int
    seed: int
    tol: float = 1e-10
    max_iter: int = 20


GRID_WORKLOADS = {
    # stand-ins for the paper's 118-bus, 1354-bus and 2224-node cases, batch 1000
    "grid118_b1000": GridWorkload("grid118_b1000", 118, 1000, 611),
    "grid1354_b1000": GridWorkload("grid1354_b1000", 1354, 1000, 612),
    "grid2224_b1000": GridWorkload("grid2224_b1000", 2224, 1000, 613),
}


def make_grid_workload(name: str, B: int | None = None):
    """(grid, P, Q, workload) of a named workload; B overrides the batch."""
    w = GRID_WORKLOADS[name]
    g = make_grid(w.N, w.seed)
    P, Q = make_injections(g, w.B if B is None else B)
    return g, P, Q, w
