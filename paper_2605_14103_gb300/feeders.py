"""Seeded synthetic three-phase radial feeders and load scenarios.

This module is the input recipe shared by the CUDA path, its tests and the
benchmark.  It draws random numbers and assembles the network description
(bus admittance matrix in COO form, slack voltages, constant-power loads); it
holds none of the Z-bus method's arithmetic (no reduced impedance, no load
currents, no fixed point).

Workloads stand in for the paper's IEEE13 / IEEE123 / EULV feeders (Sec. III),
which are not available here: random radial trees with three-phase lines and
constant-PQ wye and delta loads, scenarios formed from random per-bus load
multipliers (Sec. III: batches from random load multipliers turned into
perturbed injection vectors).

Per-unit system: 4.16 kV line-to-line, 1 MVA three-phase base, so the
line-to-neutral voltage base is 4.16/sqrt(3) kV, the per-phase power base is
1/3 MVA and the impedance base is 4.16^2 / 1 = 17.3056 ohm.

Index convention: bus 0 is the slack; bus-phase (k, p) has global index 3k+p in
the full admittance matrix and j = 3(k-1)+p among the n = 3(N-1) non-slack
unknowns.  Delta loads of bus k sit at the three slots of that bus in the
order (ab, bc, ca).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KV_LL = 4.16
MVA_BASE = 1.0
Z_BASE = KV_LL ** 2 / MVA_BASE            # ohm
P_PHASE_BASE_KW = 1000.0 * MVA_BASE / 3.0  # kW per phase
Z_SELF_OHM_KM = 0.3 + 0.6j
Z_MUT_OHM_KM = 0.1 + 0.25j
# Target of the linear voltage-drop estimate used to scale the base loads so
# that the feeder operates near 0.9 pu at the largest multiplier.
DROP_TARGET_PU = 0.08

_A = np.exp(2j * np.pi / 3.0)
V_SLACK = np.array([1.0, _A.conjugate(), _A], dtype=np.complex128)


@dataclasses.dataclass
class Feeder:
    N: int                    # buses including the slack
    parent: np.ndarray        # int64[N], parent[0] = -1
    length_km: np.ndarray     # float64[N], line k joins parent[k] - k; [0] unused
    z_line: np.ndarray        # complex128[N, 3, 3] series impedance (pu); [0] unused
    Y_row: np.ndarray         # int32[nnz]  COO of the full 3N x 3N admittance matrix
    Y_col: np.ndarray         # int32[nnz]
    Y_val: np.ndarray         # complex128[nnz]
    slack_idx: np.ndarray     # int32[3]
    v_slack: np.ndarray       # complex128[3]
    base_S: np.ndarray        # complex128[N-1, 3] base load per slot (pu), kappa applied
    is_delta: np.ndarray      # bool[N-1]
    kappa: float              # load scale applied to the drawn base loads
    seed: int

    @property
    def n(self) -> int:
        return 3 * (self.N - 1)

    @property
    def n_total(self) -> int:
        return 3 * self.N

    def dense_Y(self) -> np.ndarray:
        Y = np.zeros((self.n_total, self.n_total), dtype=np.complex128)
        np.add.at(Y, (self.Y_row, self.Y_col), self.Y_val)
        return Y


def _line_impedance_per_km_pu() -> np.ndarray:
    z = np.full((3, 3), Z_MUT_OHM_KM, dtype=np.complex128)
    np.fill_diagonal(z, Z_SELF_OHM_KM)
    return z / Z_BASE


def _assemble_Y(N: int, parent: np.ndarray, z_line: np.ndarray):
    """Bus admittance matrix of series-only three-phase lines, COO, duplicates summed."""
    blocks = {}

    def add(a, b, y):
        key = (a, b)
        if key in blocks:
            blocks[key] = blocks[key] + y
        else:
            blocks[key] = y.copy()

    for k in range(1, N):
        p = int(parent[k])
        y = np.linalg.inv(z_line[k])
        add(p, p, y)
        add(k, k, y)
        add(p, k, -y)
        add(k, p, -y)
    keys = sorted(blocks)
    nb = len(keys)
    rows = np.empty(nb * 9, dtype=np.int32)
    cols = np.empty(nb * 9, dtype=np.int32)
    vals = np.empty(nb * 9, dtype=np.complex128)
    t = 0
    for (a, b) in keys:
        blk = blocks[(a, b)]
        for p in range(3):
            for q in range(3):
                rows[t] = 3 * a + p
                cols[t] = 3 * b + q
                vals[t] = blk[p, q]
                t += 1
    return rows, cols, vals


def _load_scale(N, parent, length_km, base_S_raw, mult_hi) -> float:
    """kappa = min(1, target / max linear drop) from a LinDistFlow-style estimate.

    Downstream per-phase power of every line times its positive-sequence
    impedance, summed along each path from the slack, with every multiplier at
    its upper bound.  This is a sizing rule for the synthetic loads, not part of
    the power-flow method.
    """
    z1 = (Z_SELF_OHM_KM - Z_MUT_OHM_KM) / Z_BASE
    s_bus = base_S_raw.mean(axis=1) * mult_hi          # per-phase equivalent, [N-1]
    down = np.zeros(N, dtype=np.complex128)
    down[1:] = s_bus
    for k in range(N - 1, 0, -1):
        down[parent[k]] += down[k]
    drop = np.zeros(N)
    for k in range(1, N):
        ze = z1 * length_km[k]
        drop[k] = drop[parent[k]] + ze.real * down[k].real + ze.imag * down[k].imag
    worst = float(drop.max())
    if worst <= DROP_TARGET_PU:
        return 1.0
    return DROP_TARGET_PU / worst


def make_feeder(N: int, seed: int, delta_frac: float = 0.0, mult_hi: float = 1.2,
                kappa: float | None = None) -> Feeder:
    """Random radial three-phase feeder with N buses (bus 0 = slack).

    Draw order from numpy.random.default_rng(seed): parents (random recursive
    tree, parent[k] ~ U{0..k-1}), line lengths U(0.1, 0.5) km, delta flags
    (probability delta_frac per load bus), base real power U(10, 100) kW per
    phase, power factor U(0.90, 0.98) lagging per phase.  The loads are then
    scaled by kappa (computed by the linear drop rule unless given).
    """
    if N < 2:
        raise ValueError("a feeder needs the slack and at least one load bus")
    rng = np.random.default_rng(seed)
    parent = np.empty(N, dtype=np.int64)
    parent[0] = -1
    parent[1:] = rng.integers(0, np.arange(1, N))
    length = np.zeros(N)
    length[1:] = rng.uniform(0.1, 0.5, size=N - 1)
    is_delta = rng.random(N - 1) < delta_frac
    p_kw = rng.uniform(10.0, 100.0, size=(N - 1, 3))
    pf = rng.uniform(0.90, 0.98, size=(N - 1, 3))
    p_pu = p_kw / P_PHASE_BASE_KW
    q_pu = p_pu * np.tan(np.arccos(pf))
    base_raw = p_pu + 1j * q_pu
    z_km = _line_impedance_per_km_pu()
    z_line = np.zeros((N, 3, 3), dtype=np.complex128)
    z_line[1:] = length[1:, None, None] * z_km[None]
    if kappa is None:
        kappa = _load_scale(N, parent, length, base_raw, mult_hi)
    rows, cols, vals = _assemble_Y(N, parent, z_line)
    return Feeder(N=N, parent=parent, length_km=length, z_line=z_line,
                  Y_row=rows, Y_col=cols, Y_val=vals,
                  slack_idx=np.array([0, 1, 2], dtype=np.int32),
                  v_slack=V_SLACK.copy(), base_S=base_raw * kappa,
                  is_delta=is_delta, kappa=float(kappa), seed=seed)


def make_scenarios(feeder: Feeder, B: int, mult_lo: float, mult_hi: float,
                   seed: int | None = None):
    """Per-scenario constant-power loads, consumption convention (pu).

    One multiplier per (scenario, load bus) from default_rng(seed) (default
    feeder.seed + 1), U(mult_lo, mult_hi), applied to every phase or branch of
    that bus.  Returns (S_wye, S_delta), complex128[B, n], scenario-major.
    """
    if seed is None:
        seed = feeder.seed + 1
    rng = np.random.default_rng(seed)
    mult = rng.uniform(mult_lo, mult_hi, size=(B, feeder.N - 1))
    S = mult[:, :, None] * feeder.base_S[None, :, :]          # [B, N-1, 3]
    dmask = feeder.is_delta[None, :, None]
    S_wye = np.where(dmask, 0.0, S).reshape(B, feeder.n)
    S_delta = np.where(dmask, S, 0.0).reshape(B, feeder.n)
    return np.ascontiguousarray(S_wye), np.ascontiguousarray(S_delta)


# ---------------------------------------------------------------------------
# Partial-phase feeders: single- and two-phase laterals.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class PhasedFeeder:
    """A radial feeder whose buses carry 1, 2 or 3 of the phases a, b, c.

    Unknowns are numbered compactly: bus-major, present phases in ascending
    order, the slack's three phases first (global indices 0, 1, 2).
    bus_phase[g] = 3 k + p for global index g at bus k, phase p.  Loads are
    given per present phase ([B, n] arrays, compact order); delta loads sit on
    three-phase buses only, at the slot of the branch's first phase
    (ab, bc, ca).
    """
    N: int
    parent: np.ndarray        # int64[N]
    phases: np.ndarray        # bool[N, 3]
    z_line: np.ndarray        # complex128[N, 3, 3]; the present-phase sub-block is used
    Y_row: np.ndarray         # int32[nnz], compact global indices
    Y_col: np.ndarray
    Y_val: np.ndarray
    slack_idx: np.ndarray     # int32[3] = [0, 1, 2]
    v_slack: np.ndarray       # complex128[3]
    bus_phase: np.ndarray     # int32[n_total]
    base_S: np.ndarray        # complex128[N-1, 3], zero on absent phases
    is_delta: np.ndarray      # bool[N-1], three-phase buses only
    kappa: float
    seed: int

    @property
    def n_total(self) -> int:
        return int(self.bus_phase.size)

    @property
    def n(self) -> int:
        return self.n_total - 3


def make_partial_feeder(N: int, seed: int, lateral_frac: float = 0.3,
                        delta_frac: float = 0.0, mult_hi: float = 1.2) -> PhasedFeeder:
    """The feeder of make_feeder(N, seed) with laterals of fewer phases.

    Tree, lengths, loads and the three-phase line impedances are those of
    make_feeder.  Then, from default_rng(seed + 7), each bus in index order
    (parents first) keeps its parent's phases, except that with probability
    lateral_frac a bus whose parent has two or three phases and whose subtree
    is small (at most max(2, N / 16) buses: laterals sit at the periphery)
    starts a lateral: a random proper subset (one or two) of the parent's
    phases.  A line carries its downstream bus's phases with the matching
    sub-block of the 3x3 impedance; loads sit on present phases; delta loads
    stay on three-phase buses.
    """
    base = make_feeder(N, seed, delta_frac=delta_frac, mult_hi=mult_hi)
    rng = np.random.default_rng(seed + 7)
    size = np.ones(N, dtype=np.int64)
    for k in range(N - 1, 0, -1):
        size[base.parent[k]] += size[k]
    small = max(2, N // 16)
    phases = np.zeros((N, 3), dtype=bool)
    phases[0] = True
    for k in range(1, N):
        pp = np.nonzero(phases[base.parent[k]])[0]
        u = rng.random()
        if pp.size >= 2 and size[k] <= small and u < lateral_frac:
            m = int(rng.integers(1, pp.size))            # 1 .. |pp| - 1 phases
            keep = np.sort(rng.choice(pp, size=m, replace=False))
            phases[k, keep] = True
        else:
            phases[k, pp] = True
    gidx = -np.ones((N, 3), dtype=np.int64)
    bus_phase = []
    for k in range(N):
        for p in range(3):
            if phases[k, p]:
                gidx[k, p] = len(bus_phase)
                bus_phase.append(3 * k + p)
    rows, cols, vals = [], [], []
    for k in range(1, N):
        a = int(base.parent[k])
        ph = np.nonzero(phases[k])[0]
        y = np.linalg.inv(base.z_line[k][np.ix_(ph, ph)])
        for (u, v, sgn) in ((a, a, 1.0), (k, k, 1.0), (a, k, -1.0), (k, a, -1.0)):
            for i, p in enumerate(ph):
                for j, q in enumerate(ph):
                    rows.append(gidx[u, p])
                    cols.append(gidx[v, q])
                    vals.append(sgn * y[i, j])
    three = phases[1:].all(axis=1)
    return PhasedFeeder(N=N, parent=base.parent, phases=phases, z_line=base.z_line,
                        Y_row=np.asarray(rows, dtype=np.int32),
                        Y_col=np.asarray(cols, dtype=np.int32),
                        Y_val=np.asarray(vals, dtype=np.complex128),
                        slack_idx=np.array([0, 1, 2], dtype=np.int32),
                        v_slack=V_SLACK.copy(), bus_phase=np.asarray(bus_phase, dtype=np.int32),
                        base_S=np.where(phases[1:], base.base_S, 0.0),
                        is_delta=base.is_delta & three, kappa=base.kappa, seed=seed)


def make_partial_scenarios(feeder: PhasedFeeder, B: int, mult_lo: float, mult_hi: float,
                           seed: int | None = None):
    """(S_wye, S_delta), complex128[B, n] in the feeder's compact order.

    One multiplier per (scenario, load bus) from default_rng(seed) (default
    feeder.seed + 1), as in make_scenarios.
    """
    if seed is None:
        seed = feeder.seed + 1
    rng = np.random.default_rng(seed)
    mult = rng.uniform(mult_lo, mult_hi, size=(B, feeder.N - 1))
    S = mult[:, :, None] * feeder.base_S[None, :, :]          # [B, N-1, 3]
    dmask = feeder.is_delta[None, :, None]
    Sw = np.where(dmask, 0.0, S)
    Sd = np.where(dmask, S, 0.0)
    sel = feeder.phases[1:]                                    # [N-1, 3]
    return (np.ascontiguousarray(Sw[:, sel]), np.ascontiguousarray(Sd[:, sel]))


# ---------------------------------------------------------------------------
# Named workloads.  Each is one feeder (or a set of feeders) plus its scenario
# batch and solver settings.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    N: int
    B: int
    delta_frac: float
    mult: tuple
    seed: int
    tol: float = 1e-8
    max_iter: int = 50
    lateral_frac: float = 0.0   # > 0: partial-phase laterals (make_partial_feeder)


WORKLOADS = {
    # 13 buses (36 unknowns), 8 scenarios, wye loads only.
    "feeder13_b8": Workload("feeder13_b8", 13, 8, 0.0, (0.8, 1.2), 101),
    # 128 buses (381 unknowns), 4096 scenarios, 70 % wye / 30 % delta, U(0.5, 1.5).
    "feeder128_b4096": Workload("feeder128_b4096", 128, 4096, 0.3, (0.5, 1.5), 202),
    # 1024 buses (3069 unknowns), 16384 scenarios, 70 / 30, U(0.8, 1.2).
    "feeder1024_b16384": Workload("feeder1024_b16384", 1024, 16384, 0.3, (0.8, 1.2), 303),
    # the same feeder with single- and two-phase laterals (30 % of the small
    # subtrees start one), 16384 scenarios: a stand-in for the paper's feeder
    # counted in phase connections (Sec. III)
    "partial1024_b16384": Workload("partial1024_b16384", 1024, 16384, 0.3, (0.8, 1.2), 303,
                                   lateral_frac=0.3),
}


def make_workload(name: str, B: int | None = None):
    """(feeder, S_wye, S_delta, workload) for a named workload; B overrides the batch."""
    w = WORKLOADS[name]
    if w.lateral_frac > 0:
        f = make_partial_feeder(w.N, w.seed, lateral_frac=w.lateral_frac,
                                delta_frac=w.delta_frac, mult_hi=w.mult[1])
    else:
        f = make_feeder(w.N, w.seed, delta_frac=w.delta_frac, mult_hi=w.mult[1])
    S_wye, S_delta = workload_scenarios(f, w.B if B is None else B, w.mult[0], w.mult[1])
    return f, S_wye, S_delta, w


def workload_scenarios(f, B: int, mult_lo: float, mult_hi: float, seed: int | None = None):
    """Scenarios of a three-phase (make_scenarios) or partial-phase feeder."""
    if isinstance(f, PhasedFeeder):
        return make_partial_scenarios(f, B, mult_lo, mult_hi, seed=seed)
    return make_scenarios(f, B, mult_lo, mult_hi, seed=seed)


def heterogeneous_set(n_feeders: int = 64, seed: int = 404, n_lo: int = 50,
                      n_hi: int = 800, b_lo: int = 32, b_hi: int = 2048,
                      delta_frac: float = 0.4, mult=(0.8, 1.2)):
    """Feeder sizes N ~ U{n_lo..n_hi} and scenario counts B ~ round(logU(b_lo, b_hi)).

    Sizes come from default_rng(seed); feeder f is then drawn with seed
    1000*seed + 2f (its scenarios with that seed + 1).
    """
    rng = np.random.default_rng(seed)
    Ns = rng.integers(n_lo, n_hi + 1, size=n_feeders)
    Bs = np.rint(np.exp(rng.uniform(math.log(b_lo), math.log(b_hi), size=n_feeders))).astype(int)
    out = []
    for f in range(n_feeders):
        fs = 1000 * seed + 2 * f
        fd = make_feeder(int(Ns[f]), fs, delta_frac=delta_frac, mult_hi=mult[1])
        out.append((fd, int(Bs[f])))
    return out
