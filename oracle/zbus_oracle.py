"""Plain FP64 CPU oracle of the batched three-phase Z-bus power flow (paper Sec. II-B).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this module.  It shares no code with
the CUDA library and never imports it.

What it computes, in the paper's notation (Sec. II-B, the fixed-point map):

    v_b^{k+1} = Z i(v_b^k, S_b^wye, S_b^del) + v_0

with Z the reduced bus impedance of the non-slack phases, v_0 the no-load
voltage (called w here, to keep v_0 free for the slack) and i(.) the current
injection of constant-power wye and delta loads.

Readings where the paper is silent (each is listed with its reason in the
design notes):
  * Z = inv(Y_LL) and w = -Z Y_Ls v_s, with Y_LL / Y_Ls the non-slack rows of
    the admittance matrix split by slack / non-slack columns.
  * Start: v^0 = w (the no-load voltage) unless a warm start is given.
  * Stop: default rule 'maxabs', delta_k = max_j |v_j^{k} - v_j^{k-1}|; the
    paper's rule 'summag', delta_k = | sum_j |v_j^{k}| - sum_j |v_j^{k-1}| |.
    Converged when delta_k <= tol.  A non-finite delta_k stops the scenario as
    diverged.  Otherwise the scenario stops unconverged after max_iter maps.
  * iters counts the Z products performed, including the one that met tol.
  * The returned voltage is the last iterate v^k.
  * A load slot with S = 0 draws no current (its division is not taken).
  * Delta branches are ordered (ab, bc, ca); branch xy draws
    I_xy = conj(S_xy / (v_x - v_y)) out of phase x and returns it into phase y.

Parity status: every function below is pinned by tests that do not retype it
(closed-form two-bus solution, balanced delta equal to balanced wye, per-branch
delta power balance, lowest-common-ancestor form of Z on radial feeders,
no-load voltage, brute-force Newton-Raphson on tiny feeders, and the power
mismatch invariant).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# Setup: reduced impedance and no-load voltage (Sec. II-B, "after separating
# slack and non-slack phases" and "precomputed reduced bus-impedance matrix").
# ---------------------------------------------------------------------------

def partition(Y: np.ndarray, slack_idx) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Split the full admittance matrix into Y_LL (non-slack x non-slack) and Y_Ls.

    Returns (Y_LL, Y_Ls, load_idx) where load_idx lists the non-slack global
    indices in ascending order (the unknown ordering j).
    """
    slack_idx = np.asarray(slack_idx)
    mask = np.ones(Y.shape[0], dtype=bool)
    mask[slack_idx] = False
    load_idx = np.nonzero(mask)[0]
    Y_LL = Y[np.ix_(load_idx, load_idx)]
    Y_Ls = Y[np.ix_(load_idx, slack_idx)]
    return Y_LL, Y_Ls, load_idx


def reduced_impedance(Y_LL: np.ndarray, Y_Ls: np.ndarray, v_slack: np.ndarray):
    """Z = Y_LL^{-1}, w = -Z Y_Ls v_s (the no-load voltage of the non-slack phases)."""
    Z = np.linalg.inv(Y_LL)
    w = -Z @ (Y_Ls @ v_slack)
    return Z, w


def dense_from_coo(n_total: int, row, col, val) -> np.ndarray:
    Y = np.zeros((n_total, n_total), dtype=np.complex128)
    np.add.at(Y, (np.asarray(row), np.asarray(col)), np.asarray(val))
    return Y


# ---------------------------------------------------------------------------
# Load currents (Sec. II-B: wye currents -(S/v)^*, delta currents from
# line-to-line voltages mapped back to phase currents).
# ---------------------------------------------------------------------------

def _safe_conj_div(S: np.ndarray, V: np.ndarray) -> np.ndarray:
    """conj(S / V), zero where S == 0 (an absent load draws no current)."""
    out = np.zeros(np.broadcast_shapes(S.shape, V.shape), dtype=np.complex128)
    m = S != 0
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.conj(S / V)
    out[m] = q[m]
    return out


def load_currents(V: np.ndarray, S_wye: np.ndarray, S_del: np.ndarray,
                  bus_phase: np.ndarray | None = None) -> np.ndarray:
    """Current injection i(V) of constant-power loads, [B, n] complex.

    V, S_wye, S_del: [B, n]; consumption convention.  Without bus_phase the
    unknowns come in three-phase triples (n = 3 * load buses).  With it,
    bus_phase[j] = 3 * bus + phase names each unknown (partial-phase feeders),
    and see load_currents_phased.
    """
    if bus_phase is not None:
        return load_currents_phased(V, S_wye, S_del, bus_phase)
    B, n = V.shape
    Vb = V.reshape(B, n // 3, 3)
    i_wye = -_safe_conj_div(S_wye.reshape(B, n // 3, 3), Vb)
    # line-to-line voltages in branch order (ab, bc, ca)
    Vll = np.stack([Vb[..., 0] - Vb[..., 1],
                    Vb[..., 1] - Vb[..., 2],
                    Vb[..., 2] - Vb[..., 0]], axis=-1)
    I_br = _safe_conj_div(S_del.reshape(B, n // 3, 3), Vll)   # drawn by each branch
    I_ab, I_bc, I_ca = I_br[..., 0], I_br[..., 1], I_br[..., 2]
    drawn = np.stack([I_ab - I_ca, I_bc - I_ab, I_ca - I_bc], axis=-1)
    return (i_wye - drawn).reshape(B, n)


def load_currents_phased(V: np.ndarray, S_wye: np.ndarray, S_del: np.ndarray,
                         bus_phase: np.ndarray) -> np.ndarray:
    """i(V) on a feeder whose buses carry any subset of the phases.

    The same definitions per existing phase and branch: a wye load draws
    conj(S_j / v_j) out of its phase; the delta entry at phase x of a bus is
    the branch x -> y (y the next phase of a, b, c) and draws
    I = conj(S / (v_x - v_y)) out of phase x and returns it into phase y.  A
    delta entry whose branch lacks phase y is not a load (it must be zero).
    """
    bus_phase = np.asarray(bus_phase)
    B, n = V.shape
    where = {int(g): j for j, g in enumerate(bus_phase)}
    drawn = _safe_conj_div(S_wye, V)
    for j in range(n):
        if not np.any(S_del[:, j] != 0):
            continue
        k, x = divmod(int(bus_phase[j]), 3)
        m = where.get(3 * k + (x + 1) % 3)
        if m is None:
            raise ValueError(f"delta load at unknown {j}: branch has no second phase")
        I = _safe_conj_div(S_del[:, j], V[:, j] - V[:, m])
        drawn[:, j] += I
        drawn[:, m] -= I
    return -drawn


# ---------------------------------------------------------------------------
# The fixed point (Sec. II-B, eq. of the Z-bus map; stop rule and iteration cap).
# ---------------------------------------------------------------------------

def fixed_point(Z: np.ndarray, w: np.ndarray, S_wye: np.ndarray, S_del: np.ndarray,
                tol: float, max_iter: int, rule: str = "maxabs", V0: np.ndarray | None = None,
                bus_phase: np.ndarray | None = None):
    """Batched Z-bus fixed point.  Returns (V [B,n], iters int32[B], converged uint8[B]).

    Every scenario iterates independently; a scenario that has stopped is left
    untouched while the others continue.  bus_phase: see load_currents.
    """
    S_wye = np.asarray(S_wye, dtype=np.complex128)
    S_del = np.asarray(S_del, dtype=np.complex128)
    B, n = S_wye.shape
    if V0 is None:
        V = np.broadcast_to(w, (B, n)).copy()
    else:
        V = np.array(V0, dtype=np.complex128, copy=True)
    iters = np.zeros(B, dtype=np.int32)
    conv = np.zeros(B, dtype=np.uint8)
    active = np.arange(B)
    for k in range(1, max_iter + 1):
        if active.size == 0:
            break
        Va = V[active]
        I = load_currents(Va, S_wye[active], S_del[active], bus_phase)
        Vn = I @ Z.T + w                      # v^{k} = Z i(v^{k-1}) + w
        if rule == "maxabs":
            delta = np.abs(Vn - Va).max(axis=1)
        elif rule == "summag":
            delta = np.abs(np.abs(Vn).sum(axis=1) - np.abs(Va).sum(axis=1))
        else:
            raise ValueError(rule)
        V[active] = Vn
        iters[active] = k
        finite = np.isfinite(delta)
        done = (~finite) | (delta <= tol)
        conv[active[finite & (delta <= tol)]] = 1
        active = active[~done]
    return V, iters, conv


def power_mismatch(Y_LL: np.ndarray, Y_Ls: np.ndarray, v_slack: np.ndarray,
                   V: np.ndarray, S_wye: np.ndarray, S_del: np.ndarray,
                   bus_phase: np.ndarray | None = None) -> np.ndarray:
    """Per-scenario max_j |v_j conj((Y_LL v + Y_Ls v_s)_j - i_j(v))|, with Y, never Z."""
    net = V @ Y_LL.T + (Y_Ls @ v_slack)[None, :]
    r = net - load_currents(V, S_wye, S_del, bus_phase)
    return np.abs(V * np.conj(r)).max(axis=1)


def solve_coo(n_total, row, col, val, slack_idx, v_slack, S_wye, S_del,
              tol=1e-8, max_iter=50, rule="maxabs", V0=None, bus_phase=None):
    """Convenience: network setup from COO, then the batched fixed point.

    bus_phase: None for three-phase triples, else [n_total] (3 * bus + phase
    of every global index, slack included) for partial-phase feeders.
    """
    Y = dense_from_coo(n_total, row, col, val)
    Y_LL, Y_Ls, load_idx = partition(Y, slack_idx)
    Z, w = reduced_impedance(Y_LL, Y_Ls, np.asarray(v_slack))
    bp = None if bus_phase is None else np.asarray(bus_phase)[load_idx]
    V, it, cv = fixed_point(Z, w, S_wye, S_del, tol, max_iter, rule=rule, V0=V0, bus_phase=bp)
    return dict(V=V, iters=it, converged=cv, Z=Z, w=w, Y_LL=Y_LL, Y_Ls=Y_Ls, bus_phase=bp)
