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
mismatch invariant).  The load-gradient adjoint (solve_adjoint) is pinned by
central finite differences of the forward solve (directional and entry by
entry), by the derivative of the two-bus closed form, and on partial-phase
feeders.
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


# ---------------------------------------------------------------------------
# Gradient of the converged fixed point with respect to the loads.  The paper
# motivates the solver as a component of GPU learning pipelines (Sec. I and
# the conclusion); here the solution v*(S) of v = Z i(v, S) + w is
# differentiated through the fixed-point condition (implicit function
# theorem), not through the iterations.
#
# Convention (the one of complex autograd): for a real loss L of a complex
# array x, grad_x = dL/dRe(x) + j dL/dIm(x), so that dL = Re(sum conj(grad) dx).
# ---------------------------------------------------------------------------

def _unknown_map(n: int, bus_phase) -> tuple[np.ndarray, dict]:
    """(bus_phase of every unknown, {bus_phase value: unknown index})."""
    if bus_phase is None:
        if n % 3:
            raise ValueError("three-phase unknowns need n % 3 == 0 (give bus_phase otherwise)")
        bp = np.arange(n) + 3        # bus k >= 1, phase p -> 3 k + p
    else:
        bp = np.asarray(bus_phase)
    return bp, {int(g): j for j, g in enumerate(bp)}


def load_current_jacobians(v: np.ndarray, s_wye: np.ndarray, s_del: np.ndarray,
                           bus_phase=None):
    """Derivatives of the load currents of one scenario.

    The current i(v, S) of constant-power loads depends on conj(v) and conj(S)
    only, so its differential is di = A conj(dv) + Dw conj(dS_wye) +
    Dd conj(dS_del).  Returns the complex [n, n] matrices (A, Dw, Dd).

      wye slot j:      i_j = -conj(S_j) / conj(v_j)
                       A[j, j] = conj(S_j / v_j^2),  Dw[j, j] = -1 / conj(v_j)
      delta slot x     I = conj(S / u), u = v_x - v_y, drawn from x, returned
      (branch x -> y): into y (y the next phase of a, b, c on the same bus);
                       dI = -conj(S / u^2) conj(du) + conj(dS) / conj(u)
                       A gains c on (x, x), (y, y) and -c on (x, y), (y, x),
                       c = conj(S / u^2);  Dd[x, x] = -1 / conj(u),
                       Dd[y, x] = +1 / conj(u)
    A delta slot whose branch has no second phase is not a load (its column
    of Dd stays zero).
    """
    n = v.size
    bp, where = _unknown_map(n, bus_phase)
    A = np.zeros((n, n), dtype=np.complex128)
    Dw = np.zeros((n, n), dtype=np.complex128)
    Dd = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        Dw[j, j] = -1.0 / np.conj(v[j])
        if s_wye[j] != 0:
            A[j, j] += np.conj(s_wye[j] / v[j] ** 2)
        k, x = divmod(int(bp[j]), 3)
        m = where.get(3 * k + (x + 1) % 3)
        if m is None:
            continue
        u = v[j] - v[m]
        Dd[j, j] = -1.0 / np.conj(u)
        Dd[m, j] = 1.0 / np.conj(u)
        if s_del[j] != 0:
            c = np.conj(s_del[j] / u ** 2)
            A[j, j] += c
            A[m, m] += c
            A[j, m] -= c
            A[m, j] -= c
    return A, Dw, Dd


def _real_conj_map(M: np.ndarray) -> np.ndarray:
    """Real [2n, 2n] matrix of z -> M conj(z) acting on [Re z; Im z]."""
    return np.block([[M.real, M.imag], [M.imag, -M.real]])


def solve_adjoint(Z: np.ndarray, V: np.ndarray, S_wye: np.ndarray, S_del: np.ndarray,
                  G: np.ndarray, bus_phase=None):
    """Gradients (H_wye, H_del) of a real loss with respect to S_wye and S_del.

    V [B, n] is a fixed point v = Z i(v, S) + w of each scenario and G [B, n]
    the loss gradient with respect to V.  Differentiating the fixed-point
    condition gives dv = Z A conj(dv) + Z (Dw conj(dS_wye) + Dd conj(dS_del))
    (load_current_jacobians); written as a real map on [Re; Im],
    dx = J_v dx + J_w ds_wye + J_d ds_del, so dx/ds = (I - J_v)^{-1} J_s and
    grad_s = J_s^T (I - J_v)^{-T} g.  Dense real solve per scenario.
    """
    V = np.asarray(V, dtype=np.complex128)
    B, n = V.shape
    Hw = np.zeros((B, n), dtype=np.complex128)
    Hd = np.zeros((B, n), dtype=np.complex128)
    eye = np.eye(2 * n)
    for b in range(B):
        A, Dw, Dd = load_current_jacobians(V[b], S_wye[b], S_del[b], bus_phase)
        Jv = _real_conj_map(Z @ A)
        g = np.concatenate([G[b].real, G[b].imag])
        lam = np.linalg.solve((eye - Jv).T, g)
        hw = _real_conj_map(Z @ Dw).T @ lam
        hd = _real_conj_map(Z @ Dd).T @ lam
        Hw[b] = hw[:n] + 1j * hw[n:]
        Hd[b] = hd[:n] + 1j * hd[n:]
    return Hw, Hd
