"""Plain FP64 CPU oracle of the batched Newton-Raphson power flow (paper Sec. II-A).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this module.  It shares no code with
the CUDA library and never imports it.

What it computes, in the paper's notation (Sec. II-A, eqs. 1-3): the state
x_b = [theta_Theta; V_Q] (angles of the PV and PQ buses, magnitudes of the PQ
buses), the mismatch map

    F_b(x_b) = [P_calc,Theta(x_b) - P_b,Theta ;  Q_calc,Q(x_b) - Q_b,Q]

with S_calc = V o conj(Y_bus V), and the Newton update J_b dx = -F_b(x_b).
The method solves the Newton system with preconditioned GMRES; the solution
it converges to is the root of F_b, so the oracle takes the plain Newton
iteration with the exact polar Jacobian (H, N, M, L partition, eq. 4) and a
dense direct solve.

Readings where the paper is silent:
  * Flat start: theta = 0, |V| = 1 at PQ buses and the set-point at PV buses
    and the slack (angle 0).
  * Stop: converged when max |F_b(x_k)| <= tol; iters = Newton updates taken
    before that check passed.  Not converged after max_iter updates, or when
    F becomes non-finite (diverged).
  * The returned voltage is the last iterate.

Parity status: pinned by the two-bus closed forms (PQ and lossless PV),
finite differences of the mismatch (Jacobian), quadratic convergence, an
independent root finder on the rectangular formulation, the Z-bus oracle on
a balanced feeder's positive-sequence network, and power-balance invariants.
"""
from __future__ import annotations

import numpy as np

PQ, PV, SLACK = 0, 1, 2


def dense_Y(N: int, row, col, val) -> np.ndarray:
    Y = np.zeros((N, N), dtype=np.complex128)
    np.add.at(Y, (np.asarray(row), np.asarray(col)), np.asarray(val))
    return Y


def index_sets(bus_type):
    """(Theta, Q): the PV + PQ buses (angle block) and the PQ buses (magnitude
    block), ascending."""
    bt = np.asarray(bus_type)
    theta = np.nonzero(bt != SLACK)[0]
    q = np.nonzero(bt == PQ)[0]
    return theta, q


def power_injection(Y: np.ndarray, V: np.ndarray) -> np.ndarray:
    """S_calc = V o conj(Y V)."""
    return V * np.conj(Y @ V)


def mismatch(Y, V, P, Q, theta, q) -> np.ndarray:
    """F = [P_calc - P on Theta; Q_calc - Q on Q] (eq. 2)."""
    S = power_injection(Y, V)
    return np.concatenate([S.real[theta] - P[theta], S.imag[q] - Q[q]])


def jacobian(Y, V, theta, q) -> np.ndarray:
    """Polar Jacobian [[H, N], [M, L]] of F with respect to [theta_Theta; |V|_Q] (eq. 4).

    With I = Y V and e = V / |V|:
      dS/dtheta = j diag(V) conj(diag(I) - Y diag(V))
      dS/d|V|   = diag(V) conj(Y diag(e)) + conj(diag(I)) diag(e)
    """
    I = Y @ V
    e = V / np.abs(V)
    dS_dth = 1j * (V[:, None] * np.conj(np.diag(I) - Y * V[None, :]))
    dS_dvm = V[:, None] * np.conj(Y * e[None, :]) + np.diag(np.conj(I) * e)
    H = dS_dth.real[np.ix_(theta, theta)]
    Nn = dS_dvm.real[np.ix_(theta, q)]
    M = dS_dth.imag[np.ix_(q, theta)]
    L = dS_dvm.imag[np.ix_(q, q)]
    return np.block([[H, Nn], [M, L]])


def flat_start(bus_type, v_set) -> np.ndarray:
    bt = np.asarray(bus_type)
    vm = np.where(bt == PQ, 1.0, np.asarray(v_set, dtype=np.float64))
    return vm.astype(np.complex128)


def newton(Y, bus_type, v_set, P, Q, tol=1e-10, max_iter=20, history=None):
    """Newton-Raphson for one scenario.  Returns (V complex[N], iters, converged).

    history: optional list receiving max |F| of every iterate."""
    theta, q = index_sets(bus_type)
    V = flat_start(bus_type, v_set)
    va = np.angle(V)
    vm = np.abs(V)
    nt = theta.size
    for k in range(max_iter + 1):
        F = mismatch(Y, V, P, Q, theta, q)
        fmax = np.abs(F).max() if F.size else 0.0
        if history is not None:
            history.append(fmax)
        if not np.isfinite(fmax):
            return V, k, 0
        if fmax <= tol:
            return V, k, 1
        if k == max_iter:
            return V, k, 0
        try:
            dx = np.linalg.solve(jacobian(Y, V, theta, q), -F)
        except np.linalg.LinAlgError:
            return V, k, 0
        va[theta] += dx[:nt]
        vm[q] += dx[nt:]
        V = vm * np.exp(1j * va)
    return V, max_iter, 0


def solve_batch(N, row, col, val, bus_type, v_set, P, Q, tol=1e-10, max_iter=20):
    """Newton-Raphson over every scenario of P, Q [B, N].  Returns a dict with
    V [B, N] complex, iters int32[B], converged uint8[B] and Y."""
    Y = dense_Y(N, row, col, val)
    B = P.shape[0]
    V = np.zeros((B, N), dtype=np.complex128)
    it = np.zeros(B, dtype=np.int32)
    cv = np.zeros(B, dtype=np.uint8)
    for b in range(B):
        V[b], it[b], cv[b] = newton(Y, bus_type, v_set, P[b], Q[b], tol, max_iter)
    return dict(V=V, iters=it, converged=cv, Y=Y)
