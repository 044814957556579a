"""Brute-force Newton-Raphson power flow for tiny feeders (independent checker).

Solves the nodal current balance Y_LL v + Y_Ls v_s = -(current drawn by the
loads) for v in rectangular coordinates with a central-difference Jacobian.
It uses no reduced impedance and no fixed point, and writes its own load
model through a branch-to-phase incidence matrix, so it shares neither code
nor algorithm with the oracle.
"""
import numpy as np

# columns: branches ab, bc, ca; rows: phases a, b, c.  +1 where the branch
# current leaves the phase, -1 where it returns.
INCIDENCE = np.array([[1.0, 0.0, -1.0],
                      [-1.0, 1.0, 0.0],
                      [0.0, -1.0, 1.0]])
BRANCH_FROM = np.array([0, 1, 2])
BRANCH_TO = np.array([1, 2, 0])


def drawn_current(v, s_wye, s_del):
    """Current drawn from each phase node by wye and delta constant-power loads."""
    nb = v.size // 3
    d = np.zeros(v.size, dtype=np.complex128)
    for k in range(nb):
        vk = v[3 * k:3 * k + 3]
        for p in range(3):
            s = s_wye[3 * k + p]
            if s != 0:
                d[3 * k + p] += np.conj(s) / np.conj(vk[p])
        ibr = np.zeros(3, dtype=np.complex128)
        for br in range(3):
            s = s_del[3 * k + br]
            if s != 0:
                ibr[br] = np.conj(s) / np.conj(vk[BRANCH_FROM[br]] - vk[BRANCH_TO[br]])
        d[3 * k:3 * k + 3] += INCIDENCE @ ibr
    return d


def drawn_current_phased(v, s_wye, s_del, bus_phase):
    """The same load model on a feeder whose buses carry any subset of phases.

    bus_phase[j] = 3 * bus + phase of unknown j.  Each bus gathers its present
    phases into a 3-slot vector (absent slots zero) and applies the branch
    incidence to the branches whose two phases are present.
    """
    d = np.zeros(v.size, dtype=np.complex128)
    buses = {}
    for j, g in enumerate(bus_phase):
        buses.setdefault(int(g) // 3, {})[int(g) % 3] = j
    for k, slots in buses.items():
        for p, j in slots.items():
            if s_wye[j] != 0:
                d[j] += np.conj(s_wye[j]) / np.conj(v[j])
        for br in range(3):
            x, y = BRANCH_FROM[br], BRANCH_TO[br]
            if x not in slots or s_del[slots[x]] == 0:
                continue
            assert y in slots, "delta branch without its second phase"
            ib = np.conj(s_del[slots[x]]) / np.conj(v[slots[x]] - v[slots[y]])
            for p in (x, y):
                d[slots[p]] += INCIDENCE[p, br] * ib
    return d


def newton_solve(Y_LL, Y_Ls, v_s, s_wye, s_del, v_start, tol=1e-13, max_iter=50,
                 bus_phase=None):
    n = Y_LL.shape[0]

    def drawn(v):
        if bus_phase is None:
            return drawn_current(v, s_wye, s_del)
        return drawn_current_phased(v, s_wye, s_del, bus_phase)

    def F(x):
        v = x[:n] + 1j * x[n:]
        g = Y_LL @ v + Y_Ls @ v_s + drawn(v)
        return np.concatenate([g.real, g.imag])

    x = np.concatenate([v_start.real, v_start.imag]).astype(float)
    h = 1e-7
    for _ in range(max_iter):
        f = F(x)
        if np.abs(f).max() < tol:
            break
        J = np.empty((2 * n, 2 * n))
        for c in range(2 * n):
            e = np.zeros(2 * n)
            e[c] = h
            J[:, c] = (F(x + e) - F(x - e)) / (2 * h)
        x = x - np.linalg.solve(J, f)
    f = F(x)
    return x[:n] + 1j * x[n:], float(np.abs(f).max())
