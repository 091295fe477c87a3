"""Virtual-Z compensation of the gate fidelity (oracle; test infrastructure).

The paper's gate metric assumes errorless single-qubit gates before and after the
simulated pulses (the compensation options of its Evolve listing, App. C step 6).
The kind computed here is the virtual Z gate, a phase diag(1, e^{i phi}) on each
qubit before and after the pulses: the fidelity of the computational block U
(D_c x D_c) against the target T is taken for

    M = T^dag (Z(a_1) (x) ... (x) Z(a_n)) U (Z(b_1) (x) ... (x) Z(b_n)),

with the phases chosen to bring U as close as possible to T.  Both fidelities
(F_state = |tr M / D_c|^2, F_avg = (tr M M^dag + |tr M|^2) / (D_c (D_c + 1)))
depend on the phases only through |tr M| (tr M M^dag = ||U||_F^2 for diagonal
unitaries), so the phases maximise |tr M|.

Readings taken here (the paper does not state the optimiser): coordinate ascent
from zero phases, sweeping a_1..a_n, then b_1..b_n; with the other phases fixed
tr M = X_0 + e^{i phi} X_1 (X_1 the terms in which the qubit is in |1>), whose
modulus is largest at phi = arg X_0 - arg X_1.  The sweeps stop at the first one
that does not raise |tr M| (the ascent is monotone, so this is convergence to
rounding), at most 2000.  The result is the local maximum that the ascent reaches
from zero phases.  The label j of a computational state counts the qubits with
the first qubit most significant: a_q acts on bit n - 1 - q of the row label,
b_q on that of the column label.

At the maximiser F is stationary in the phases, so dF/dtheta is the derivative
with the phases held fixed: the co-state is that of the uncompensated fidelity
against the effective target T_eff = Z(a)^dag T Z(b)^dag (tr(T_eff^dag U) = tr M).
"""
import numpy as np


def _bits(Dc, n):
    """bits[j, q] = bit n - 1 - q of label j (qubit q, first qubit most significant)."""
    j = np.arange(Dc)
    return np.array([[(jj >> (n - 1 - q)) & 1 for q in range(n)] for jj in j])


def trace_m(T, U, a, b):
    """tr(T^dag Z(a) U Z(b)) written out over the labels."""
    n = len(a)
    bits = _bits(U.shape[0], n)
    za = np.exp(1j * (bits @ np.asarray(a)))
    zb = np.exp(1j * (bits @ np.asarray(b)))
    return np.sum(np.conj(T) * (za[:, None] * U * zb[None, :]))


def compensate(T, U, nqb, max_sweeps=2000):
    """Phases (a, b), |tr M| and T_eff for target T and block U (D_c x D_c)."""
    T = np.asarray(T, dtype=np.complex128)
    U = np.asarray(U, dtype=np.complex128)
    n = nqb
    bits = _bits(U.shape[0], n)
    a = np.zeros(n)
    b = np.zeros(n)
    best = abs(trace_m(T, U, a, b))
    for _ in range(max_sweeps):
        for side in ("a", "b"):
            for q in range(n):
                ph = a if side == "a" else b
                ph[q] = 0.0
                za = np.exp(1j * (bits @ a))
                zb = np.exp(1j * (bits @ b))
                terms = np.conj(T) * (za[:, None] * U * zb[None, :])
                sel = bits[:, q] == 1
                if side == "a":
                    x1 = np.sum(terms[sel, :])
                    x0 = np.sum(terms[~sel, :])
                else:
                    x1 = np.sum(terms[:, sel])
                    x0 = np.sum(terms[:, ~sel])
                ph[q] = np.angle(x0) - np.angle(x1) if abs(x1) > 0 else 0.0
        now = abs(trace_m(T, U, a, b))
        if not now > best:
            break
        best = now
    za = np.exp(1j * (bits @ a))
    zb = np.exp(1j * (bits @ b))
    T_eff = np.conj(za)[:, None] * T * np.conj(zb)[None, :]
    return a, b, abs(trace_m(T, U, a, b)), T_eff


def comp_block(sys, psi_lab):
    """The computational block U[:, j] = <c_.|psi_s> of the evolved columns (every
    computational state evolved exactly once)."""
    from .evolve import comp_map
    comp, cols = comp_map(sys)
    Dc = len(comp)
    U = np.zeros((Dc, Dc), dtype=np.complex128)
    seen = sorted(j for j in cols if j >= 0)
    if seen != list(range(Dc)):
        raise ValueError("compensation needs every computational state evolved exactly once")
    for s, j in enumerate(cols):
        if j >= 0:
            U[:, j] = psi_lab[comp, s]
    return U


def compensated_fidelities(sys, psi_lab):
    """(F_avg, F_state, T_eff) of the lab-frame columns with virtual-Z compensation."""
    T = np.asarray(sys.wl["target"], dtype=np.complex128)
    U = comp_block(sys, psi_lab)
    nqb = int(round(np.log2(U.shape[0])))
    _, _, best, T_eff = compensate(T, U, nqb)
    Dc = U.shape[0]
    F_avg = (np.linalg.norm(U) ** 2 + best ** 2) / (Dc * (Dc + 1))
    F_state = (best / Dc) ** 2
    return F_avg, F_state, T_eff
