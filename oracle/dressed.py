"""Dressed (multi-qubit eigen-) basis of the gate metric (oracle; test infrastructure).

App. C: the gate is represented in the eigenbasis of the idle Hamiltonian while the
evolution runs in the product basis, U -> V^dag U V (its Eq. for the basis
transform), absorbed into the states: the initial states are V|comp>, the final
states are projected with V^dag.  Only the computational block is needed, so V is
kept as the D x D_c matrix V_c of the dressed computational states.

Readings taken here (the paper fixes the idea, not these details):

* the idle Hamiltonian is the lab-frame Hamiltonian without drives: every mode's
  level energies E_k - E_0 and the couplings J A (x) B;
* the dressed state of computational label j is the eigenvector with the largest
  overlap |<bare_j|v>| on the bare computational state (a distinct eigenvector for
  every label, else the basis is refused), its phase fixed so that <bare_j|v> is
  real and positive (the paper's "adjusting the phases of its eigenstates");
* the evolved columns are exactly the dressed computational states, each once.

The pulse gradient needs no derivative of V (V does not depend on the pulses): the
co-state of the final states is V_c times the co-state of the projected block.  The
Hamiltonian-parameter gradient adds V's derivative: each dressed vector moves by the
first-order perturbation formula dv_k = sum_{m != k} v_m <v_m|dH0|v_k> / (lam_k - lam_m)
of the idle Hamiltonian H0 (real symmetric, non-degenerate levels), contracted with the
co-vector of V_c from the initial columns (the co-state pulled back to t = 0) and from
the projection (psi(T) times the block's co-state).
"""
import numpy as np

from .evolve import (comp_map, rk4_evolve, frame_epilogue, block_fidelity_and_costate,
                     adjoint_from_costate)
from .system import OracleSystem, n_pulse_params


def idle_hamiltonian(sys):
    """Dense lab-frame idle Hamiltonian: level energies and couplings (Eq. 1, no drives)."""
    H = np.diag(sys.hd_diag()).astype(np.complex128)
    for c in sys.couplings:
        H += c["J"] * sys.embed({c["a"]: sys.op(c["a"], c["op_a"]), c["b"]: sys.op(c["b"], c["op_b"])})
    return H


def dressed_vectors(sys):
    """V_c (D x D_c): per computational label j the assigned eigenvector of the idle
    Hamiltonian, phase-fixed; and the assigned eigenvalues."""
    w, V = np.linalg.eigh(idle_hamiltonian(sys))
    comp, _ = comp_map(sys)
    Vc = np.zeros((sys.D, len(comp)), dtype=np.complex128)
    taken = set()
    lam = np.zeros(len(comp))
    for j, r in enumerate(comp):
        k = int(np.argmax(np.abs(V[r, :])))
        if k in taken:
            raise ValueError("two computational states share a dressed state")
        taken.add(k)
        v = V[:, k]
        Vc[:, j] = v * (np.conj(v[r]) / abs(v[r]))
        lam[j] = w[k]
    return Vc, lam


def dressed_evolve(wl):
    """Lab-frame final states of the dressed computational columns (RK4, the
    workload's frame) with their labels, and the stored history."""
    sys = OracleSystem(wl)
    comp, cols = comp_map(sys)
    if sorted(cols) != list(range(len(comp))):
        raise ValueError("the dressed basis evolves every computational state exactly once")
    Vc, _ = dressed_vectors(sys)
    psi0 = Vc[:, cols]
    psiT, hist = rk4_evolve(sys, psi0, store=True)
    return sys, Vc, cols, frame_epilogue(sys, psiT), hist


def dressed_fidelities(wl):
    """(F_avg, F_state, U_c) in the dressed basis, U_c[j', s] = <v_j'|psi_s>."""
    sys, Vc, cols, psi_lab, _ = dressed_evolve(wl)
    T = np.asarray(wl["target"], dtype=np.complex128)
    Uc = Vc.conj().T @ psi_lab
    Fa, _ = block_fidelity_and_costate(T, Uc, cols, "avg")
    Fs, _ = block_fidelity_and_costate(T, Uc, cols, "state")
    return Fa, Fs, Uc


def dressed_pulse_gradient(wl, kind=None):
    """F and dF/d(pulse parameters) in the dressed basis by the exact discrete RK4
    adjoint, the co-state of the final states being V_c times that of U_c."""
    kind = kind or wl["fid_kind"]
    sys, Vc, cols, psi_lab, hist = dressed_evolve(wl)
    T = np.asarray(wl["target"], dtype=np.complex128)
    F, barc = block_fidelity_and_costate(T, Vc.conj().T @ psi_lab, cols, kind)
    grad, _ = adjoint_from_costate(sys, hist, psi_lab, Vc @ barc, sys.N)
    npul = sum(n_pulse_params(dr) for dr in wl["drives"])
    return F, grad[:npul]


def idle_hamiltonian_derivative(sys, prm):
    """dH0/dtheta of the idle Hamiltonian for one parameter of sys.param_list(): zero for
    pulse parameters; A (x) B for a coupling's J; for a device parameter of mode i its
    energies' derivative on the diagonal and J times the derivative of its coupling
    operators (eigen-derivatives of the subsystem, as in the evolution's dH)."""
    kind, a, b = prm
    D = sys.D
    if kind == "pulse":
        return np.zeros((D, D), dtype=np.complex128)
    if kind == "J":
        c = sys.couplings[a]
        return sys.embed({c["a"]: sys.op(c["a"], c["op_a"]), c["b"]: sys.op(c["b"], c["op_b"])})
    i, p = a, b
    _, dops = sys.mode_derivs(i, p)
    out = np.diag(sys.dHd_diag(prm)).astype(np.complex128)
    for c in sys.couplings:
        if c["a"] == i:
            out += c["J"] * sys.embed({i: sys.dop(dops, i, c["op_a"]), c["b"]: sys.op(c["b"], c["op_b"])})
        elif c["b"] == i:
            out += c["J"] * sys.embed({c["a"]: sys.op(c["a"], c["op_a"]), i: sys.dop(dops, i, c["op_b"])})
    return out


def dressed_full_gradient(wl, kind=None):
    """F and dF/dtheta for every parameter (pulse, then E_J, E_C, E_L per mode, then J
    per coupling) in the dressed basis: the evolution's discrete RK4 adjoint with the
    co-state V_c barc, plus V_c's derivative contracted with
    W = psi(T) barc^dag (projection) + lambda(0) on the labels' columns (initial states)."""
    kind = kind or wl["fid_kind"]
    sys, Vc, cols, psi_lab, hist = dressed_evolve(wl)
    T = np.asarray(wl["target"], dtype=np.complex128)
    F, barc = block_fidelity_and_costate(T, Vc.conj().T @ psi_lab, cols, kind)
    grad, prms, bar0 = adjoint_from_costate(sys, hist, psi_lab, Vc @ barc, sys.N, with_bar=True)
    H0 = idle_hamiltonian(sys)
    if np.max(np.abs(H0.imag)) > 1e-12 * max(1.0, np.max(np.abs(H0.real))):
        raise ValueError("the dressed gradient needs a real idle Hamiltonian")
    w, V = np.linalg.eigh(H0.real)
    comp, _ = comp_map(sys)
    Dc = len(comp)
    W = psi_lab @ barc.conj().T                     # D x Dc, from U_c = V_c^dag psi(T)
    for s_, j in enumerate(cols):
        W[:, j] += bar0[:, s_]                      # from the initial columns V_c[:, j]
    ks, sg = [], []
    for j, r in enumerate(comp):
        k = int(np.argmax(np.abs(V[r, :])))
        ks.append(k)
        sg.append(1.0 if V[r, k] > 0 else -1.0)
    for p_, prm in enumerate(prms):
        if prm[0] == "pulse":
            continue
        dH = idle_hamiltonian_derivative(sys, prm)
        M = V.T @ dH @ V                            # <v_m|dH0|v_k>
        for j in range(Dc):
            k = ks[j]
            den = w[k] - w
            den[k] = np.inf
            dv = V @ (M[:, k] / den)
            grad[p_] += np.real(np.vdot(W[:, j], sg[j] * dv))
    return F, grad
