"""Open-system evolution by the vectorised Lindblad master equation (oracle; test
infrastructure).

The paper notes (App. C, last paragraph; Sec. 2) that the dynamics of a density
matrix is characterised by a superoperator obtained from the vectorised Lindblad
master equation, and that its solver and back-propagation carry over to it.  What is
computed here, in the frame of the workload (R1):

    d rho / dt = -i [H(t), rho] + sum_c gamma_c (L_c rho L_c^dag - {L_c^dag L_c, rho} / 2),

with row-major vectorisation vec(A rho B) = (A (x) B^T) vec(rho), so that

    Lv(t) = -i (H (x) I - I (x) H^T)
            + sum_c gamma_c (L (x) L^* - (L^dag L) (x) I / 2 - I (x) (L^dag L)^T / 2),

evolved by the same fixed-step RK4 as the state columns (stage times of R2).
Readings taken here (the paper gives no formulas for it):

* a collapse operator acts on one mode: workload key "collapse", a list of
  {"mode": i, "L": d x d matrix in the truncated eigenbasis, "rate": gamma (1/ns)};
* in the interaction frame the collapse operators rotate with the frame like every
  other operator, L_I(t) = exp(i H_d t) L exp(-i H_d t), and the lab-frame density
  matrix is exp(-i H_d T) rho_I exp(i H_d T);
* the state fidelity of rho against a pure target |t> is <t| rho |t>.
"""
import numpy as np

from .system import OracleSystem, stage_time


def liouvillian(sys, n, j):
    """Dense D^2 x D^2 generator at stage j of step n (frame of the system)."""
    D = sys.D
    H = sys.hamiltonian(n, j)
    I = np.eye(D, dtype=np.complex128)
    Lv = -1j * (np.kron(H, I) - np.kron(I, H.T))
    t = stage_time(n, j, sys.dt)
    for c in sys.wl.get("collapse", []):
        L = sys.embed({c["mode"]: sys.frame_op(np.asarray(c["L"], dtype=np.complex128), c["mode"], t)})
        LdL = L.conj().T @ L
        Lv += c["rate"] * (np.kron(L, L.conj()) - 0.5 * np.kron(LdL, I) - 0.5 * np.kron(I, LdL.T))
    return Lv


def rk4_density(sys, rho0, nsteps=None):
    """RK4 of vec(rho) under the generator; rho0 and the result are D x D."""
    N = sys.N if nsteps is None else nsteps
    dt = sys.dt
    v = np.array(rho0, dtype=np.complex128).reshape(-1)
    for n in range(N):
        A1, A2, A4 = liouvillian(sys, n, 0), liouvillian(sys, n, 1), liouvillian(sys, n, 2)
        k1 = A1 @ v
        k2 = A2 @ (v + 0.5 * dt * k1)
        k3 = A2 @ (v + 0.5 * dt * k2)
        k4 = A4 @ (v + dt * k3)
        v = v + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return v.reshape(sys.D, sys.D)


def to_lab(sys, rho_frame, nsteps=None):
    """Lab-frame density matrix from the frame's (exact diagonal phases, R1)."""
    if sys.frame == "lab":
        return rho_frame
    N = sys.N if nsteps is None else nsteps
    ph = np.exp(-1j * sys.hd_diag() * N * sys.dt)
    return ph[:, None] * rho_frame * np.conj(ph)[None, :]


def evolve_density(wl, rho0, nsteps=None):
    """Lab-frame rho(T) of the workload from rho0 (D x D)."""
    sys = OracleSystem(wl)
    return to_lab(sys, rk4_density(sys, rho0, nsteps), nsteps)


def gate_fidelity(wl, nsteps=None):
    """Average gate fidelity of the open evolution on the computational states against
    the workload's target unitary T (D_c x D_c): the channel's superoperator on the
    computational block, S[(a, b), (j, k)] = <c_a| E(|c_j><c_k|) |c_b>, one density-matrix
    evolution per (j, k); the entanglement (process) fidelity F_pro = sum conj(S_T) S / D_c^2
    with S_T = T (x) T^*; and F_avg = (D_c^2 F_pro + P) / (D_c (D_c + 1)) with P = sum_j
    tr P_c E(|c_j><c_j|) P_c the population kept in the computational block (Nielsen's
    relation, which Eq. D2 restates through an operator basis, written for a channel
    that may leak: P = D_c without leakage, and F_avg reduces to R10's
    (tr M M^dag + |tr M|^2) / (D_c (D_c + 1)) for a closed evolution)."""
    from .evolve import comp_map
    sys = OracleSystem(wl)
    comp, _ = comp_map(sys)
    Dc = len(comp)
    T = np.asarray(wl["target"], dtype=np.complex128)
    S = np.zeros((Dc * Dc, Dc * Dc), dtype=np.complex128)
    for j in range(Dc):
        for k in range(Dc):
            rho0 = np.zeros((sys.D, sys.D), dtype=np.complex128)
            rho0[comp[j], comp[k]] = 1.0
            rho = to_lab(sys, rk4_density(sys, rho0, nsteps), nsteps)
            S[:, j * Dc + k] = rho[np.ix_(comp, comp)].reshape(-1)
    S_T = np.kron(T, T.conj())
    F_pro = np.real(np.sum(np.conj(S_T) * S)) / Dc ** 2
    kept = sum(np.real(S[a * Dc + a, j * Dc + j]) for a in range(Dc) for j in range(Dc))
    return (Dc * Dc * F_pro + kept) / (Dc * (Dc + 1.0)), F_pro


def gate_fidelity_pulse_gradient(wl):
    """F_avg of gate_fidelity and dF/d(pulse parameters) by the discrete adjoint of the
    superoperator RK4.  F is linear in S, F = Re sum conj(W) S with W = (S_T + K) /
    (D_c (D_c + 1)), K[(a, a), (j, j)] = 1 the kept-population indicator, so the co-state
    of each evolved |c_j><c_k| is W's column (j, k) on the computational block; it is
    pulled back through the frame phases and the RK4 steps with the generator's adjoint
    and contracted with dLv/dtheta = -i (dH (x) I - I (x) dH^T) at every stage (Sec. 2.5
    on the vectorised equation).  Pulse parameters only."""
    from .evolve import comp_map
    from .system import n_pulse_params
    sys = OracleSystem(wl)
    comp, _ = comp_map(sys)
    Dc, D, N, dt = len(comp), sys.D, sys.N, sys.dt
    T = np.asarray(wl["target"], dtype=np.complex128)
    S_T = np.kron(T, T.conj())
    W = S_T / (Dc * (Dc + 1.0))
    for a in range(Dc):
        for j in range(Dc):
            W[a * Dc + a, j * Dc + j] += 1.0 / (Dc * (Dc + 1.0))
    prms = [p for p in sys.param_list() if p[0] == "pulse"]
    I = np.eye(D, dtype=np.complex128)
    grad = np.zeros(len(prms))
    F = 0.0
    for j in range(Dc):
        for k in range(Dc):
            v = np.zeros(D * D, dtype=np.complex128)
            v[comp[j] * D + comp[k]] = 1.0
            hist = [v.copy()]
            for n in range(N):
                A1, A2, A4 = liouvillian(sys, n, 0), liouvillian(sys, n, 1), liouvillian(sys, n, 2)
                k1 = A1 @ v
                k2 = A2 @ (v + 0.5 * dt * k1)
                k3 = A2 @ (v + 0.5 * dt * k2)
                k4 = A4 @ (v + dt * k3)
                v = v + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
                hist.append(v.copy())
            rho = to_lab(sys, v.reshape(D, D))
            col = W[:, j * Dc + k].reshape(Dc, Dc)
            F += np.real(np.sum(np.conj(col) * rho[np.ix_(comp, comp)]))
            bar_lab = np.zeros((D, D), dtype=np.complex128)
            bar_lab[np.ix_(comp, comp)] = col
            if sys.frame == "lab":
                bar = bar_lab.reshape(-1)
            else:
                ph = np.exp(-1j * sys.hd_diag() * N * dt)
                bar = (np.conj(ph)[:, None] * bar_lab * ph[None, :]).reshape(-1)
            for n in range(N - 1, -1, -1):
                y1 = hist[n]
                A1, A2, A4 = liouvillian(sys, n, 0), liouvillian(sys, n, 1), liouvillian(sys, n, 2)
                k1 = A1 @ y1
                y2 = y1 + 0.5 * dt * k1
                k2 = A2 @ y2
                y3 = y1 + 0.5 * dt * k2
                k3 = A2 @ y3
                y4 = y1 + dt * k3
                kb4 = (dt / 6.0) * bar
                yb4 = A4.conj().T @ kb4
                kb3 = (dt / 3.0) * bar + dt * yb4
                yb3 = A2.conj().T @ kb3
                kb2 = (dt / 3.0) * bar + 0.5 * dt * yb3
                yb2 = A2.conj().T @ kb2
                kb1 = (dt / 6.0) * bar + 0.5 * dt * yb2
                for p, prm in enumerate(prms):
                    d = []
                    for jj in (0, 1, 2):
                        dH = sys.dH(n, jj, prm)
                        d.append(-1j * (np.kron(dH, I) - np.kron(I, dH.T)))
                    grad[p] += np.real(np.vdot(kb1, d[0] @ y1) + np.vdot(kb2, d[1] @ y2)
                                       + np.vdot(kb3, d[1] @ y3) + np.vdot(kb4, d[2] @ y4))
                bar = bar + yb2 + yb3 + yb4 + A1.conj().T @ kb1
    return F, grad


def doubled_terms(sys, n, j):
    """The generator as local terms on 2 nq doubled modes (ket modes 0..nq-1, bra modes
    nq..2nq-1, row-major vec(rho) index = ket index * D + bra index): Lv = -i H_eff with
    H_eff = sum of 1-body terms {mode: d x d} and 2-body terms (mode a, A, mode b, B)
    of the Kronecker form the evolution kernels apply, with complex, non-Hermitian
    factors:
      ket 1-body  H_i(t) - (i/2) sum_c gamma_c L_c^dag L_c        (c on mode i)
      bra 1-body -H_i(t)^T - (i/2) sum_c gamma_c (L_c^dag L_c)^T
      ket 2-body  J A (x) B;   bra 2-body  -J A^T (x) B^T
      jump        i gamma_c L_c (ket i) (x) L_c^* (bra i).
    Returns (one, two): one[m] a d x d matrix per doubled mode, two a list of
    (a, A, b, B)."""
    t = stage_time(n, j, sys.dt)
    nq = sys.nq
    one = []
    for side in (0, 1):
        for i in range(nq):
            d = sys.dims[i]
            h = np.zeros((d, d), dtype=np.complex128)
            if sys.frame == "lab":
                h += np.diag(sys.modes[i]["E"])
            for k, dr in enumerate(sys.drives):
                if dr["mode"] == i:
                    h += sys.coeff(k, n, j) * sys.frame_op(sys.op(i, dr["op"]), i, t)
            anti = np.zeros((d, d), dtype=np.complex128)
            for c in sys.wl.get("collapse", []):
                if c["mode"] == i:
                    L = sys.frame_op(np.asarray(c["L"], dtype=np.complex128), i, t)
                    anti += c["rate"] * (L.conj().T @ L)
            one.append(h - 0.5j * anti if side == 0 else -h.T - 0.5j * anti.T)
    two = []
    for cpl in sys.couplings:
        A = sys.frame_op(sys.op(cpl["a"], cpl["op_a"]), cpl["a"], t)
        B = sys.frame_op(sys.op(cpl["b"], cpl["op_b"]), cpl["b"], t)
        two.append((cpl["a"], cpl["J"] * A, cpl["b"], B))
        two.append((nq + cpl["a"], -cpl["J"] * A.T, nq + cpl["b"], B.T))
    for c in sys.wl.get("collapse", []):
        i = c["mode"]
        L = sys.frame_op(np.asarray(c["L"], dtype=np.complex128), i, t)
        two.append((i, 1j * c["rate"] * L, nq + i, L.conj()))
    return one, two
