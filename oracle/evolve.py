"""Fixed-step RK4 evolution, fidelity, discrete adjoint, tangent-linear and
finite differences (oracle; test infrastructure).

RK4 (classic, reading R1/R2) for dy/dt = -i H(t) y, stage times t_n + {0, 1/2, 1/2, 1} dt:
    k1 = A(t_n) psi,          y2 = psi + dt/2 k1
    k2 = A(t_n + dt/2) y2,    y3 = psi + dt/2 k2
    k3 = A(t_n + dt/2) y3,    y4 = psi + dt k3
    k4 = A(t_n + dt) y4,      psi' = psi + dt/6 (k1 + 2 k2 + 2 k3 + k4)
with A = -i H.  In the interaction frame the lab-frame result is
psi_lab(T) = exp(-i H_d T) psi_I(T).

Fidelities (reading R10): with U_c the computational-subspace block of the
evolved columns and T the target (Dc x Dc), M = T^dag U_c,
    F_avg   = (tr(M M^dag) + |tr M|^2) / (Dc (Dc + 1))          (Eq. D2)
    F_state = |(1/S) sum_s <t_s | psi_s>|^2                      (Eq. 13)

Gradient (Sec. 2.5, Eqs. 7-12; reading R12): the exact derivative of the
discrete RK4 map.  Complex co-states follow dL = Re <xbar, dx>, <a,b> = sum conj(a) b,
so a linear map x' = A x pulls back as xbar = A^dag x'bar and
dL/dtheta = sum over stages Re <kbar_s, (dA_s/dtheta) y_s>.
"""
import numpy as np

from .system import OracleSystem


# ----------------------------------------------------------------------------
# forward evolution
# ----------------------------------------------------------------------------
def initial_columns(sys, col_index):
    psi = np.zeros((sys.D, len(col_index)), dtype=np.complex128)
    for s, r in enumerate(col_index):
        psi[int(r), s] = 1.0
    return psi


def rk4_evolve(sys, psi0, nsteps=None, store=False):
    """Dense RK4: H(t) formed by np.kron at every stage time."""
    N = sys.N if nsteps is None else nsteps
    dt = sys.dt
    psi = np.array(psi0, dtype=np.complex128)
    hist = [psi.copy()] if store else None
    for n in range(N):
        A1 = -1j * sys.hamiltonian(n, 0)
        A2 = -1j * sys.hamiltonian(n, 1)
        A4 = -1j * sys.hamiltonian(n, 2)
        k1 = A1 @ psi
        k2 = A2 @ (psi + 0.5 * dt * k1)
        k3 = A2 @ (psi + 0.5 * dt * k2)
        k4 = A4 @ (psi + dt * k3)
        psi = psi + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if store:
            hist.append(psi.copy())
    return (psi, hist) if store else psi


def rk4_evolve_matrix_free(sys, psi0, nsteps=None):
    """Same RK4, with H(t) applied by per-mode tensor contraction (App. B)."""
    N = sys.N if nsteps is None else nsteps
    dt = sys.dt
    psi = np.array(psi0, dtype=np.complex128)
    for n in range(N):
        f = lambda j, y: -1j * sys.apply_matrix_free(n, j, y)
        k1 = f(0, psi)
        k2 = f(1, psi + 0.5 * dt * k1)
        k3 = f(1, psi + 0.5 * dt * k2)
        k4 = f(2, psi + dt * k3)
        psi = psi + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return psi


def frame_epilogue(sys, psi_i, nsteps=None):
    """psi_lab = exp(-i H_d T) psi_I (identity in the lab frame)."""
    if sys.frame == "lab":
        return psi_i
    N = sys.N if nsteps is None else nsteps
    T = N * sys.dt
    return np.exp(-1j * sys.hd_diag() * T)[:, None] * psi_i


# ----------------------------------------------------------------------------
# fidelity (Eq. 13, Eq. D2, reading R10)
# ----------------------------------------------------------------------------
def comp_map(sys):
    """Flat indices of the computational states and the comp label of each evolved
    column (-1 if it is not a computational state).  A computational state has
    every qubit mode in level 0 or 1 and every coupler mode (workload mode flag
    "coupler") in level 0; label j counts over the qubit modes, first qubit most
    significant."""
    qubits = [i for i in range(sys.nq) if not sys.wl["modes"][i].get("coupler")]
    comp = []
    for j in range(2 ** len(qubits)):
        level = [0] * sys.nq
        for b, i in enumerate(qubits):
            level[i] = (j >> (len(qubits) - 1 - b)) & 1
        r = 0
        for i in range(sys.nq):
            r = r * sys.dims[i] + level[i]
        comp.append(r)
    label = {r: j for j, r in enumerate(comp)}
    cols = [label.get(int(r), -1) for r in sys.wl["col_index"]]
    return np.array(comp), cols


def fidelities(sys, psi_lab):
    """Returns (F_avg, F_state, U_c) where U_c[j', s] = <c_j'|psi_s> over comp rows."""
    comp, cols = comp_map(sys)
    T = np.asarray(sys.wl["target"], dtype=np.complex128)
    Dc = len(comp)
    Uc = psi_lab[comp, :]
    sel = [s for s, j in enumerate(cols) if j >= 0]
    z = sum(np.vdot(T[:, cols[s]], Uc[:, s]) for s in sel)
    F_state = abs(z / len(sel)) ** 2
    labels = sorted(cols[s] for s in sel)
    if labels == list(range(Dc)):
        U = np.zeros((Dc, Dc), dtype=np.complex128)
        for s in sel:
            U[:, cols[s]] = Uc[:, s]
        M = T.conj().T @ U
        F_avg = (np.real(np.trace(M @ M.conj().T)) + abs(np.trace(M)) ** 2) / (Dc * (Dc + 1))
    else:
        F_avg = float("nan")
    return F_avg, F_state, Uc


def fidelity_and_costate(sys, psi_lab, kind):
    """F (kind 'avg' or 'state') and its co-state Fbar = dF/dRe psi + i dF/dIm psi
    (lab frame, shape D x S)."""
    comp, cols = comp_map(sys)
    T = np.asarray(sys.wl["target"], dtype=np.complex128)
    F, barc = block_fidelity_and_costate(T, psi_lab[comp, :], cols, kind)
    bar = np.zeros_like(psi_lab)
    bar[comp, :] = barc
    return F, bar


def block_fidelity_and_costate(T, Uc, cols, kind):
    """F of the computational block Uc[j', s] = <c_j'|psi_s> (column s carrying label
    cols[s], -1 for none) and its co-state dF/dRe Uc + i dF/dIm Uc (D_c x S)."""
    Dc = T.shape[0]
    sel = [s for s, j in enumerate(cols) if j >= 0]
    barc = np.zeros_like(Uc)
    if kind == "state":
        S = len(sel)
        z = sum(np.vdot(T[:, cols[s]], Uc[:, s]) for s in sel)
        for s in sel:
            barc[:, s] = (2.0 * z / S ** 2) * T[:, cols[s]]
        return abs(z / S) ** 2, barc
    U = np.zeros((Dc, Dc), dtype=np.complex128)
    for s in sel:
        U[:, cols[s]] = Uc[:, s]
    M = T.conj().T @ U
    trM = np.trace(M)
    F = (np.real(np.trace(M @ M.conj().T)) + abs(trM) ** 2) / (Dc * (Dc + 1))
    Ubar = 2.0 * (T @ M + trM * T) / (Dc * (Dc + 1))
    for s in sel:
        barc[:, s] = Ubar[:, cols[s]]
    return F, barc


def evolve_and_fidelity(wl, matrix_free=False):
    sys = OracleSystem(wl)
    psi0 = initial_columns(sys, wl["col_index"])
    psi = rk4_evolve_matrix_free(sys, psi0) if matrix_free else rk4_evolve(sys, psi0)
    psi_lab = frame_epilogue(sys, psi)
    Favg, Fst, Uc = fidelities(sys, psi_lab)
    return {"psi_lab": psi_lab, "F_avg": Favg, "F_state": Fst, "Uc": Uc, "sys": sys}


# ----------------------------------------------------------------------------
# parameters
# ----------------------------------------------------------------------------
def param_vector(wl):
    """Flat parameter values in OracleSystem.param_list order."""
    out = []
    for dr in wl["drives"]:
        if dr["env"] == "pwc":
            out.extend(dr["amps"])
        else:
            out.append(dr["amp"])
    for m in wl["modes"]:
        out.extend([m["ej"], m["ec"], m.get("el", 0.0)])
    for c in wl["couplings"]:
        out.append(c["J"])
    return np.array(out, dtype=np.float64)


def set_param_vector(wl, theta):
    import copy
    w = copy.deepcopy(wl)
    i = 0
    for dr in w["drives"]:
        if dr["env"] == "pwc":
            n = len(dr["amps"])
            dr["amps"] = list(theta[i:i + n])
            i += n
        else:
            dr["amp"] = float(theta[i])
            i += 1
    for m in w["modes"]:
        m["ej"], m["ec"] = float(theta[i]), float(theta[i + 1])
        if m["kind"] == "fluxonium":
            m["el"] = float(theta[i + 2])
        i += 3
    for c in w["couplings"]:
        c["J"] = float(theta[i])
        i += 1
    return w


# ----------------------------------------------------------------------------
# discrete adjoint (Sec. 2.5)
# ----------------------------------------------------------------------------
def adjoint_gradient(wl, kind=None, nsteps=None):
    """dF/dtheta for every parameter by the exact discrete adjoint of RK4.
    Forward states are stored (the oracle does not need checkpointing)."""
    sys = OracleSystem(wl)
    kind = kind or wl["fid_kind"]
    N = sys.N if nsteps is None else nsteps
    psi0 = initial_columns(sys, wl["col_index"])
    psiT, hist = rk4_evolve(sys, psi0, N, store=True)
    psi_lab = frame_epilogue(sys, psiT, N)
    F, bar_lab = fidelity_and_costate(sys, psi_lab, kind)
    grad, prms = adjoint_from_costate(sys, hist, psi_lab, bar_lab, N)
    return F, grad, prms


def adjoint_from_costate(sys, hist, psi_lab, bar_lab, N, with_bar=False):
    """Pull a lab-frame co-state back through the frame epilogue and N RK4 steps:
    returns (sum over stages of Re <kbar_s, dA_s/dtheta y_s> + the frame term, params),
    and with with_bar the co-state of the initial columns as a third item (the frame is
    the identity at t = 0)."""
    dt = sys.dt
    prms = sys.param_list()
    grad = np.zeros(len(prms))
    # frame epilogue: psi_lab = Phi psi_I, Phi = exp(-i Hd T)
    if sys.frame == "lab":
        bar = bar_lab.copy()
    else:
        T = N * dt
        phi = np.exp(-1j * sys.hd_diag() * T)
        bar = np.conj(phi)[:, None] * bar_lab
        for p, prm in enumerate(prms):
            dd = sys.dHd_diag(prm)
            if np.any(dd):
                dpsi = (-1j * T * dd)[:, None] * psi_lab
                grad[p] += np.real(np.vdot(bar_lab, dpsi))
    for n in range(N - 1, -1, -1):
        psi = hist[n]
        H1 = sys.hamiltonian(n, 0)
        H2 = sys.hamiltonian(n, 1)
        H4 = sys.hamiltonian(n, 2)
        A1, A2, A4 = -1j * H1, -1j * H2, -1j * H4
        y1 = psi
        k1 = A1 @ y1
        y2 = psi + 0.5 * dt * k1
        k2 = A2 @ y2
        y3 = psi + 0.5 * dt * k2
        k3 = A2 @ y3
        y4 = psi + dt * k3
        kb4 = (dt / 6.0) * bar
        yb4 = A4.conj().T @ kb4
        kb3 = (dt / 3.0) * bar + dt * yb4
        yb3 = A2.conj().T @ kb3
        kb2 = (dt / 3.0) * bar + 0.5 * dt * yb3
        yb2 = A2.conj().T @ kb2
        kb1 = (dt / 6.0) * bar + 0.5 * dt * yb2
        for p, prm in enumerate(prms):
            dA1 = -1j * sys.dH(n, 0, prm)
            dA2 = -1j * sys.dH(n, 1, prm)
            dA4 = -1j * sys.dH(n, 2, prm)
            grad[p] += np.real(np.vdot(kb1, dA1 @ y1) + np.vdot(kb2, dA2 @ y2)
                               + np.vdot(kb3, dA2 @ y3) + np.vdot(kb4, dA4 @ y4))
        bar = bar + yb2 + yb3 + yb4 + A1.conj().T @ kb1
    if with_bar:
        return grad, prms, bar
    return grad, prms


# ----------------------------------------------------------------------------
# independent checks of the adjoint
# ----------------------------------------------------------------------------
def tangent_linear_derivative(wl, prm_index, kind=None, nsteps=None):
    """dF/dtheta for ONE parameter by forward-mode differentiation of the same
    discrete RK4 map (an independent derivative of the same function)."""
    sys = OracleSystem(wl)
    kind = kind or wl["fid_kind"]
    N = sys.N if nsteps is None else nsteps
    dt = sys.dt
    prm = sys.param_list()[prm_index]
    psi = initial_columns(sys, wl["col_index"])
    dpsi = np.zeros_like(psi)
    for n in range(N):
        A = [-1j * sys.hamiltonian(n, j) for j in (0, 1, 2)]
        dA = [-1j * sys.dH(n, j, prm) for j in (0, 1, 2)]
        k1 = A[0] @ psi
        dk1 = A[0] @ dpsi + dA[0] @ psi
        y2, dy2 = psi + 0.5 * dt * k1, dpsi + 0.5 * dt * dk1
        k2 = A[1] @ y2
        dk2 = A[1] @ dy2 + dA[1] @ y2
        y3, dy3 = psi + 0.5 * dt * k2, dpsi + 0.5 * dt * dk2
        k3 = A[1] @ y3
        dk3 = A[1] @ dy3 + dA[1] @ y3
        y4, dy4 = psi + dt * k3, dpsi + dt * dk3
        k4 = A[2] @ y4
        dk4 = A[2] @ dy4 + dA[2] @ y4
        psi = psi + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        dpsi = dpsi + (dt / 6.0) * (dk1 + 2 * dk2 + 2 * dk3 + dk4)
    psi_lab = frame_epilogue(sys, psi, N)
    if sys.frame == "lab":
        dpsi_lab = dpsi
    else:
        T = N * dt
        ph = np.exp(-1j * sys.hd_diag() * T)[:, None]
        dpsi_lab = ph * dpsi + (-1j * T * sys.dHd_diag(prm))[:, None] * psi_lab
    F, bar = fidelity_and_costate(sys, psi_lab, kind)
    return np.real(np.vdot(bar, dpsi_lab))


def finite_difference_gradient(wl, prm_indices, h_rel=1e-5, h_amp=1e-7, kind=None,
                               nsteps=None):
    """Central differences of F through the whole pipeline (eigensolve included)."""
    kind = kind or wl["fid_kind"]
    theta = param_vector(wl)
    sys0 = OracleSystem(wl)
    prms = sys0.param_list()
    out = []

    def F_of(th):
        w = set_param_vector(wl, th)
        s = OracleSystem(w)
        N = s.N if nsteps is None else nsteps
        psi = rk4_evolve(s, initial_columns(s, w["col_index"]), N)
        F, _ = fidelity_and_costate(s, frame_epilogue(s, psi, N), kind)
        return F

    for p in prm_indices:
        kindp = prms[p][0]
        h = h_amp if kindp == "pulse" else h_rel * max(abs(theta[p]), 1e-3)
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        out.append((F_of(tp) - F_of(tm)) / (2.0 * h))
    return np.array(out)
