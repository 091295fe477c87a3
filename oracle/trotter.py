"""Second-order Suzuki-Trotter evolution (oracle; test infrastructure).

The paper's own solver (Sec. 2.3, App. A): the evolution over one step of length
dt is approximated by the palindromic product of local exponentials

    Q2(dt) = prod_{k=1..K} exp(-i H_k dt/2)  prod_{k=K..1} exp(-i H_k dt/2),

with H = sum_k H_k split into local terms acting on one or two subsystems
(Eq. 1).  Readings taken here (the paper does not fix them):

* the evolution runs in the lab frame, the 1-body terms carry the mode's level
  energies: H_i(t) = diag(E^(i)) + sum_{drives k on i} f_k(t) O_k, and the 2-body
  terms are the couplings J_e A_e (x) B_e (time independent);
* the terms are ordered 1-body in mode order, then the couplings in term order;
  the first factor in that order acts on the state first;
* a time-dependent term is evaluated at the step's midpoint t_n + dt/2 (where a
  piecewise-constant envelope takes its segment, reading R8), which keeps the
  product second order.

Each exponential is scipy.linalg.expm of the d x d (1-body) or d^2 x d^2
(np.kron, 2-body) matrix, applied to the state tensor along its modes.
"""
import numpy as np
from scipy.linalg import expm

from .system import OracleSystem


def _apply_1body(psi, U, i):
    """psi[..., a_i, ...] <- sum_b U[a, b] psi[..., b, ...] along mode axis i."""
    out = np.tensordot(U, psi, axes=([1], [i]))
    return np.moveaxis(out, 0, i)


def _apply_2body(psi, G, i, j, di, dj):
    """The d_i d_j x d_i d_j matrix G (row index a * d_j + b) on mode axes i, j."""
    G4 = G.reshape(di, dj, di, dj)
    out = np.tensordot(G4, psi, axes=([2, 3], [i, j]))
    return np.moveaxis(out, [0, 1], [i, j])


def local_terms(sys, n):
    """The 1-body matrices H_i(t_n + dt/2) and 2-body matrices J A (x) B of step n."""
    one = []
    for i, m in enumerate(sys.modes):
        H = np.diag(m["E"]).astype(np.complex128)
        for k, dr in enumerate(sys.drives):
            if dr["mode"] == i:
                H = H + sys.coeff(k, n, 1) * sys.op(i, dr["op"])
        one.append(H)
    two = []
    for c in sys.couplings:
        two.append((c["a"], c["b"], c["J"] * np.kron(sys.op(c["a"], c["op_a"]), sys.op(c["b"], c["op_b"]))))
    return one, two


def q2_evolve(sys, psi0, nsteps=None):
    """Lab-frame columns after N steps of Q2 from the columns psi0 (D x S)."""
    N = sys.N if nsteps is None else nsteps
    dt = sys.dt
    S = psi0.shape[1]
    psi = np.array(psi0, dtype=np.complex128).reshape(list(sys.dims) + [S])
    _, two = local_terms(sys, 0)
    G = [(a, b, expm(-1j * M * dt / 2)) for a, b, M in two]
    for n in range(N):
        one, _ = local_terms(sys, n)
        U = [expm(-1j * H * dt / 2) for H in one]
        seq = [("1", i, U[i]) for i in range(sys.nq)] + [("2", e, G[e]) for e in range(len(G))]
        for kind, idx, X in seq + seq[::-1]:
            if kind == "1":
                psi = _apply_1body(psi, X, idx)
            else:
                a, b, M = X
                psi = _apply_2body(psi, M, a, b, sys.dims[a], sys.dims[b])
    return psi.reshape(sys.D, S)


def q2_evolve_and_fidelity(wl):
    """Q2 evolution of the workload's columns and the fidelities of the lab-frame
    states (the frame of a Q2 solve is always the lab frame)."""
    from .evolve import initial_columns, fidelities
    sys = OracleSystem(dict(wl, frame="lab"))
    psi = q2_evolve(sys, initial_columns(sys, wl["col_index"]))
    Favg, Fst, Uc = fidelities(sys, psi)
    return {"psi_lab": psi, "F_avg": Favg, "F_state": Fst, "Uc": Uc, "sys": sys}


def q2_pulse_gradient(wl, kind=None):
    """F and dF/d(pulse parameters) of the Q2 evolution, by its discrete adjoint.

    With psi_m = X_m psi_{m-1} over the factors X_m of every step in order and the
    co-state psibar = dF/dRe psi + i dF/dIm psi of the final lab-frame columns,
    psibar_{m-1} = X_m^dag psibar_m and dF/dtheta = sum_m Re <psibar_m, dX_m/dtheta psi_{m-1}>.
    A 1-body factor is X = exp(A), A = -i (dt/2) H_i(t_n + dt/2), so
    dX/df_k = L(A, -i (dt/2) O_k), the Frechet derivative of expm (scipy's
    expm_frechet), for each drive k on mode i; f_k(t) = E_k(t) cos(omega t + phase)
    carries the pulse parameters through the envelope (reading R8 for PWC).
    Returns (F, gradient over the pulse parameters in sg_param order)."""
    from scipy.linalg import expm_frechet
    from .evolve import initial_columns, fidelity_and_costate
    from .system import envelope, n_pulse_params, stage_time
    sys = OracleSystem(dict(wl, frame="lab"))
    kind = kind or wl["fid_kind"]
    dt, N, S = sys.dt, sys.N, len(wl["col_index"])
    psi = initial_columns(sys, wl["col_index"]).reshape(list(sys.dims) + [S])
    _, two = local_terms(sys, 0)
    G = [(a, b, expm(-1j * M * dt / 2)) for a, b, M in two]
    tape = []                                   # (factor, mode/edge, state before, step)
    for n in range(N):
        one, _ = local_terms(sys, n)
        A = [-1j * (dt / 2) * H for H in one]
        seq = [("1", i, A[i]) for i in range(sys.nq)] + [("2", e, None) for e in range(len(G))]
        for kind_f, idx, Ai in seq + seq[::-1]:
            tape.append((kind_f, idx, Ai, psi.copy(), n))
            if kind_f == "1":
                psi = _apply_1body(psi, expm(Ai), idx)
            else:
                a, b, M = G[idx]
                psi = _apply_2body(psi, M, a, b, sys.dims[a], sys.dims[b])
    F, bar = fidelity_and_costate(sys, psi.reshape(sys.D, S), kind)
    bar = bar.reshape(list(sys.dims) + [S])
    gf = np.zeros((len(sys.drives), N))          # dF/df_k at the midpoint of step n
    for kind_f, idx, Ai, before, n in reversed(tape):
        if kind_f == "1":
            X = expm(Ai)
            for k, dr in enumerate(sys.drives):
                if dr["mode"] != idx:
                    continue
                L = expm_frechet(Ai, -1j * (dt / 2) * sys.op(idx, dr["op"]), compute_expm=False)
                gf[k, n] += np.real(np.vdot(bar, _apply_1body(before, L, idx)))
            bar = _apply_1body(bar, X.conj().T, idx)
        else:
            a, b, M = G[idx]
            bar = _apply_2body(bar, M.conj().T, a, b, sys.dims[a], sys.dims[b])
    grad = []
    for k, dr in enumerate(sys.drives):
        g = np.zeros(n_pulse_params(dr))
        for n in range(N):
            t = stage_time(n, 1, dt)
            _, dE = envelope(dr, n, 1, dt)
            c = np.cos(sys.omega_d[k] * t + dr.get("phase", 0.0))
            g += gf[k, n] * c * np.asarray(dE)
        grad.extend(g)
    return F, np.array(grad)


def q2_fidelity(wl, kind=None):
    """F of the Q2 evolution (for finite differences)."""
    r = q2_evolve_and_fidelity(wl)
    return r["F_avg"] if (kind or wl["fid_kind"]) == "avg" else r["F_state"]
