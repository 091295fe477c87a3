"""Suzuki-Trotter evolution, orders 1, 2 and 4 (oracle; test infrastructure).

The paper's own solver (Sec. 2.3, App. A): the evolution over one step of length
dt is approximated by the first-order product of local exponentials

    Q1(dt) = prod_{k=1..K} exp(-i H_k dt)

or by the palindromic one

    Q2(dt) = prod_{k=1..K} exp(-i H_k dt/2)  prod_{k=K..1} exp(-i H_k dt/2),

with H = sum_k H_k split into local terms acting on one or two subsystems
(Eq. 1), and the fourth-order products of App. A built from it:

    Q4(dt)  = Q2(p dt) Q2((1 - 2p) dt) Q2(p dt),   p = 1 / (2 - 2^(1/3))   (real),
    Q4j(dt) = Q2(p dt) Q2(p* dt),                  p = (3 - i sqrt(3)) / 6 (complex).

Readings taken here (the paper does not fix them):

* the evolution runs in the lab frame, the 1-body terms carry the mode's level
  energies: H_i(t) = diag(E^(i)) + sum_{drives k on i} f_k(t) O_k, and the 2-body
  terms are the couplings J_e A_e (x) B_e (time independent);
* the terms are ordered 1-body in mode order, then the couplings in term order;
  the first factor in that order acts on the state first;
* Q1 applies the terms once each, in that order, over the full step, with the
  time-dependent terms at the step's midpoint t_n + dt/2;
* a time-dependent term is evaluated at the midpoint of its Q2 sub-step: for a
  sub-step c dt that starts after the fraction s of the step, at t_n + (s + c/2) dt
  (Q2: t_n + dt/2, which keeps the product second order; Q4: t_n + {p/2, 1/2,
  1 - p/2} dt, the time-symmetric composition that keeps fourth order).  For the
  complex Q4j these midpoints are complex, t_n + {p/2, p + p*/2} dt, and the drive
  coefficient is continued analytically there (Gaussian and cosine envelopes and the
  carrier cos(omega t + phase) at the complex time); taking the real parts instead
  makes Q4j first order under a time-dependent drive;
* a piecewise-constant envelope takes the segment of the step's midpoint (reading
  R8) for every sub-step of the step; the carrier is evaluated at the sub-step time.

App. A prints p of Q4j garbled ("3 - sqrt(3) i / 6"); the reading (3 - i sqrt(3))/6
is the one with p + p* = 1 and p^3 + p*^3 = 0.  Those conditions cancel the local
error term of order dt^3, so the product's local error is O(dt^4) and its global
error O(dt^3): the composition (p, p*) is not palindromic, so the even term of the
next order does not cancel as it does for Q4.

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


_P4 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
_P4J = (3.0 - 1j * np.sqrt(3.0)) / 6.0
# per scheme its Q2 sub-steps: (c, tau) = step fraction (complex for Q4j) and the
# fraction of the step at which the time-dependent terms are evaluated
SCHEMES = {
    "q2": [(1.0, 0.5)],
    "q4": [(_P4, _P4 / 2), (1.0 - 2.0 * _P4, 0.5), (_P4, 1.0 - _P4 / 2)],
    "q4j": [(_P4J, _P4J / 2), (np.conj(_P4J), _P4J + np.conj(_P4J) / 2)],
}


def sub_envelope(dr, n, t, dt):
    """E(t) and dE/dparams of drive dr at time t inside step n: Gaussian and cosine
    envelopes at t (cosine cut where the step's midpoint lies past the pulse), a
    piecewise-constant envelope from the segment of the step's midpoint (R8)."""
    from .system import envelope, pulse_half_steps
    if dr["env"] == "gaussian":
        g = np.exp(-((t - dr["t0"]) ** 2) / (2.0 * dr["sigma"] ** 2))
        return dr["amp"] * g, [g]
    if dr["env"] == "cosine":
        if 2 * n + 1 > pulse_half_steps(dr["length"], dt):
            return 0.0, [0.0]
        c = 0.5 * (1.0 - np.cos(2.0 * np.pi * t / dr["length"]))
        return dr["amp"] * c, [c]
    return envelope(dr, n, 1, dt)


def sub_time(sys, n, tau):
    """t_n + tau dt (exactly the stage time of the midpoint for tau = 1/2; complex
    for the sub-steps of Q4j)."""
    from .system import stage_time
    return stage_time(n, 1, sys.dt) + (tau - 0.5) * sys.dt


def local_terms(sys, n, tau=0.5):
    """The 1-body matrices H_i(t_n + tau dt) and 2-body matrices J A (x) B of step n."""
    t = sub_time(sys, n, tau)
    one = []
    for i, m in enumerate(sys.modes):
        H = np.diag(m["E"]).astype(np.complex128)
        for k, dr in enumerate(sys.drives):
            if dr["mode"] == i:
                E, _ = sub_envelope(dr, n, t, sys.dt)
                f = E * np.cos(sys.omega_d[k] * t + dr.get("phase", 0.0))
                H = H + f * sys.op(i, dr["op"])
        one.append(H)
    two = []
    for c in sys.couplings:
        two.append((c["a"], c["b"], c["J"] * np.kron(sys.op(c["a"], c["op_a"]), sys.op(c["b"], c["op_b"]))))
    return one, two


def q2_evolve(sys, psi0, nsteps=None, scheme="q2"):
    """Lab-frame columns after N steps of the scheme ("q1", "q2", "q4", "q4j") from the
    columns psi0 (D x S): per step, Q1's product once, or the Q2 sub-steps in order."""
    N = sys.N if nsteps is None else nsteps
    dt = sys.dt
    S = psi0.shape[1]
    psi = np.array(psi0, dtype=np.complex128).reshape(list(sys.dims) + [S])
    _, two = local_terms(sys, 0)
    if scheme == "q1":
        for n in range(N):
            one, _ = local_terms(sys, n, 0.5)
            for i, H in enumerate(one):
                psi = _apply_1body(psi, expm(-1j * H * dt), i)
            for a, b, M in two:
                psi = _apply_2body(psi, expm(-1j * M * dt), a, b, sys.dims[a], sys.dims[b])
        return psi.reshape(sys.D, S)
    for n in range(N):
        for c, tau in SCHEMES[scheme]:
            one, _ = local_terms(sys, n, tau)
            U = [expm(-1j * c * H * dt / 2) for H in one]
            G = [(a, b, expm(-1j * c * M * dt / 2)) for a, b, M in two]
            seq = [("1", i, U[i]) for i in range(sys.nq)] + [("2", e, G[e]) for e in range(len(G))]
            for kind, idx, X in seq + seq[::-1]:
                if kind == "1":
                    psi = _apply_1body(psi, X, idx)
                else:
                    a, b, M = X
                    psi = _apply_2body(psi, M, a, b, sys.dims[a], sys.dims[b])
    return psi.reshape(sys.D, S)


def q2_evolve_and_fidelity(wl, scheme="q2"):
    """Evolution of the workload's columns by the scheme and the fidelities of the
    lab-frame states (the frame of a Suzuki-Trotter solve is always the lab frame)."""
    from .evolve import initial_columns, fidelities
    sys = OracleSystem(dict(wl, frame="lab"))
    psi = q2_evolve(sys, initial_columns(sys, wl["col_index"]), scheme=scheme)
    Favg, Fst, Uc = fidelities(sys, psi)
    return {"psi_lab": psi, "F_avg": Favg, "F_state": Fst, "Uc": Uc, "sys": sys}


def q2_pulse_gradient(wl, kind=None, scheme="q2"):
    """F and dF/d(pulse parameters) of the scheme's evolution, by its discrete adjoint.

    With psi_m = X_m psi_{m-1} over the factors X_m of every step in order and the
    co-state psibar = dF/dRe psi + i dF/dIm psi of the final lab-frame columns,
    psibar_{m-1} = X_m^dag psibar_m and dF/dtheta = sum_m Re <psibar_m, dX_m/dtheta psi_{m-1}>.
    A 1-body factor is X = exp(A), A = -i c h H_i(t_n + tau dt) with h = dt/2 for the
    Q2 sub-steps and h = dt for Q1 (each term once per step, at the step's midpoint), so
    dX/df_k = L(A, -i c h O_k), the Frechet derivative of expm (scipy's
    expm_frechet), for each drive k on mode i; f_k(t) = E_k(t) cos(omega t + phase)
    carries the pulse parameters through the envelope (sub_envelope).
    Returns (F, gradient over the pulse parameters in sg_param order)."""
    from scipy.linalg import expm_frechet
    from .evolve import initial_columns, fidelity_and_costate
    from .system import n_pulse_params
    sys = OracleSystem(dict(wl, frame="lab"))
    kind = kind or wl["fid_kind"]
    dt, N, S = sys.dt, sys.N, len(wl["col_index"])
    q1 = scheme == "q1"
    subs = [(1.0, 0.5)] if q1 else SCHEMES[scheme]
    h = dt if q1 else dt / 2
    psi = initial_columns(sys, wl["col_index"]).reshape(list(sys.dims) + [S])
    _, two = local_terms(sys, 0)
    tape = []                                   # (factor, mode/edge, A or G, state before, step, sub-step)
    for n in range(N):
        for j, (c, tau) in enumerate(subs):
            one, _ = local_terms(sys, n, tau)
            A = [-1j * c * h * H for H in one]
            G = [(a, b, expm(-1j * c * M * h)) for a, b, M in two]
            seq = [("1", i, A[i]) for i in range(sys.nq)] + [("2", e, G[e]) for e in range(len(G))]
            for kind_f, idx, X in (seq if q1 else seq + seq[::-1]):
                tape.append((kind_f, idx, X, psi.copy(), n, j))
                if kind_f == "1":
                    psi = _apply_1body(psi, expm(X), idx)
                else:
                    a, b, M = X
                    psi = _apply_2body(psi, M, a, b, sys.dims[a], sys.dims[b])
    F, bar = fidelity_and_costate(sys, psi.reshape(sys.D, S), kind)
    bar = bar.reshape(list(sys.dims) + [S])
    # <psibar, dX/df_k psi> at each sub-step (complex: f_k is complex on the complex
    # time path of Q4j, where dF/dtheta = Re sum gf df_k/dtheta)
    gf = np.zeros((len(sys.drives), N, len(subs)), dtype=np.complex128)
    for kind_f, idx, X, before, n, j in reversed(tape):
        if kind_f == "1":
            c = subs[j][0]
            for k, dr in enumerate(sys.drives):
                if dr["mode"] != idx:
                    continue
                L = expm_frechet(X, -1j * c * h * sys.op(idx, dr["op"]), compute_expm=False)
                gf[k, n, j] += np.vdot(bar, _apply_1body(before, L, idx))
            bar = _apply_1body(bar, expm(X).conj().T, idx)
        else:
            a, b, M = X
            bar = _apply_2body(bar, M.conj().T, a, b, sys.dims[a], sys.dims[b])
    grad = []
    for k, dr in enumerate(sys.drives):
        g = np.zeros(n_pulse_params(dr))
        for n in range(N):
            for j, (c, tau) in enumerate(subs):
                t = sub_time(sys, n, tau)
                _, dE = sub_envelope(dr, n, t, dt)
                g += np.real(gf[k, n, j] * np.cos(sys.omega_d[k] * t + dr.get("phase", 0.0)) * np.asarray(dE))
        grad.extend(g)
    return F, np.array(grad)


def q2_fidelity(wl, kind=None, scheme="q2"):
    """F of the scheme's evolution (for finite differences)."""
    r = q2_evolve_and_fidelity(wl, scheme)
    return r["F_avg"] if (kind or wl["fid_kind"]) == "avg" else r["F_state"]


def trotter_full_gradient(wl, kind=None, scheme="q2"):
    """F and dF/dtheta for every parameter (pulse, device E_J/E_C/E_L, couplings J) of
    the scheme's evolution, by the discrete adjoint over its factors: for a factor
    X = exp(G) with generator G = -i c (dt/2) H_loc, dX/dtheta = L(G, -i c (dt/2) dH_loc/dtheta)
    (expm_frechet); a 1-body H_loc = diag(E_i) + sum f_k O_k varies with the pulse
    parameters (through f_k), the mode's device parameters (energies and operators,
    through the eigen-derivatives, and carriers tied to its 0-1 frequency); a coupling
    H_loc = J A (x) B with J and the two modes' device parameters.  Lab frame.  Returns
    (F, gradient in OracleSystem.param_list order)."""
    from scipy.linalg import expm_frechet
    from .evolve import initial_columns, fidelity_and_costate
    sys = OracleSystem(dict(wl, frame="lab"))
    kind = kind or wl["fid_kind"]
    dt, N, S = sys.dt, sys.N, len(wl["col_index"])
    subs = SCHEMES[scheme]
    prms = sys.param_list()
    derivs = {(i, p): sys.mode_derivs(i, p) for (pk, i, p) in prms if pk == "ham"}
    psi = initial_columns(sys, wl["col_index"]).reshape(list(sys.dims) + [S])
    _, two = local_terms(sys, 0)
    tape = []
    for n in range(N):
        for j, (c, tau) in enumerate(subs):
            one, _ = local_terms(sys, n, tau)
            seq = [("1", i, -1j * c * (dt / 2) * one[i]) for i in range(sys.nq)]
            seq += [("2", e, -1j * c * (dt / 2) * two[e][2]) for e in range(len(two))]
            for kind_f, idx, G in seq + seq[::-1]:
                tape.append((kind_f, idx, G, psi.copy(), n, j))
                X = expm(G)
                if kind_f == "1":
                    psi = _apply_1body(psi, X, idx)
                else:
                    a, b, _ = two[idx]
                    psi = _apply_2body(psi, X, a, b, sys.dims[a], sys.dims[b])
    F, bar = fidelity_and_costate(sys, psi.reshape(sys.D, S), kind)
    bar = bar.reshape(list(sys.dims) + [S])
    grad = np.zeros(len(prms))
    for kind_f, idx, G, before, n, j in reversed(tape):
        c, tau = subs[j]
        t = sub_time(sys, n, tau)
        scale = -1j * c * (dt / 2)
        for p, prm in enumerate(prms):
            pk, a, b = prm
            dH = None
            if kind_f == "1":
                i = idx
                if pk == "pulse" and sys.drives[a]["mode"] == i:
                    dr = sys.drives[a]
                    _, dE = sub_envelope(dr, n, t, dt)
                    dH = dE[b] * np.cos(sys.omega_d[a] * t + dr.get("phase", 0.0)) * sys.op(i, dr["op"])
                elif pk == "ham":
                    dEm, dops = derivs[(a, b)]
                    dH = np.zeros((sys.dims[i], sys.dims[i]), dtype=np.complex128)
                    if a == i:
                        dH += np.diag(dEm)
                    for k, dr in enumerate(sys.drives):
                        if dr["mode"] != i:
                            continue
                        E, _ = sub_envelope(dr, n, t, dt)
                        f = E * np.cos(sys.omega_d[k] * t + dr.get("phase", 0.0))
                        if a == i:
                            dH += f * sys.dop(dops, i, dr["op"])
                        if dr.get("omega_mode") == a:
                            df = -E * np.sin(sys.omega_d[k] * t + dr.get("phase", 0.0)) * t * dEm[1]
                            dH += df * sys.op(i, dr["op"])
                    if not np.any(dH):
                        dH = None
            else:
                cpl = sys.couplings[idx]
                A, B = sys.op(cpl["a"], cpl["op_a"]), sys.op(cpl["b"], cpl["op_b"])
                if pk == "J" and a == idx:
                    dH = np.kron(A, B)
                elif pk == "ham" and a in (cpl["a"], cpl["b"]):
                    dEm, dops = derivs[(a, b)]
                    if a == cpl["a"]:
                        dH = cpl["J"] * np.kron(sys.dop(dops, a, cpl["op_a"]), B)
                    else:
                        dH = cpl["J"] * np.kron(A, sys.dop(dops, a, cpl["op_b"]))
                    if not np.any(dH):
                        dH = None
            if dH is None:
                continue
            L = expm_frechet(G, scale * dH, compute_expm=False)
            if kind_f == "1":
                dpsi = _apply_1body(before, L, idx)
            else:
                aa, bb, _ = two[idx]
                dpsi = _apply_2body(before, L, aa, bb, sys.dims[aa], sys.dims[bb])
            grad[p] += np.real(np.vdot(bar, dpsi))
        X = expm(G)                                   # the co-state goes back through X^dag
        if kind_f == "1":
            bar = _apply_1body(bar, X.conj().T, idx)
        else:
            aa, bb, _ = two[idx]
            bar = _apply_2body(bar, X.conj().T, aa, bb, sys.dims[aa], sys.dims[bb])
    return F, grad
