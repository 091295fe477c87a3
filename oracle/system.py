"""Composite system: local operators, pulses and the Kronecker-sum Hamiltonian
(oracle; test infrastructure).

Eq. 1: H(t) = sum_i H_i(t) + sum_{e in G} H_ij, each term acting non-trivially
on one or two subsystems.  Here

    H_lab(t) = H_d + sum_k f_k(t) O_k + sum_e J_e A_e (x) B_e,
    H_d      = sum_i diag(E^(i))                   (ground-shifted levels, R1)

and the default frame is the interaction picture of H_d (reading R1):

    H_I(t) = sum_k f_k(t) O_k(t) + sum_e J_e A_e(t) (x) B_e(t),
    X(t)_ab = X_ab exp(i (E_a - E_b) t).

Drive coefficient (Eq. C1): f(t) = E(t) cos(omega_d t + phase), with the
envelopes of reading R8 (Gaussian, piecewise-constant, and the cosine
envelope of Eq. C2).  RK4 stage j in {0, 1, 2} of step n sits at the half step
t = (2n + j) dt / 2 (stages 2 and 3 of RK4 share j = 1).  A piecewise-constant
envelope takes the segment that holds the step's midpoint, so a step never
straddles a jump and RK4 keeps its order (reading R8).
"""
import numpy as np

from .subsystems import build_mode, mode_derivatives, PARAMS


def half_step_time(m, dt):
    return m * dt * 0.5


def stage_time(n, j, dt):
    return half_step_time(2 * n + j, dt)


def pulse_half_steps(length, dt):
    """Number of half steps that the pulse covers; must be an integer (R2, R8)."""
    x = 2.0 * length / dt
    mp = int(round(x))
    if abs(x - mp) > 1e-9 * max(1.0, x):
        raise ValueError("pulse length is not a whole number of half steps")
    return mp


def envelope(drive, n, j, dt):
    """E(t) at stage j of step n, and dE/dparams (list, one per pulse parameter)."""
    env = drive["env"]
    m = 2 * n + j
    t = half_step_time(m, dt)
    mp = pulse_half_steps(drive["length"], dt)
    if env == "gaussian":
        g = np.exp(-((t - drive["t0"]) ** 2) / (2.0 * drive["sigma"] ** 2))
        return drive["amp"] * g, [g]
    if env == "cosine":
        if m > mp:
            return 0.0, [0.0]
        c = 0.5 * (1.0 - np.cos(2.0 * np.pi * t / drive["length"]))
        return drive["amp"] * c, [c]
    if env == "pwc":
        amps = drive["amps"]
        nseg = len(amps)
        grads = [0.0] * nseg
        mid = 2 * n + 1                      # the step's midpoint half step
        if mid >= mp:
            return 0.0, grads
        seg = min((mid * nseg) // mp, nseg - 1)
        grads[seg] = 1.0
        return amps[seg], grads
    raise ValueError(env)


def n_pulse_params(drive):
    return len(drive["amps"]) if drive["env"] == "pwc" else 1


class OracleSystem:
    """Modes, couplings and drives of one workload dict (see workloads)."""

    def __init__(self, wl):
        self.wl = wl
        self.modes = [build_mode(s) for s in wl["modes"]]
        self.dims = [m["d"] for m in self.modes]
        self.nq = len(self.modes)
        self.D = int(np.prod(self.dims))
        self.dt = float(wl["dt"])
        x = wl["T"] / wl["dt"]
        self.N = int(round(x))
        if abs(x - self.N) > 1e-9 * max(1.0, x):
            raise ValueError("T/dt is not an integer (R2)")
        self.frame = wl.get("frame", "interaction")
        self.couplings = wl["couplings"]
        self.drives = wl["drives"]
        self.omega_d = [self._omega(dr) for dr in self.drives]

    # ---- carrier frequency (R8) ------------------------------------------------
    def _omega(self, dr):
        if dr.get("omega_mode") is not None:
            return float(self.modes[dr["omega_mode"]]["E"][1])
        return float(dr["omega_d"])

    def coeff(self, k, n, j):
        """f_k at stage j of step n (Eq. C1)."""
        dr = self.drives[k]
        E, _ = envelope(dr, n, j, self.dt)
        t = stage_time(n, j, self.dt)
        return E * np.cos(self.omega_d[k] * t + dr.get("phase", 0.0))

    # ---- local operators ---------------------------------------------------------
    def op(self, mode, name):
        """n, phi, or a mode's user-given local operator (workload mode dict
        "local_ops": {name: d x d Hermitian matrix in the truncated eigenbasis})."""
        if name in self.modes[mode]["ops"]:
            return self.modes[mode]["ops"][name]
        return np.asarray(self.wl["modes"][mode]["local_ops"][name], dtype=np.complex128)

    def dop(self, dops, mode, name):
        """d(op)/dtheta: local operators have fixed matrix elements in the truncated
        eigenbasis, so they do not depend on the device parameters."""
        if name in dops:
            return dops[name]
        return np.zeros((self.dims[mode], self.dims[mode]), dtype=np.complex128)

    def phases(self, mode, t):
        return np.exp(1j * self.modes[mode]["E"] * t)

    def frame_op(self, X, mode, t):
        """X(t) = exp(i H_d t) X exp(-i H_d t) restricted to one mode (R1)."""
        if self.frame == "lab":
            return X
        p = self.phases(mode, t)
        return X * p[:, None] * np.conj(p)[None, :]

    def embed(self, factors):
        """Dense kron over all modes of {mode: d x d matrix}, identity elsewhere."""
        out = np.ones((1, 1), dtype=np.complex128)
        for i, d in enumerate(self.dims):
            out = np.kron(out, factors.get(i, np.eye(d)))
        return out

    def hamiltonian(self, n, j):
        """Dense D x D H_I(t) (interaction frame) or H_lab(t) (lab frame) at stage
        j of step n, built term by term from explicit Kronecker products (Eq. 1)."""
        t = stage_time(n, j, self.dt)
        H = np.zeros((self.D, self.D), dtype=np.complex128)
        if self.frame == "lab":
            for i, md in enumerate(self.modes):
                H += self.embed({i: np.diag(md["E"]).astype(np.complex128)})
        for k, dr in enumerate(self.drives):
            f = self.coeff(k, n, j)
            O = self.frame_op(self.op(dr["mode"], dr["op"]), dr["mode"], t)
            H += f * self.embed({dr["mode"]: O})
        for c in self.couplings:
            A = self.frame_op(self.op(c["a"], c["op_a"]), c["a"], t)
            B = self.frame_op(self.op(c["b"], c["op_b"]), c["b"], t)
            if c["a"] == c["b"]:
                raise ValueError("coupling needs two distinct modes")
            H += c["J"] * self.embed({c["a"]: A, c["b"]: B})
        return H

    def hd_diag(self):
        """Diagonal of H_d = sum_i diag(E^(i)) over the composite index."""
        out = np.zeros(1)
        for md in self.modes:
            out = (out[:, None] + md["E"][None, :]).reshape(-1)
        return out

    # ---- matrix-free application (App. B: contraction one mode at a time) -------
    def apply_matrix_free(self, n, j, y):
        """H(t) @ y at stage j of step n, y of shape (D, S), contracting each local
        operator into the state tensor of shape (d_0, ..., d_{N-1}, S) (App. B)."""
        t = stage_time(n, j, self.dt)
        S = y.shape[1]
        yt = y.reshape(self.dims + [S])
        out = np.zeros_like(yt)
        nq = self.nq
        letters = "abcdefghijklmnopqrstuvw"

        def contract(op, mode, ten):
            idx_in = list(letters[:nq]) + ["z"]
            idx_out = idx_in.copy()
            idx_out[mode] = "y"
            spec = "y" + idx_in[mode] + "," + "".join(idx_in) + "->" + "".join(idx_out)
            return np.einsum(spec, op, ten)

        if self.frame == "lab":
            out += (self.hd_diag().reshape(self.dims))[..., None] * yt
        for k, dr in enumerate(self.drives):
            O = self.frame_op(self.op(dr["mode"], dr["op"]), dr["mode"], t)
            out += self.coeff(k, n, j) * contract(O, dr["mode"], yt)
        for c in self.couplings:
            A = self.frame_op(self.op(c["a"], c["op_a"]), c["a"], t)
            B = self.frame_op(self.op(c["b"], c["op_b"]), c["b"], t)
            out += c["J"] * contract(A, c["a"], contract(B, c["b"], yt))
        return out.reshape(self.D, S)

    # ---- parameter derivatives of the dense Hamiltonian -----------------------
    def param_list(self):
        """Flat parameter list: pulse params (per drive, in order), then per mode
        (E_J, E_C, E_L), then per coupling J."""
        out = []
        for k, dr in enumerate(self.drives):
            for j in range(n_pulse_params(dr)):
                out.append(("pulse", k, j))
        for i in range(self.nq):
            for p in PARAMS:
                out.append(("ham", i, p))
        for e in range(len(self.couplings)):
            out.append(("J", e, None))
        return out

    def mode_derivs(self, i, p):
        if self.wl["modes"][i]["kind"] == "transmon" and p == "el":
            d = self.dims[i]
            return np.zeros(d), {n: np.zeros((d, d), complex) for n in self.modes[i]["ops"]}
        return mode_derivatives(self.modes[i], p)

    def dH(self, n, j, prm):
        """Dense dH/dtheta at stage j of step n for one parameter (exact, using the
        eigen-derivative formulas for device parameters)."""
        t = stage_time(n, j, self.dt)
        kind, a, b = prm
        D = self.D
        out = np.zeros((D, D), dtype=np.complex128)
        if kind == "pulse":
            dr = self.drives[a]
            _, g = envelope(dr, n, j, self.dt)
            c = np.cos(self.omega_d[a] * t + dr.get("phase", 0.0))
            O = self.frame_op(self.op(dr["mode"], dr["op"]), dr["mode"], t)
            return g[b] * c * self.embed({dr["mode"]: O})
        if kind == "J":
            c = self.couplings[a]
            A = self.frame_op(self.op(c["a"], c["op_a"]), c["a"], t)
            B = self.frame_op(self.op(c["b"], c["op_b"]), c["b"], t)
            return self.embed({c["a"]: A, c["b"]: B})
        # device parameter p of mode i
        i, p = a, b
        dE, dops = self.mode_derivs(i, p)

        def dframe(X, dX):
            # d/dtheta of X_ab exp(i(E_a - E_b)t)
            if self.frame == "lab":
                return dX
            ph = self.phases(i, t)
            P = ph[:, None] * np.conj(ph)[None, :]
            return (dX + X * 1j * t * (dE[:, None] - dE[None, :])) * P

        if self.frame == "lab":
            out += self.embed({i: np.diag(dE).astype(np.complex128)})
        for k, dr in enumerate(self.drives):
            f = self.coeff(k, n, j)
            if dr["mode"] == i:
                X = self.op(i, dr["op"])
                out += f * self.embed({i: dframe(X, self.dop(dops, i, dr["op"]))})
            if dr.get("omega_mode") == i:
                # carrier tied to this mode's 0-1 frequency (R8)
                E, _ = envelope(dr, n, j, self.dt)
                df = -E * np.sin(self.omega_d[k] * t + dr.get("phase", 0.0)) * t * dE[1]
                O = self.frame_op(self.op(dr["mode"], dr["op"]), dr["mode"], t)
                out += df * self.embed({dr["mode"]: O})
        for c in self.couplings:
            if c["a"] == i or c["b"] == i:
                A = self.frame_op(self.op(c["a"], c["op_a"]), c["a"], t)
                B = self.frame_op(self.op(c["b"], c["op_b"]), c["b"], t)
                if c["a"] == i:
                    A = dframe(self.op(i, c["op_a"]), self.dop(dops, i, c["op_a"]))
                    out += c["J"] * self.embed({c["a"]: A, c["b"]: B})
                else:
                    B = dframe(self.op(i, c["op_b"]), self.dop(dops, i, c["op_b"]))
                    out += c["J"] * self.embed({c["a"]: A, c["b"]: B})
        return out

    def dHd_diag(self, prm):
        """d/dtheta of the diagonal of H_d (non-zero only for device parameters)."""
        kind, i, p = prm
        if kind != "ham":
            return np.zeros(self.D)
        dE, _ = self.mode_derivs(i, p)
        out = np.zeros(1)
        for j, md in enumerate(self.modes):
            e = dE if j == i else np.zeros(md["d"])
            out = (out[:, None] + e[None, :]).reshape(-1)
        return out
