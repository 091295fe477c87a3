"""Subsystem Hamiltonians, diagonalisation, truncation (oracle; test infrastructure).

All energies are angular, in rad/ns (the paper quotes them as 2*pi*GHz, Sec. 3.1).

Transmon (charge basis, reading R3):
    H = 4 E_C (n - n_g)^2 - E_J cos(phi),  n in [-ncut, ncut],
    cos(phi) = (|n><n+1| + |n+1><n|) / 2,   charge operator  n - n_g.

Fluxonium (oscillator basis, Eq. 8 shifted so that the external flux sits in
the cosine, reading R5):
    H = 4 E_C n^2 + E_L phi^2 / 2 - E_J cos(phi - phi_ext)
      = omega_p (a^dag a + 1/2) - E_J cos(phi - phi_ext),
    phi_osc = (8 E_C / E_L)^(1/4),  omega_p = sqrt(8 E_C E_L),
    phi = phi_osc X,  n = P / phi_osc,  X = (a + a^dag)/sqrt2,  P = i(a^dag - a)/sqrt2,
    cos(phi - phi_ext) = W diag(cos(phi_osc x_j - phi_ext)) W^T  with X = W diag(x) W^T.

Every builder also returns dH/dtheta and dOp/dtheta for theta in (E_J, E_C, E_L),
which the gradient chain uses.
"""
import numpy as np

PARAMS = ("ej", "ec", "el")


def transmon(ej, ec, ng=0.0, ncut=10):
    """Charge-basis transmon (Sec. 2.1 names E_J, E_C; matrix form is reading R3)."""
    n = np.arange(-ncut, ncut + 1, dtype=np.float64)
    m = n.size
    hop = np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)
    cosphi = 0.5 * hop
    h = np.diag(4.0 * ec * (n - ng) ** 2) - ej * cosphi
    ops = {"n": np.diag(n - ng).astype(np.complex128)}
    dh = {"ej": -cosphi, "ec": np.diag(4.0 * (n - ng) ** 2), "el": np.zeros((m, m))}
    zero = np.zeros((m, m), dtype=np.complex128)
    dops = {"n": {"ej": zero, "ec": zero, "el": zero}}
    return h, ops, dh, dops


def fluxonium(ej, ec, el, phi_ext=np.pi, n_osc=50):
    """Oscillator-basis fluxonium (Eq. 8; basis and cosine construction: reading R5)."""
    k = np.arange(n_osc, dtype=np.float64)
    a = np.diag(np.sqrt(k[1:]), 1)                  # a|k> = sqrt(k)|k-1>
    X = (a + a.T) / np.sqrt(2.0)
    P = 1j * (a.T - a) / np.sqrt(2.0)
    x, W = np.linalg.eigh(X)                        # Gauss-Hermite nodes
    phi_osc = (8.0 * ec / el) ** 0.25
    omega_p = np.sqrt(8.0 * ec * el)
    arg = phi_osc * x - phi_ext
    cos_m = (W * np.cos(arg)) @ W.T
    h = np.diag(omega_p * (k + 0.5)) - ej * cos_m
    ops = {"phi": (phi_osc * X).astype(np.complex128), "n": P / phi_osc}
    # derivatives of phi_osc and omega_p
    dpo = {"ej": 0.0, "ec": phi_osc / (4.0 * ec), "el": -phi_osc / (4.0 * el)}
    dwp = {"ej": 0.0, "ec": omega_p / (2.0 * ec), "el": omega_p / (2.0 * el)}
    sin_x = (W * (np.sin(arg) * x)) @ W.T           # d/dphi_osc of cos(phi_osc x - phi_ext) is -sin * x
    dh = {}
    for p in PARAMS:
        d = np.diag(dwp[p] * (k + 0.5)) + ej * dpo[p] * sin_x
        if p == "ej":
            d = d - cos_m
        dh[p] = d
    dops = {"phi": {p: (dpo[p] * X).astype(np.complex128) for p in PARAMS},
            "n": {p: -P * dpo[p] / phi_osc ** 2 for p in PARAMS}}
    return h, ops, dh, dops


def gauge_fix(v):
    """Reading R6: flip each eigenvector so that its first component with
    |v_i| >= 1e-3 max|v| is positive."""
    v = v.copy()
    for j in range(v.shape[1]):
        col = v[:, j]
        thr = 1e-3 * np.max(np.abs(col))
        i = int(np.nonzero(np.abs(col) >= thr)[0][0])
        if col[i] < 0:
            v[:, j] = -col
    return v


def diagonalise(h):
    """Full eigendecomposition of a real symmetric subsystem Hamiltonian, ascending,
    gauge-fixed (R6)."""
    w, v = np.linalg.eigh(h)
    return w, gauge_fix(v)


def build_mode(spec):
    """Build one truncated mode from a spec dict (see workloads): returns a dict with
    d, energies E (ground-shifted, length d), truncated operators (d x d complex),
    and the pieces the gradient chain needs (full eigensystem, dH, dops)."""
    kind = spec["kind"]
    if kind == "transmon":
        h, ops, dh, dops = transmon(spec["ej"], spec["ec"], spec.get("ng", 0.0),
                                    spec.get("ncut", 10))
    elif kind == "fluxonium":
        h, ops, dh, dops = fluxonium(spec["ej"], spec["ec"], spec["el"],
                                     spec.get("phi_ext", np.pi), spec.get("n_osc", 50))
    else:
        raise ValueError(kind)
    d = int(spec["levels"])
    w, v = diagonalise(h)
    vd = v[:, :d]
    E = w[:d] - w[0]
    tops = {name: vd.T @ op @ vd for name, op in ops.items()}
    return {"kind": kind, "d": d, "E": E, "ops": tops, "w": w, "v": v, "h": h,
            "full_ops": ops, "dh": dh, "dops": dops}


def mode_derivatives(mode, param):
    """Forward-mode derivative of the truncated energies and operators w.r.t. one
    device parameter, by the standard first-order perturbation formulas
    (Hellmann-Feynman for eigenvalues; sum over all other eigenvectors for the
    eigenvector derivative; non-degenerate spectrum assumed)."""
    w, v, d = mode["w"], mode["v"], mode["d"]
    dh = mode["dh"][param]
    hv = v.T @ dh @ v                                  # dH in the eigenbasis
    dw = np.diag(hv).copy()
    M = w.size
    dv = np.zeros((M, d))
    for a in range(d):
        for c in range(M):
            if c != a:
                dv[:, a] += v[:, c] * hv[c, a] / (w[a] - w[c])
    dE = dw[:d] - dw[0]
    vd = v[:, :d]
    dops = {}
    for name, op in mode["full_ops"].items():
        dop = mode["dops"][name][param]
        dops[name] = dv.T @ op @ vd + vd.T @ op @ dv + vd.T @ dop @ vd
    return dE, dops


def mathieu_transmon_levels(ej, ec, nlev):
    """Exact n_g = 0 transmon levels from Mathieu characteristic values
    (E = E_C * {a_0, b_2, a_2, b_4, ...}(q = -E_J / 2E_C)); used only as a pin."""
    from scipy.special import mathieu_a, mathieu_b
    q = -ej / (2.0 * ec)
    out = []
    for k in range(nlev):
        if k % 2 == 0:
            out.append(ec * mathieu_a(k, q))
        else:
            out.append(ec * mathieu_b(k + 1, q))
    return np.array(out)
