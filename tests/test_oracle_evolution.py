"""Pins of the oracle's evolution, fidelity and gradient against closed forms,
brute force and independent derivatives."""
import copy

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from oracle.evolve import (initial_columns, rk4_evolve, rk4_evolve_matrix_free,
                           frame_epilogue, fidelities, fidelity_and_costate,
                           adjoint_gradient, tangent_linear_derivative,
                           finite_difference_gradient)
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W

GHZ = 2 * np.pi


def _flux(el=1.0, levels=4):
    return {"kind": "fluxonium", "ej": 4.0 * GHZ, "ec": 1.0 * GHZ, "el": el * GHZ,
            "phi_ext": np.pi, "n_osc": 50, "levels": levels}


def _wl(modes, couplings=(), drives=(), T=1.0, dt=0.01, frame="interaction", cols=None):
    dims = [m["levels"] for m in modes]
    D = int(np.prod(dims))
    nq = len(modes)
    return {"name": "t", "modes": list(modes), "couplings": list(couplings),
            "drives": list(drives), "T": T, "dt": dt, "frame": frame,
            "col_index": list(range(D)) if cols is None else cols,
            "target": np.eye(2 ** nq, dtype=complex), "fid_kind": "avg"}


def R4(z):
    """RK4 stability polynomial."""
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


def test_undriven_uncoupled_interaction_frame_is_exact_phase():
    wl = _wl([_flux(0.9, 3), _flux(1.1, 3)], T=5.0, dt=0.01)
    s = OracleSystem(wl)
    psi0 = initial_columns(s, wl["col_index"])
    psi_i = rk4_evolve(s, psi0)
    assert np.array_equal(psi_i, psi0)                  # H_I = 0 exactly
    psi = frame_epilogue(s, psi_i)
    E = s.hd_diag()
    assert np.allclose(psi, np.diag(np.exp(-1j * E * 5.0)), atol=1e-14)


def test_undriven_uncoupled_lab_frame_is_rk4_polynomial():
    wl = _wl([_flux(0.9, 3), _flux(1.1, 3)], T=2.0, dt=0.02, frame="lab")
    s = OracleSystem(wl)
    psi = rk4_evolve(s, initial_columns(s, wl["col_index"]))
    E = s.hd_diag()
    exact_rk4 = R4(-1j * E * s.dt) ** s.N
    assert np.allclose(np.diag(psi), exact_rk4, atol=1e-13)
    # and within the RK4 error bound of exp(-i E T)
    err = np.abs(np.diag(psi) - np.exp(-1j * E * 2.0))
    assert np.all(err <= s.N * np.abs(E * s.dt) ** 5 / 120 * 1.01 + 1e-14)


def test_rabi_two_level_constant_drive():
    # 2-level fluxonium, lab frame, constant envelope with omega_d = 0:
    # H = [[0, g], [g, Delta]] -> P1(t) = 4g^2/(4g^2+Delta^2) sin^2(sqrt(4g^2+Delta^2) t/2)
    a = 1.0
    wl = _wl([_flux(1.0, 2)], drives=[{"mode": 0, "op": "phi", "env": "pwc", "amps": [a],
                                       "length": 2.0, "omega_d": 0.0, "phase": 0.0}],
             T=2.0, dt=0.001, frame="lab", cols=[0])
    s = OracleSystem(wl)
    psi = rk4_evolve(s, initial_columns(s, [0]))
    g = a * abs(s.op(0, "phi")[0, 1])
    delta = s.modes[0]["E"][1]
    Om = np.sqrt(4 * g ** 2 + delta ** 2)
    p1 = 4 * g ** 2 / Om ** 2 * np.sin(Om * 2.0 / 2) ** 2
    assert abs(abs(psi[1, 0]) ** 2 - p1) < 1e-8
    # the interaction frame reaches the same lab-frame state
    wi = dict(wl, frame="interaction")
    si = OracleSystem(wi)
    psi_i = frame_epilogue(si, rk4_evolve(si, initial_columns(si, [0])))
    assert np.max(np.abs(psi_i - psi)) < 1e-8


def _pwc_lab_system(dt):
    drives = [{"mode": 0, "op": "phi", "env": "pwc", "amps": [0.3, -0.5, 0.8],
               "length": 1.2, "omega_d": 0.0, "phase": 0.0},
              {"mode": 1, "op": "n", "env": "pwc", "amps": [0.4, 0.1, -0.2],
               "length": 1.2, "omega_d": 0.0, "phase": 0.0}]
    cpl = [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": 0.2}]
    return _wl([_flux(0.9, 2), _flux(1.1, 2)], cpl, drives, T=1.2, dt=dt, frame="lab")


def test_piecewise_constant_matches_brute_force_expm_and_converges_4th_order():
    errs = []
    for dt in (0.02, 0.01, 0.005):
        wl = _pwc_lab_system(dt)
        s = OracleSystem(wl)
        psi = rk4_evolve(s, initial_columns(s, wl["col_index"]))
        # brute force: U = prod over segments of V exp(-i L tau) V^dag (eigh per segment)
        U = np.eye(s.D, dtype=complex)
        for seg in range(3):
            n_mid = int(round((seg + 0.5) * 0.4 / dt - 0.5))
            H = s.hamiltonian(n_mid, 1)
            lam, V = np.linalg.eigh(H)
            U = (V * np.exp(-1j * lam * 0.4)) @ V.conj().T @ U
        errs.append(np.max(np.abs(psi - U)))
    assert errs[-1] < 3e-7
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20


def test_dense_and_matrix_free_agree():
    wl = W.fluxonium_chain(seed=3, nq=3, levels=3, T=0.5, dt=0.01, ring=True)
    s = OracleSystem(wl)
    psi0 = initial_columns(s, wl["col_index"])
    a = rk4_evolve(s, psi0)
    b = rk4_evolve_matrix_free(s, psi0)
    assert np.max(np.abs(a - b)) < 1e-13
    # a single application, every stage kind, against the explicit Kronecker matrix
    y = W.random_columns(s.D, 3, seed=1)
    for j in (0, 1, 2):
        assert np.max(np.abs(s.hamiltonian(4, j) @ y - s.apply_matrix_free(4, j, y))) < 1e-12


def test_matrix_free_term_by_term_against_explicit_kron():
    # (A (x) B) acting on modes 0 and 2 of a 3-mode tensor, written with np.kron
    wl = W.fluxonium_chain(seed=5, nq=3, levels=3, T=0.1, dt=0.01)
    wl["drives"] = []
    wl["couplings"] = [{"a": 0, "op_a": "n", "b": 2, "op_b": "phi", "J": 0.7}]
    s = OracleSystem(wl)
    A = s.frame_op(s.op(0, "n"), 0, 0.05)
    B = s.frame_op(s.op(2, "phi"), 2, 0.05)
    full = 0.7 * np.kron(np.kron(A, np.eye(3)), B)
    y = W.random_columns(s.D, 2, seed=2)
    assert np.max(np.abs(full @ y - s.apply_matrix_free(5, 0, y))) < 1e-12   # t = 0.05


def test_norm_and_unitarity_within_rk4_bound():
    wl = W.transmon_pair(seed=1, T=5.0)
    s = OracleSystem(wl)
    psi = rk4_evolve(s, initial_columns(s, wl["col_index"]))
    U = frame_epilogue(s, psi)
    dev = np.max(np.abs(U.conj().T @ U - np.eye(16)))
    assert dev < 1e-6
    assert np.max(np.abs(np.linalg.norm(psi, axis=0) - 1)) < 1e-6


def test_fidelity_formula_against_nielsen_operator_basis():
    # Eq. D2 evaluated by brute force with the Weyl operator basis for a unitary
    # channel E(X) = M X M^dag, compared with the closed form used by the oracle.
    rng = np.random.default_rng(7)
    D = 4
    M = W.haar_unitary(D, rng)
    w = np.exp(2j * np.pi / D)
    X = np.roll(np.eye(D), 1, axis=0)
    Z = np.diag(w ** np.arange(D))
    basis = [np.linalg.matrix_power(X, a) @ np.linalg.matrix_power(Z, b)
             for a in range(D) for b in range(D)]
    num = sum(np.trace(Uj.conj().T @ M @ Uj @ M.conj().T) for Uj in basis) + D ** 2
    nielsen = np.real(num) / (D ** 2 * (D + 1))
    closed = (np.real(np.trace(M @ M.conj().T)) + abs(np.trace(M)) ** 2) / (D * (D + 1))
    assert abs(nielsen - closed) < 1e-13


def test_fidelity_identities():
    wl = W.transmon_pair(seed=2, T=1.0)
    s = OracleSystem(wl)
    psi = frame_epilogue(s, rk4_evolve(s, initial_columns(s, wl["col_index"])))
    Fa, Fs, Uc = fidelities(s, psi)
    # global phase of the target does not matter
    w2 = copy.deepcopy(wl)
    w2["target"] = wl["target"] * np.exp(0.37j)
    Fa2, Fs2, _ = fidelities(OracleSystem(w2), psi)
    assert abs(Fa - Fa2) < 1e-14 and abs(Fs - Fs2) < 1e-14
    # target = the unitary polar factor of the comp block: F_avg is then fixed by
    # the singular values alone, (sum s^2 + (sum s)^2) / (Dc (Dc + 1))
    cols = [0, 1, 4, 5]
    U = Uc[:, cols]
    u, sv, vh = np.linalg.svd(U)
    w3 = copy.deepcopy(wl)
    w3["target"] = u @ vh
    Fa3, Fs3, _ = fidelities(OracleSystem(w3), psi)
    assert abs(Fa3 - (np.sum(sv ** 2) + np.sum(sv) ** 2) / 20.0) < 1e-13
    assert abs(Fs3 - (np.sum(sv) / 4) ** 2) < 1e-13
    # F_state with S = Dc equals |tr M / Dc|^2
    M = wl["target"].conj().T @ U
    assert abs(Fs - abs(np.trace(M) / 4) ** 2) < 1e-14


def test_costate_matches_finite_differences_of_fidelity():
    wl = W.fluxonium_pair_cr(seed=1, T=0.5)
    s = OracleSystem(wl)
    psi = frame_epilogue(s, rk4_evolve(s, initial_columns(s, wl["col_index"])))
    rng = np.random.default_rng(3)
    for kind in ("avg", "state"):
        F, bar = fidelity_and_costate(s, psi, kind)
        dpsi = rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape)
        h = 1e-6
        Fp, _ = fidelity_and_costate(s, psi + h * dpsi, kind)
        Fm, _ = fidelity_and_costate(s, psi - h * dpsi, kind)
        assert abs((Fp - Fm) / (2 * h) - np.real(np.vdot(bar, dpsi))) < 1e-8


@pytest.mark.parametrize("frame", ["interaction", "lab"])
def test_adjoint_matches_tangent_linear_and_finite_differences(frame):
    wl = W.fluxonium_pair_cr(seed=4, T=0.4)
    wl["frame"] = frame
    wl["drives"].append({"mode": 1, "op": "n", "env": "gaussian", "amp": 0.2,
                         "sigma": 0.1, "t0": 0.2, "length": 0.4, "omega_mode": 0,
                         "phase": 0.3})
    F, g, prms = adjoint_gradient(wl)
    idx = [0, 7, 19, 20, 21, 22, 23, 24, 25, 26, 27]
    fd = finite_difference_gradient(wl, idx)
    for k, p in enumerate(idx):
        tl = tangent_linear_derivative(wl, p)
        scale = max(abs(g[p]), 1e-8)
        assert abs(g[p] - tl) <= 1e-11 * max(scale, np.max(np.abs(g)))
        assert abs(g[p] - fd[k]) <= 1e-5 * max(scale, 1e-6), (prms[p], g[p], fd[k])


def test_adjoint_state_fidelity_on_chain():
    wl = W.fluxonium_chain(seed=2, nq=3, levels=3, T=0.3, dt=0.01, nseg=3)
    F, g, prms = adjoint_gradient(wl)
    idx = [0, 4, 9, 10, 11, 12, 18, 19]
    fd = finite_difference_gradient(wl, idx)
    for k, p in enumerate(idx):
        assert abs(g[p] - fd[k]) <= 1e-5 * max(abs(g[p]), 1e-7), (prms[p], g[p], fd[k])


def test_decoupled_coupler_mode_leaves_fidelity_and_gradient_unchanged():
    # A coupler mode that nothing couples to or drives stays in its ground state:
    # the fidelity over the qubit modes and every shared gradient component equal
    # those of the same qubits without it (checks the coupler's place in the
    # computational map, the labels and the padded parameter vector).
    import copy
    from oracle.evolve import evolve_and_fidelity, adjoint_gradient
    wl2 = W.fluxonium_pair_multipath(seed=3, T=0.3, dt=0.01, nseg=3, levels=3)
    wl3 = copy.deepcopy(wl2)
    coupler = {"kind": "transmon", "ej": 20.0 * GHZ, "ec": 0.25 * GHZ, "ng": 0.0, "ncut": 10,
               "levels": 3, "coupler": True}
    wl3["modes"] = [wl2["modes"][0], coupler, wl2["modes"][1]]
    remap = {0: 0, 1: 2}
    for c in wl3["couplings"]:
        c["a"], c["b"] = remap[c["a"]], remap[c["b"]]
    for d in wl3["drives"]:
        d["mode"], d["omega_mode"] = remap[d["mode"]], remap[d["omega_mode"]]
    wl3["col_index"] = W.comp_states([3, 3, 3], couplers=(1,))
    r2, r3 = evolve_and_fidelity(wl2), evolve_and_fidelity(wl3)
    assert abs(r2["F_avg"] - r3["F_avg"]) < 1e-12 and abs(r2["F_state"] - r3["F_state"]) < 1e-12
    assert np.max(np.abs(r2["Uc"] - r3["Uc"])) < 1e-12
    F2, g2, p2 = adjoint_gradient(wl2)
    F3, g3, p3 = adjoint_gradient(wl3)
    assert abs(F2 - F3) < 1e-12
    g3d = {p: v for p, v in zip(p3, g3)}
    # pulse amplitudes and couplings keep their index; mode parameters follow the remap
    for p, v in zip(p2, g2):
        q = ("ham", remap[p[1]], p[2]) if p[0] == "ham" else p
        assert abs(g3d[q] - v) <= 1e-10 * max(1.0, abs(v)), p
    # nothing couples to or drives the coupler, so its own parameters have no effect
    assert all(abs(g3d[("ham", 1, x)]) < 1e-12 for x in ("ej", "ec", "el"))


def test_local_operator_equal_to_n_reproduces_the_builtin_term():
    # A local operator given as the mode's own truncated n must drive the same
    # evolution as "n": same F and the same pulse and coupling gradients.  Only the
    # device-parameter gradients differ (a local operator's matrix elements are
    # fixed, the builtin n moves with the eigenbasis).
    import copy
    from oracle.evolve import evolve_and_fidelity, adjoint_gradient
    from oracle.subsystems import build_mode
    wl = W.fluxonium_pair_multipath(seed=9, T=0.3, dt=0.01, nseg=3, levels=3)
    wl2 = copy.deepcopy(wl)
    for i, m in enumerate(wl2["modes"]):
        spec = {k: v for k, v in m.items() if k != "local_ops"}
        m["local_ops"] = {"nn": build_mode(spec)["ops"]["n"]}
    wl2["couplings"][0]["op_a"] = wl2["couplings"][0]["op_b"] = "nn"
    r1, r2 = evolve_and_fidelity(wl), evolve_and_fidelity(wl2)
    assert abs(r1["F_avg"] - r2["F_avg"]) < 1e-13
    F1, g1, p1 = adjoint_gradient(wl)
    F2, g2, p2 = adjoint_gradient(wl2)
    assert p1 == p2 and abs(F1 - F2) < 1e-13
    for p, a, b in zip(p1, g1, g2):
        if p[0] != "ham":
            assert abs(a - b) <= 1e-11 * max(1.0, abs(a)), p
    assert any(abs(a - b) > 1e-9 for p, a, b in zip(p1, g1, g2) if p[0] == "ham")
