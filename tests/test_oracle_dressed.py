"""Pins of the oracle's dressed (idle-Hamiltonian eigen-) basis of the gate metric
(App. C): reduction to the product basis without couplings, eigen-residual, the
phase gauge, second-order perturbation theory for the leaked weight of a dressed
state, and the pulse gradient against central differences."""
import copy

import numpy as np

from oracle.dressed import (dressed_fidelities, dressed_pulse_gradient, dressed_vectors,
                            idle_hamiltonian)
from oracle.evolve import comp_map, evolve_and_fidelity
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W


def _pair(seed=3, T=0.5, J_scale=1.0):
    wl = W.fluxonium_pair_cr(seed=seed, nseg=4, T=T)
    wl["drives"][0]["length"] = T
    for c in wl["couplings"]:
        c["J"] *= J_scale
    return wl


def test_without_couplings_the_dressed_basis_is_the_product_basis():
    wl = _pair(J_scale=0.0)
    sys = OracleSystem(wl)
    Vc, _ = dressed_vectors(sys)
    comp, _ = comp_map(sys)
    E = np.zeros((sys.D, len(comp)))
    E[comp, range(len(comp))] = 1.0
    assert np.max(np.abs(Vc - E)) < 1e-12
    Fa, Fs, _ = dressed_fidelities(wl)
    r = evolve_and_fidelity(wl)
    assert abs(Fa - r["F_avg"]) < 1e-12 and abs(Fs - r["F_state"]) < 1e-12


def test_dressed_vectors_are_gauged_eigenvectors():
    wl = _pair()
    sys = OracleSystem(wl)
    Vc, lam = dressed_vectors(sys)
    H = idle_hamiltonian(sys)
    assert np.max(np.abs(H @ Vc - Vc * lam[None, :])) < 1e-10
    assert np.max(np.abs(Vc.conj().T @ Vc - np.eye(Vc.shape[1]))) < 1e-12
    comp, _ = comp_map(sys)
    diag = Vc[comp, range(len(comp))]
    assert np.all(np.abs(diag.imag) < 1e-15) and np.all(diag.real > 0.5)


def test_leaked_weight_follows_second_order_perturbation_theory():
    # weak coupling: 1 - |<bare_j|v_j>|^2 = sum_k |<k|V|bare_j>|^2 / (E_j - E_k)^2 + O(J^3)
    wl = _pair(J_scale=0.05)
    sys = OracleSystem(wl)
    Vc, _ = dressed_vectors(sys)
    comp, _ = comp_map(sys)
    H = idle_hamiltonian(sys)
    E0 = np.real(np.diag(H))
    Vcp = H - np.diag(np.diag(H))
    for j, r in enumerate(comp):
        leaked = 1.0 - abs(Vc[r, j]) ** 2
        pt = sum(abs(Vcp[k, r]) ** 2 / (E0[r] - E0[k]) ** 2 for k in range(sys.D) if k != r)
        assert abs(leaked - pt) <= 0.05 * pt + 1e-14, (j, leaked, pt)


def test_dressed_pulse_gradient_matches_central_differences():
    wl = _pair(T=0.4)
    F, g = dressed_pulse_gradient(wl)
    assert abs(F - dressed_fidelities(wl)[0 if wl["fid_kind"] == "avg" else 1]) < 1e-14
    k = 0 if wl["fid_kind"] == "avg" else 1
    fd = []
    for j in range(len(wl["drives"][0]["amps"])):
        vals = []
        h = 1e-7 * max(1.0, abs(wl["drives"][0]["amps"][j]))
        for sgn in (1, -1):
            w2 = copy.deepcopy(wl)
            w2["drives"][0]["amps"][j] += sgn * h
            vals.append(dressed_fidelities(w2)[k])
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    assert np.max(np.abs(g - fd)) <= 1e-6 * max(1e-6, np.max(np.abs(fd))), (g, fd)


def test_dressed_full_gradient_matches_central_differences_through_the_eigensolves():
    """The Hamiltonian-parameter gradient in the dressed basis (E_J, E_C, E_L per mode, J
    per coupling) against central differences of F through both eigensolves (each
    subsystem's and the idle Hamiltonian's).  The derivative of the dressed vectors is
    about 1 % of the gradient here, far above the tolerance, so dropping it (or a sign
    slip in it) fails."""
    from oracle.dressed import dressed_evolve, dressed_full_gradient
    from oracle.evolve import adjoint_from_costate, block_fidelity_and_costate, param_vector, set_param_vector
    wl = W.fluxonium_chain(seed=7, nq=3, levels=3, T=0.3, dt=0.01, nseg=2)
    theta = np.asarray(param_vector(wl), dtype=float)
    for kind in ("avg", "state"):
        F, g = dressed_full_gradient(wl, kind)
        _, gp = dressed_pulse_gradient(wl, kind)
        npul = len(gp)
        assert np.array_equal(g[:npul], gp)
        fd = []
        for i in range(npul, len(theta)):
            h = 1e-6 * max(1.0, abs(theta[i]))
            vals = []
            for sgn in (1, -1):
                t2 = theta.copy()
                t2[i] += sgn * h
                Fa, Fs, _ = dressed_fidelities(set_param_vector(wl, t2))
                vals.append(Fa if kind == "avg" else Fs)
            fd.append((vals[0] - vals[1]) / (2 * h))
        fd = np.array(fd)
        assert np.max(np.abs(g[npul:] - fd)) <= 1e-5 * np.max(np.abs(fd)), (kind, g[npul:], fd)
        if kind == "avg":
            sys_, Vc, cols, psi_lab, hist = dressed_evolve(wl)
            T = np.asarray(wl["target"], dtype=complex)
            _, barc = block_fidelity_and_costate(T, Vc.conj().T @ psi_lab, cols, kind)
            g_evo, _ = adjoint_from_costate(sys_, hist, psi_lab, Vc @ barc, sys_.N)
            assert np.max(np.abs(g_evo[npul:] - fd)) > 100 * 1e-5 * np.max(np.abs(fd))


def test_paper_multipath_chain_dressed_frequencies_and_zero_zz_coupling():
    # Sec. 3.1's 3-qubit multipath chain: the printed dressed 0-1 frequencies, and the
    # capacitive coupling at which the static ZZ rate of the left pair vanishes
    import json
    import os
    from scipy.optimize import brentq
    with open(os.path.join(os.path.dirname(__file__), "golden", "multipath_zz.json")) as f:
        g = json.load(f)
    GHZ, MHZ = W.GHZ, W.MHZ

    def chain(jc):
        modes = [dict(kind="fluxonium", ej=m["ej_GHz"] * GHZ, ec=m["ec_GHz"] * GHZ, el=m["el_GHz"] * GHZ,
                      phi_ext=np.pi, levels=5, n_osc=50) for m in g["modes"]]
        cpl = []
        for a, b in ((0, 1), (1, 2)):
            cpl.append({"a": a, "op_a": "n", "b": b, "op_b": "n", "J": jc})
            cpl.append({"a": a, "op_a": "phi", "b": b, "op_b": "phi", "J": -g["J_L_MHz"] * MHZ})
        return {"modes": modes, "couplings": cpl, "drives": [], "T": 1.0, "dt": 0.01, "frame": "lab",
                "col_index": list(range(8)), "target": np.eye(8), "fid_kind": "avg"}

    def levels(jc):
        _, lam = dressed_vectors(OracleSystem(chain(jc)))
        return lam                                  # labels |q1 q2 q3>, first qubit most significant

    lam = levels(g["J_C_spectrum_MHz"] * MHZ)
    f1, f2 = (lam[4] - lam[0]) / GHZ, (lam[2] - lam[0]) / GHZ
    assert abs(f1 - g["dressed_f01_GHz"][0]) < g["f01_tolerance_GHz"]
    assert abs(f2 - g["dressed_f01_GHz"][1]) < g["f01_tolerance_GHz"]

    def zz(jc):
        lam = levels(jc)
        return lam[0] + lam[6] - lam[4] - lam[2]

    root = brentq(zz, 5.0 * MHZ, 20.0 * MHZ, xtol=1e-9) / MHZ
    assert abs(root - g["zz_zero_J_C_MHz"]) < g["J_C_tolerance_MHz"], root
