"""Pins of the oracle's Suzuki-Trotter evolutions (Sec. 2.3, App. A) against what
the mathematics fixes: exactness when the local terms commute, the convergence
order of Q1 (1), Q2 (2), Q4 (4) and Q4j (3: see oracle/trotter.py), Q2 as the
symmetric composition of Q1 and its reverse, unitarity, and the pulse gradient
against central differences."""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle.evolve import initial_columns, rk4_evolve, frame_epilogue
from oracle.system import OracleSystem
from oracle.trotter import q2_evolve
from paper_2406_18155_gb300 import workloads as W

GHZ, MHZ = W.GHZ, W.MHZ


def _lab(wl, T, dt):
    wl = dict(wl, frame="lab", T=T, dt=dt)
    wl["drives"] = [dict(d, length=T) if d.get("env") != "gaussian" else
                    dict(d, length=T, sigma=T / 4, t0=T / 2) for d in wl["drives"]]
    return wl


def test_commuting_terms_are_exact():
    # two uncoupled driven modes: the 1-body factors commute, so Q2 is the exact
    # midpoint propagator exp(-i H(t_n + dt/2) dt) of the dense Kronecker sum
    wl = W.fluxonium_pair_multipath(seed=2, levels=3, nseg=4)
    wl["couplings"] = []
    wl = _lab(wl, 0.2, 0.01)
    sys = OracleSystem(wl)
    psi0 = initial_columns(sys, range(sys.D))
    got = q2_evolve(sys, psi0)
    U = np.eye(sys.D, dtype=complex)
    for n in range(sys.N):
        U = expm(-1j * sys.hamiltonian(n, 1) * sys.dt) @ U
    assert np.max(np.abs(got - U)) < 1e-12


def test_second_order_convergence():
    # coupled, driven pair with a smooth (Gaussian) drive: the Q2 error against a
    # fine RK4 reference falls 4x per halving of dt
    base = W.transmon_pair(seed=4)
    base["modes"] = [dict(m, levels=3) for m in base["modes"]]
    base["col_index"] = list(range(9))
    T = 1.0
    # reference: RK4 in the interaction frame (the level energies removed, so it is
    # converged at this step) and the exact frame phase back to the lab frame
    ref_wl = dict(_lab(base, T, 0.00125), frame="interaction")
    ref_sys = OracleSystem(ref_wl)
    ref = frame_epilogue(ref_sys, rk4_evolve(ref_sys, initial_columns(ref_sys, base["col_index"])))
    errs = []
    for dt in (0.02, 0.01, 0.005):
        s = OracleSystem(_lab(base, T, dt))
        errs.append(np.max(np.abs(q2_evolve(s, initial_columns(s, base["col_index"])) - ref)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def _converged_reference(base, T):
    # RK4 in the interaction frame at a fine step (the level energies removed, so it
    # is converged) and the exact frame phase back to the lab frame
    ref_wl = dict(_lab(base, T, 0.000625), frame="interaction")
    ref_sys = OracleSystem(ref_wl)
    return frame_epilogue(ref_sys, rk4_evolve(ref_sys, initial_columns(ref_sys, base["col_index"])))


def _errors(base, T, ref, scheme, dts):
    errs = []
    for dt in dts:
        s = OracleSystem(_lab(base, T, dt))
        errs.append(np.max(np.abs(q2_evolve(s, initial_columns(s, base["col_index"]), scheme=scheme) - ref)))
    return errs


def test_fourth_order_convergence_of_q4_and_third_of_q4j():
    # Gaussian-driven coupled pair: Q4's error falls 16x per halving of dt; the
    # complex Q4j's 8x (p + p* = 1 and p^3 + p*^3 = 0 cancel the dt^3 local term);
    # a wrong p, or the sub-step times off their midpoints, drops either to order 2
    # or below
    base = W.transmon_pair(seed=4)
    base["modes"] = [dict(m, levels=3) for m in base["modes"]]
    base["col_index"] = list(range(9))
    ref = _converged_reference(base, 1.0)
    e4 = _errors(base, 1.0, ref, "q4", (0.02, 0.01, 0.005))
    assert 14.0 < e4[0] / e4[1] < 17.0 and 14.0 < e4[1] / e4[2] < 17.0, e4
    e4j = _errors(base, 1.0, ref, "q4j", (0.02, 0.01, 0.005))
    assert 7.0 < e4j[0] / e4j[1] < 11.0 and 7.0 < e4j[1] / e4j[2] < 11.0, e4j
    e2 = _errors(base, 1.0, ref, "q2", (0.01,))
    assert e4[1] < e4j[1] < e2[0]


def test_unitary_to_round_off():
    wl = _lab(W.coupler_scheme(seed=5, kind="ftf", nseg=4, levels=(3, 3, 3)), 0.3, 0.01)
    sys = OracleSystem(wl)
    U = q2_evolve(sys, initial_columns(sys, range(sys.D)))
    assert np.max(np.abs(U.conj().T @ U - np.eye(sys.D))) < 1e-12
    U4 = q2_evolve(sys, initial_columns(sys, range(sys.D)), scheme="q4")
    assert np.max(np.abs(U4.conj().T @ U4 - np.eye(sys.D))) < 1e-12
    # Q4j's factors are not unitary (complex time steps); its product is, to its order
    U4j = q2_evolve(sys, initial_columns(sys, range(sys.D)), scheme="q4j")
    dev = np.max(np.abs(U4j.conj().T @ U4j - np.eye(sys.D)))
    assert 1e-12 < dev < 1e-4, dev


@pytest.mark.parametrize("scheme", ["q1", "q2", "q4", "q4j"])
def test_pulse_gradient_matches_central_differences(scheme):
    import copy
    from oracle.trotter import q2_pulse_gradient, q2_fidelity
    for wl in (W.fluxonium_pair_multipath(seed=11, levels=3, nseg=3),
               W.transmon_pair(seed=12)):
        wl = _lab(wl, 0.2, 0.01)
        if wl["modes"][0]["kind"] == "transmon":
            wl["modes"] = [dict(m, levels=3) for m in wl["modes"]]
            wl["col_index"] = W.comp_states([3, 3])
        F, g = q2_pulse_gradient(wl, scheme=scheme)
        assert abs(F - q2_fidelity(wl, scheme=scheme)) < 1e-14
        fd = []
        for k, dr in enumerate(wl["drives"]):
            keys = [("amps", j) for j in range(len(dr["amps"]))] if dr["env"] == "pwc" else [("amp", None)]
            for key, j in keys:
                vals = []
                for sgn in (1, -1):
                    w2 = copy.deepcopy(wl)
                    h = 1e-5 * max(1.0, abs(dr[key][j] if j is not None else dr[key]))
                    if j is None:
                        w2["drives"][k][key] += sgn * h
                    else:
                        w2["drives"][k][key][j] += sgn * h
                    vals.append(q2_fidelity(w2, scheme=scheme))
                fd.append((vals[0] - vals[1]) / (2 * h))
        fd = np.array(fd)
        assert np.max(np.abs(g - fd)) <= 1e-6 * max(1e-3, np.max(np.abs(fd))), (g, fd)


@pytest.mark.parametrize("scheme", ["q2", "q4"])
def test_full_gradient_matches_central_differences_through_the_eigensolve(scheme):
    # every parameter: pulse segments, E_J / E_C / E_L of each mode (through the
    # subsystem eigendecomposition) and the coupling J
    from oracle.evolve import param_vector, set_param_vector
    from oracle.system import OracleSystem
    from oracle.trotter import trotter_full_gradient, q2_fidelity, q2_pulse_gradient
    wl = _lab(W.fluxonium_pair_multipath(seed=11, levels=3, nseg=2), 0.1, 0.01)
    F, g = trotter_full_gradient(wl, scheme=scheme)
    Fp, gp = q2_pulse_gradient(wl, scheme=scheme)
    assert abs(F - Fp) < 1e-14 and np.max(np.abs(g[:len(gp)] - gp)) < 1e-12
    theta = param_vector(wl)
    prms = OracleSystem(wl).param_list()
    for p, prm in enumerate(prms):
        h = 1e-7 if prm[0] == "pulse" else 1e-5 * max(abs(theta[p]), 1e-3)
        vals = []
        for sgn in (1, -1):
            th = theta.copy()
            th[p] += sgn * h
            vals.append(q2_fidelity(set_param_vector(wl, th), scheme=scheme))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g[p] - fd) <= 1e-6 * max(1e-4, np.max(np.abs(g))), (prm, g[p], fd)


def test_q1_exact_for_commuting_terms_and_first_order():
    # uncoupled driven modes: Q1's factors commute, so a step is the exact midpoint
    # propagator; coupled and Gaussian-driven: the error halves with dt (ratio 2)
    wl = W.fluxonium_pair_multipath(seed=2, levels=3, nseg=4)
    wl["couplings"] = []
    wl = _lab(wl, 0.2, 0.01)
    sys = OracleSystem(wl)
    got = q2_evolve(sys, initial_columns(sys, range(sys.D)), scheme="q1")
    U = np.eye(sys.D, dtype=complex)
    for n in range(sys.N):
        U = expm(-1j * sys.hamiltonian(n, 1) * sys.dt) @ U
    assert np.max(np.abs(got - U)) < 1e-12
    base = W.transmon_pair(seed=4)
    base["modes"] = [dict(m, levels=3) for m in base["modes"]]
    base["col_index"] = list(range(9))
    ref = _converged_reference(base, 1.0)
    e1 = _errors(base, 1.0, ref, "q1", (0.01, 0.005, 0.0025))
    assert 1.8 < e1[0] / e1[1] < 2.2 and 1.8 < e1[1] / e1[2] < 2.2, e1
    e2 = _errors(base, 1.0, ref, "q2", (0.01,))
    assert e2[0] < e1[0]


def test_q2_is_q1_then_its_reverse_at_half_steps():
    # with time-independent terms, Q2(dt) = Q1rev(dt/2) Q1(dt/2): Q1 over half a step,
    # then the same factors in reverse order (App. A's symmetric composition)
    wl = W.fluxonium_pair_multipath(seed=3, levels=3, nseg=4)
    wl["drives"] = []
    wl = _lab(wl, 0.02, 0.01)
    sys = OracleSystem(wl)
    psi0 = initial_columns(sys, range(sys.D))
    q2 = q2_evolve(sys, psi0, nsteps=1, scheme="q2")
    half = OracleSystem(dict(wl, dt=0.005, T=0.005))
    psi = q2_evolve(half, psi0, nsteps=1, scheme="q1").reshape(list(sys.dims) + [sys.D])
    from oracle.trotter import local_terms, _apply_1body, _apply_2body
    one, two = local_terms(half, 0)
    for a, b, M in reversed(two):
        psi = _apply_2body(psi, expm(-1j * M * 0.005), a, b, sys.dims[a], sys.dims[b])
    for i in reversed(range(sys.nq)):
        psi = _apply_1body(psi, expm(-1j * one[i] * 0.005), i)
    assert np.max(np.abs(psi.reshape(sys.D, sys.D) - q2)) < 1e-12
