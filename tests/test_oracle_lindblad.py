"""Pins of the oracle's vectorised Lindblad evolution: closed forms for amplitude
damping and pure dephasing of one two-level mode, exact trace and Hermiticity
preservation by RK4 of a trace-preserving generator, and the closed-system limit
(no collapse operators) against the pure-state evolution."""
import numpy as np

from oracle.evolve import initial_columns, rk4_evolve, frame_epilogue
from oracle.lindblad import evolve_density, liouvillian
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W


def _two_level(collapse, T=2.0, dt=0.002, frame="lab"):
    # one transmon truncated to 2 levels, no drives and no couplings
    wl = W.transmon_pair(seed=1, T=T, dt=dt)
    wl["modes"] = [dict(wl["modes"][0], levels=2)]
    wl["drives"], wl["couplings"] = [], []
    wl["col_index"] = [0, 1]
    wl["frame"] = frame
    wl["collapse"] = collapse
    return wl


def test_amplitude_damping_closed_form():
    # rho_11 = rho_11(0) e^{-g T}, rho_01 = rho_01(0) e^{-g T / 2} e^{i E T}: exact to
    # rounding in the interaction frame (the generator is then constant and slow), within
    # RK4's phase error N |E dt|^5 / 120 in the lab frame
    g = 0.7
    for frame in ("interaction", "lab"):
        wl = _two_level([{"mode": 0, "L": [[0, 1], [0, 0]], "rate": g}], frame=frame)
        sys = OracleSystem(wl)
        E = sys.modes[0]["E"][1] - sys.modes[0]["E"][0]
        rho0 = 0.5 * np.array([[1, 1], [1, 1]], dtype=complex)          # |+><+|
        rho = evolve_density(wl, rho0)
        T = wl["T"]
        tol = 1e-12 if frame == "interaction" else sys.N * abs(E * sys.dt) ** 5 / 120
        assert abs(rho[1, 1] - 0.5 * np.exp(-g * T)) < 1e-12
        assert abs(rho[0, 1] - 0.5 * np.exp(-g * T / 2) * np.exp(1j * E * T)) < tol


def test_pure_dephasing_closed_form():
    g = 0.9
    wl = _two_level([{"mode": 0, "L": [[0, 0], [0, 1]], "rate": g}], frame="interaction")
    sys = OracleSystem(wl)
    E = sys.modes[0]["E"][1] - sys.modes[0]["E"][0]
    rho0 = 0.5 * np.array([[1, 1], [1, 1]], dtype=complex)
    rho = evolve_density(wl, rho0)
    T = wl["T"]
    assert abs(rho[1, 1] - 0.5) < 1e-12
    assert abs(rho[0, 1] - 0.5 * np.exp(-g * T / 2) * np.exp(1j * E * T)) < 1e-12


def test_trace_and_hermiticity_are_preserved():
    wl = W.fluxonium_pair_cr(seed=2, nseg=3, T=0.3)
    wl["drives"][0]["length"] = 0.3
    d = wl["modes"][0]["levels"]
    low = np.diag(np.sqrt(np.arange(1, d)), 1)
    wl["collapse"] = [{"mode": 0, "L": low, "rate": 0.05}, {"mode": 1, "L": np.diag(np.arange(d)), "rate": 0.02}]
    sys = OracleSystem(wl)
    # the generator is trace preserving: the identity's row-vector annihilates it
    Lv = liouvillian(sys, 3, 1)
    assert np.max(np.abs(np.eye(sys.D).reshape(-1) @ Lv)) < 1e-10
    rng = np.random.default_rng(0)
    X = rng.normal(size=(sys.D, sys.D)) + 1j * rng.normal(size=(sys.D, sys.D))
    rho0 = X @ X.conj().T
    rho0 /= np.trace(rho0)
    rho = evolve_density(wl, rho0)
    assert abs(np.trace(rho) - 1.0) < 1e-12
    assert np.max(np.abs(rho - rho.conj().T)) < 1e-12
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-10


def test_without_collapse_the_density_matrix_follows_the_pure_states():
    wl = W.fluxonium_pair_cr(seed=4, nseg=3, T=0.2)
    wl["drives"][0]["length"] = 0.2
    sys = OracleSystem(wl)
    psi = frame_epilogue(sys, rk4_evolve(sys, initial_columns(sys, [1])))
    rho0 = np.zeros((sys.D, sys.D), dtype=complex)
    rho0[1, 1] = 1.0
    rho = evolve_density(wl, rho0)
    # RK4 of the superoperator and U rho U^dag with RK4's U agree to the RK4 error
    assert np.max(np.abs(rho - psi @ psi.conj().T)) < 1e-8


def test_gate_fidelity_of_amplitude_damping_closed_form():
    # the idle qubit under amplitude damping against the ideal idle gate diag(1, e^{-iET}):
    # Kraus operators diag(1, sqrt(1-p)) and sqrt(p)|0><1|, p = 1 - e^{-g T}, so
    # F_avg = (|1 + sqrt(1-p)|^2 + 2) / 6
    from oracle.lindblad import gate_fidelity
    g = 0.4
    wl = _two_level([{"mode": 0, "L": [[0, 1], [0, 0]], "rate": g}], frame="interaction")
    sys = OracleSystem(wl)
    E = sys.modes[0]["E"][1] - sys.modes[0]["E"][0]
    T = wl["T"]
    wl["target"] = np.diag([1.0, np.exp(-1j * E * T)])
    F, _ = gate_fidelity(wl)
    p = 1.0 - np.exp(-g * T)
    assert abs(F - ((1.0 + np.sqrt(1.0 - p)) ** 2 + 2.0) / 6.0) < 1e-12


def test_gate_fidelity_without_collapse_matches_the_closed_system():
    from oracle.evolve import evolve_and_fidelity
    from oracle.lindblad import gate_fidelity
    wl = W.fluxonium_pair_cr(seed=6, nseg=3, T=0.2)
    wl["drives"][0]["length"] = 0.2
    F, _ = gate_fidelity(wl)
    assert abs(F - evolve_and_fidelity(wl)["F_avg"]) < 1e-8


def test_gate_fidelity_pulse_gradient_matches_central_differences():
    import copy
    from oracle.lindblad import gate_fidelity, gate_fidelity_pulse_gradient
    wl = W.transmon_pair(seed=2, T=0.06, dt=0.01)
    wl["modes"] = [dict(m, levels=2) for m in wl["modes"]]
    wl["col_index"] = [0, 1, 2, 3]
    wl["drives"][0]["length"] = 0.06
    wl["drives"][0]["sigma"], wl["drives"][0]["t0"] = 0.015, 0.03
    wl["collapse"] = [{"mode": 0, "L": [[0, 1], [0, 0]], "rate": 0.5}, {"mode": 1, "L": [[0, 0], [0, 1]], "rate": 0.3}]
    F, g = gate_fidelity_pulse_gradient(wl)
    assert abs(F - gate_fidelity(wl)[0]) < 1e-13
    amp = wl["drives"][0]["amp"]
    h = 1e-6 * max(1.0, abs(amp))
    vals = []
    for sgn in (1, -1):
        w2 = copy.deepcopy(wl)
        w2["drives"][0]["amp"] = amp + sgn * h
        vals.append(gate_fidelity(w2)[0])
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(g[0] - fd) <= 1e-6 * max(1e-6, abs(fd)), (g[0], fd)


def test_doubled_mode_terms_reproduce_the_generator():
    # the Kronecker-term form on ket and bra modes (what the evolution kernels would
    # apply) equals the dense vectorised generator: Lv = -i H_eff
    from oracle.lindblad import doubled_terms
    for frame in ("interaction", "lab"):
        wl = W.fluxonium_pair_cr(seed=3, nseg=3, T=0.3)
        wl["drives"][0]["length"] = 0.3
        wl["frame"] = frame
        d = wl["modes"][0]["levels"]
        wl["collapse"] = [{"mode": 0, "L": np.diag(np.sqrt(np.arange(1, d)), 1), "rate": 0.05},
                          {"mode": 1, "L": np.diag(np.arange(d)), "rate": 0.02}]
        sys = OracleSystem(wl)
        one, two = doubled_terms(sys, 7, 1)
        dims2 = list(sys.dims) * 2

        def embed(f):
            out = np.ones((1, 1), dtype=complex)
            for m, dm in enumerate(dims2):
                out = np.kron(out, f.get(m, np.eye(dm)))
            return out

        Heff = sum(embed({m: X}) for m, X in enumerate(one))
        Heff = Heff + sum(embed({a: A, b: B}) for a, A, b, B in two)
        assert np.max(np.abs(-1j * Heff - liouvillian(sys, 7, 1))) < 1e-9
