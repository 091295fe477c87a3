"""Pins of the oracle's virtual-Z compensation of the gate fidelity (the errorless
phase gates around the pulses of the paper's gate metric): brute force for one
qubit, exact recovery of known phase gates, stationarity, and the envelope-theorem
gradient against central differences."""
import copy

import numpy as np
from scipy.optimize import minimize

from oracle.compensation import compensate, compensated_fidelities
from oracle.evolve import adjoint_gradient, rk4_evolve, frame_epilogue, initial_columns
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W


def _haar(n, rng):
    z = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _z(phases):
    g = np.eye(1, dtype=complex)
    for p in phases:
        g = np.kron(g, np.diag([1.0, np.exp(1j * p)]))
    return g


def test_one_qubit_matches_brute_force():
    rng = np.random.default_rng(1)
    for _ in range(4):
        T, U = _haar(2, rng), _haar(2, rng)
        f = lambda p: -abs(np.trace(T.conj().T @ _z([p[0]]) @ U @ _z([p[1]])))
        grid = np.linspace(0, 2 * np.pi, 73)
        start = min(((x, y) for x in grid for y in grid), key=f)
        ref = -minimize(f, start, method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-15}).fun
        _, _, best, _ = compensate(T, U, 1)
        assert best >= ref - 1e-9


def test_known_phase_gates_are_recovered():
    # U = Z(a) T Z(b) on three qubits with phases within +-0.5: the compensated F is 1
    rng = np.random.default_rng(3)
    T = _haar(8, rng)
    a0, b0 = rng.uniform(-0.5, 0.5, 3), rng.uniform(-0.5, 0.5, 3)
    U = _z(a0) @ T @ _z(b0)
    a, b, best, T_eff = compensate(T, U, 3)
    assert abs(best - 8) < 1e-12
    assert abs(abs(np.trace(T_eff.conj().T @ U)) - best) < 1e-12
    # the Kronecker product of the found gates reproduces tr M
    assert abs(abs(np.trace(T.conj().T @ _z(a) @ U @ _z(b))) - best) < 1e-12


def test_result_is_stationary_and_not_below_the_uncompensated():
    rng = np.random.default_rng(4)
    T, U = _haar(4, rng), 0.97 * _haar(4, rng)              # a little leakage
    a, b, best, _ = compensate(T, U, 2)
    assert best >= abs(np.trace(T.conj().T @ U))
    f = lambda a, b: abs(np.trace(T.conj().T @ _z(a) @ U @ _z(b)))
    eps = 1e-6
    for k in range(4):
        d = np.zeros(4)
        d[k] = eps
        up = f(a + d[:2], b + d[2:])
        dn = f(a - d[:2], b - d[2:])
        assert abs(up - dn) / (2 * eps) < 1e-7


def test_compensated_gradient_matches_central_differences():
    # at the maximiser F is stationary in the phases, so the co-state of the plain
    # fidelity against T_eff gives dF/dtheta of the compensated fidelity
    wl = W.transmon_pair(seed=5, T=0.5, dt=0.005)
    wl["drives"][0]["length"] = 0.5
    wl["drives"][0]["sigma"], wl["drives"][0]["t0"] = 0.125, 0.25
    wl["col_index"] = W.comp_states([m["levels"] for m in wl["modes"]])
    wl["fid_kind"] = "avg"

    def comp_F(w):
        s = OracleSystem(w)
        psi = frame_epilogue(s, rk4_evolve(s, initial_columns(s, w["col_index"])))
        return compensated_fidelities(s, psi)

    Fa, _, T_eff = comp_F(wl)
    F_eff, g, _ = adjoint_gradient(dict(wl, target=T_eff), kind="avg")
    assert abs(F_eff - Fa) < 1e-13
    amp = wl["drives"][0]["amp"]
    h = 1e-5 * max(1.0, abs(amp))
    vals = []
    for sgn in (1, -1):
        w2 = copy.deepcopy(wl)
        w2["drives"][0]["amp"] = amp + sgn * h
        vals.append(comp_F(w2)[0])
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(g[0] - fd) <= 1e-6 * max(1e-6, abs(fd)), (g[0], fd)
