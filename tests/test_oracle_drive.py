"""Pins of the oracle's time-dependent drive: the carrier cos(omega_d t + phase) of
Eq. C1, the Gaussian envelope, the cosine envelope of Eq. C2 and the RK4 stage
times t_n + {0, 1/2, 1/2, 1} dt at which a smoothly varying f_k(t) is sampled.

Each pin is fixed by physics or by an independent integrator, not by the oracle:
  * the rotating-wave Rabi solution of a resonant or detuned two-level drive, held
    within the Bloch-Siegert scale Omega/omega of the counter-rotating term;
  * the pulse-area theorem of a resonant shaped pulse (the rotation angle is g times
    the envelope's integral, a closed form for the Gaussian and the cosine shape);
  * fourth-order convergence (error ratio ~16 per halving of dt) against a
    lab-frame DOP853 solution with the Hamiltonian written out from the mode data;
  * planted mistakes (a stage sampled at the step's start, sigma^2 for 2 sigma^2)
    that each of these pins rejects.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.special import erf

import oracle.system as osys
from oracle.evolve import initial_columns, rk4_evolve, frame_epilogue
from oracle.system import OracleSystem, envelope

GHZ = 2 * np.pi


def _flux(el=1.0, levels=4):
    return {"kind": "fluxonium", "ej": 4.0 * GHZ, "ec": 1.0 * GHZ, "el": el * GHZ,
            "phi_ext": np.pi, "n_osc": 50, "levels": levels}


def _wl(modes, couplings=(), drives=(), T=1.0, dt=0.01, frame="interaction", cols=None):
    dims = [m["levels"] for m in modes]
    D = int(np.prod(dims))
    return {"name": "t", "modes": list(modes), "couplings": list(couplings),
            "drives": list(drives), "T": T, "dt": dt, "frame": frame,
            "col_index": list(range(D)) if cols is None else cols,
            "target": np.eye(2 ** len(modes), dtype=complex), "fid_kind": "avg"}


def _two_level():
    s = OracleSystem(_wl([_flux(1.0, 2)], cols=[0]))
    return s.modes[0]["E"][1], float(s.op(0, "phi")[0, 1].real)


# ----------------------------------------------------------------------------
# rotating-wave Rabi solution (Eq. C1 carrier) and pulse areas (Gaussian, Eq. C2)
# ----------------------------------------------------------------------------
def _rabi_run(drive, T, dt, frame="interaction"):
    wl = _wl([_flux(1.0, 2)], drives=[drive], T=T, dt=dt, frame=frame, cols=[0])
    s = OracleSystem(wl)
    return s, rk4_evolve(s, initial_columns(s, [0]))[:, 0]


def _rwa_state(theta, phase):
    """exp(-i (theta/2) (cos(phase) sx - sin(phase) sy)) |0>: the resonant RWA
    propagator of H_I,01 = (g E(t)/2) exp(i phase)."""
    return np.array([np.cos(theta / 2), -1j * np.exp(-1j * phase) * np.sin(theta / 2)])


@pytest.mark.parametrize("env", ["constant", "gaussian", "cosine"])
def test_resonant_carrier_matches_rwa_within_bloch_siegert_scale(env):
    w, g = _two_level()
    T, dt, phase = 200.0, 0.02, 0.7
    om = 0.005             # Rabi rate g E of the constant drive; the shaped ones peak at 2 om
    if env == "constant":
        A = om / g
        dr = {"mode": 0, "op": "phi", "env": "pwc", "amps": [A], "length": T,
              "omega_d": w, "phase": phase}
        theta, peak = g * A * T, g * A
    elif env == "gaussian":
        A, sig = 2 * om / g, T / 4
        dr = {"mode": 0, "op": "phi", "env": "gaussian", "amp": A, "sigma": sig, "t0": T / 2,
              "length": T, "omega_d": w, "phase": phase}
        # area of A exp(-(t - T/2)^2 / (2 sigma^2)) over [0, T]
        theta, peak = g * A * sig * np.sqrt(2 * np.pi) * erf(T / (2 * np.sqrt(2) * sig)), g * A
    else:
        A = 2 * om / g
        dr = {"mode": 0, "op": "phi", "env": "cosine", "amp": A, "length": T,
              "omega_d": w, "phase": phase}
        # area of (A/2)(1 - cos(2 pi t / T)) over [0, T] is A T / 2 (Eq. C2)
        theta, peak = g * A * T / 2, g * A
    bound = peak / w                               # Bloch-Siegert scale Omega / omega
    assert bound < 3e-3
    s, psi = _rabi_run(dr, T, dt)
    ref = _rwa_state(theta, phase)
    assert np.max(np.abs(psi - ref)) < bound
    # the lab frame carries the same state times the free phases exp(-i E t)
    s_lab, psi_lab = _rabi_run(dr, T, dt, frame="lab")
    ref_lab = np.exp(-1j * s_lab.modes[0]["E"] * T) * ref
    assert np.max(np.abs(psi_lab - ref_lab)) < bound


def test_detuned_carrier_population_matches_rabi_formula():
    # omega_d = omega + Delta: P1 = Om^2/(Om^2+Delta^2) sin^2(sqrt(Om^2+Delta^2) T / 2)
    w, g = _two_level()
    T, dt = 300.0, 0.02
    om = 0.006
    delta = 0.8 * om
    dr = {"mode": 0, "op": "phi", "env": "pwc", "amps": [om / g], "length": T,
          "omega_d": w + delta, "phase": 0.0}
    _, psi = _rabi_run(dr, T, dt)
    W = np.sqrt(om ** 2 + delta ** 2)
    p1 = om ** 2 / W ** 2 * np.sin(W * T / 2) ** 2
    assert abs(abs(psi[1]) ** 2 - p1) < 2 * om / w
    # and the population differs from the resonant one by far more than the bound
    assert abs(p1 - np.sin(om * T / 2) ** 2) > 20 * om / w


def test_cosine_envelope_shape_eq_c2():
    # (A/2)(1 - cos(2 pi t / tau)): zero at both ends, A at the centre, A/2 at a
    # quarter, symmetric about the centre, zero after the pulse
    dt, L, A = 0.01, 4.0, 1.7
    dr = {"env": "cosine", "amp": A, "length": L}

    def E(m):                                      # at half step m (t = m dt / 2)
        return envelope(dr, m // 2, m % 2, dt)[0]
    M = int(round(2 * L / dt))
    assert abs(E(0)) < 1e-15 and abs(E(M)) < 1e-15
    assert abs(E(M // 2) - A) < 1e-15
    assert abs(E(M // 4) - A / 2) < 1e-14
    for m in (3, 17, 101, 250):
        assert abs(E(m) - E(M - m)) < 1e-13
    assert E(M + 1) == 0.0


def test_gaussian_envelope_width():
    # E(t0 +- sigma) / E(t0) = exp(-1/2); the derivative of E w.r.t. the amplitude
    # is the unit-height shape
    dt, sig, t0, A = 0.01, 0.5, 1.0, 2.3
    dr = {"env": "gaussian", "amp": A, "sigma": sig, "t0": t0, "length": 2.0}
    e0, g0 = envelope(dr, 100, 0, dt)              # t = 1.0
    e1, _ = envelope(dr, 150, 0, dt)               # t = 1.5 = t0 + sigma
    e2, _ = envelope(dr, 50, 0, dt)                # t = 0.5 = t0 - sigma
    assert abs(e0 - A) < 1e-15 and abs(g0[0] - 1.0) < 1e-15
    assert abs(e1 / e0 - np.exp(-0.5)) < 1e-14 and abs(e2 / e0 - np.exp(-0.5)) < 1e-14


# ----------------------------------------------------------------------------
# stage times: fourth-order convergence against an independent integrator
# ----------------------------------------------------------------------------
T_SLOPE = 2.0


def _slope_wl(dt, frame):
    dr = [{"mode": 0, "op": "phi", "env": "gaussian", "amp": 0.6, "sigma": T_SLOPE / 4,
           "t0": T_SLOPE / 2, "length": T_SLOPE, "omega_mode": 0, "phase": 0.3},
          {"mode": 1, "op": "n", "env": "cosine", "amp": 0.5, "length": T_SLOPE,
           "omega_d": 2.9, "phase": -0.4}]
    cp = [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": 0.15}]
    return _wl([_flux(0.9, 3), _flux(1.1, 3)], cp, dr, T=T_SLOPE, dt=dt, frame=frame)


def _reference_propagators():
    """Lab-frame propagator by DOP853 (rtol 1e-13) with H_lab(t) written out from
    the mode energies and operators: diag levels, the two drives of Eq. C1 with
    their envelopes, and the n (x) n coupling; and its interaction-frame image
    exp(i H_d T) U_lab."""
    s = OracleSystem(_slope_wl(0.02, "lab"))
    E0, E1 = s.modes[0]["E"], s.modes[1]["E"]
    I3 = np.eye(3)
    Hd = np.kron(np.diag(E0), I3) + np.kron(I3, np.diag(E1))
    O0 = np.kron(s.op(0, "phi"), I3)
    O1 = np.kron(I3, s.op(1, "n"))
    C = 0.15 * np.kron(s.op(0, "n"), s.op(1, "n"))
    w0, T = E0[1], T_SLOPE

    def H(t):
        f0 = 0.6 * np.exp(-(t - T / 2) ** 2 / (2 * (T / 4) ** 2)) * np.cos(w0 * t + 0.3)
        f1 = 0.25 * (1 - np.cos(2 * np.pi * t / T)) * np.cos(2.9 * t - 0.4)
        return Hd + f0 * O0 + f1 * O1 + C

    sol = solve_ivp(lambda t, y: (-1j * (H(t) @ y.reshape(9, 9))).reshape(-1), (0.0, T),
                    np.eye(9, dtype=complex).reshape(-1), method="DOP853", rtol=1e-13, atol=1e-13)
    U_lab = sol.y[:, -1].reshape(9, 9)
    return U_lab, np.exp(1j * np.diag(Hd) * T)[:, None] * U_lab


def _errors(ref, frame, dts):
    out = []
    for dt in dts:
        s = OracleSystem(_slope_wl(dt, frame))
        psi = rk4_evolve(s, initial_columns(s, s.wl["col_index"]))
        out.append(np.max(np.abs(psi - ref)))
    return np.array(out)


@pytest.fixture(scope="module")
def refs():
    return _reference_propagators()


def test_smooth_drive_converges_fourth_order_interaction_frame(refs):
    _, U_int = refs
    e = _errors(U_int, "interaction", (0.02, 0.01, 0.005))
    r = e[:-1] / e[1:]
    assert np.all((14 < r) & (r < 18)), (e, r)
    assert e[-1] < 1e-7


def test_smooth_drive_converges_fourth_order_lab_frame(refs):
    U_lab, _ = refs
    e = _errors(U_lab, "lab", (0.01, 0.005, 0.0025))
    r = e[:-1] / e[1:]
    assert np.all((14 < r) & (r < 18)), (e, r)


def test_frames_agree_on_the_reference(refs):
    # frame_epilogue maps the interaction-frame result onto the lab frame
    U_lab, _ = refs
    s = OracleSystem(_slope_wl(0.005, "interaction"))
    psi = frame_epilogue(s, rk4_evolve(s, initial_columns(s, s.wl["col_index"])))
    assert np.max(np.abs(psi - U_lab)) < 1e-7


# ----------------------------------------------------------------------------
# planted mistakes (in the oracle, on the CPU) that the pins above reject
# ----------------------------------------------------------------------------
def test_planted_stage_time_mistake_breaks_the_order(refs, monkeypatch):
    # the midpoint stages sampled at the step's start: t(2n+1) -> t_n
    _, U_int = refs
    monkeypatch.setattr(osys, "half_step_time", lambda m, dt: (m // 2) * dt)
    e = _errors(U_int, "interaction", (0.02, 0.01, 0.005))
    r = e[:-1] / e[1:]
    assert not np.all((14 < r) & (r < 18))


def test_planted_carrier_offset_breaks_rwa(monkeypatch):
    # the carrier evaluated half a step late: outside the Bloch-Siegert scale
    w, g = _two_level()
    T, dt, phase, om = 200.0, 0.02, 0.7, 0.005
    dr = {"mode": 0, "op": "phi", "env": "pwc", "amps": [om / g], "length": T,
          "omega_d": w, "phase": phase}
    orig = OracleSystem.coeff

    def late(self, k, n, j):
        E, _ = envelope(self.drives[k], n, j, self.dt)
        t = osys.stage_time(n, j, self.dt) + self.dt / 2
        return E * np.cos(self.omega_d[k] * t + self.drives[k].get("phase", 0.0))
    monkeypatch.setattr(OracleSystem, "coeff", late)
    _, psi = _rabi_run(dr, T, dt)
    assert np.max(np.abs(psi - _rwa_state(om * T, phase))) > om / w
    monkeypatch.setattr(OracleSystem, "coeff", orig)


def test_planted_gaussian_width_mistake_breaks_pulse_area(monkeypatch):
    # exp(-(t - t0)^2 / sigma^2) instead of / (2 sigma^2)
    w, g = _two_level()
    T, dt, phase, om = 200.0, 0.02, 0.7, 0.005
    A, sig = 2 * om / g, T / 4
    dr = {"mode": 0, "op": "phi", "env": "gaussian", "amp": A, "sigma": sig, "t0": T / 2,
          "length": T, "omega_d": w, "phase": phase}
    theta = g * A * sig * np.sqrt(2 * np.pi) * erf(T / (2 * np.sqrt(2) * sig))
    orig = osys.envelope

    def narrow(drive, n, j, dt_):
        if drive["env"] != "gaussian":
            return orig(drive, n, j, dt_)
        t = osys.stage_time(n, j, dt_)
        gg = np.exp(-((t - drive["t0"]) ** 2) / drive["sigma"] ** 2)
        return drive["amp"] * gg, [gg]
    monkeypatch.setattr(osys, "envelope", narrow)
    _, psi = _rabi_run(dr, T, dt)
    assert np.max(np.abs(psi - _rwa_state(theta, phase))) > 10 * g * A / w
