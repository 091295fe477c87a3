"""GPU parity of the open-system (Lindblad) evolution (sg_evolve_open,
sg_gate_fidelity_open: vec(rho) on the doubled ket/bra modes, run by the RK4
kernels) against the FP64 oracle's dense superoperator RK4 (oracle/lindblad.py),
through the C ABI.  FP64 within 1e-10 on every density-matrix entry and on F,
mixed within 1e-5; the closed-system limit matches the oracle's and, within RK4's
truncation, the pure-state fidelity; the amplitude-damping closed form holds on
the GPU too.  The pulse-parameter gradient of the gate fidelity
(sg_gate_fidelity_open_grad) against the oracle's discrete adjoint of the
superoperator RK4 (FP64 within 1e-8 of its largest component, mixed 1e-3) on all
three kernel families, and its process-fidelity variant against central
differences; the Hamiltonian-parameter gradient (E_J, E_C, E_L, J through the
eigen-derivatives) against central differences of the oracle's gate fidelity and,
without collapse operators, against the closed-system gradient."""
import numpy as np
import pytest

from oracle.lindblad import evolve_density, gate_fidelity, gate_fidelity_pulse_gradient
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system(sgctx, wl):
    from paper_2406_18155_gb300.api import System
    s = System.from_workload(sgctx, wl)
    s.prepare()
    return s


def _lowering(d):
    return np.diag(np.sqrt(np.arange(1, d)), 1).astype(complex)


def _flux_cr(levels=3, T=0.3, frame="interaction"):
    wl = W.fluxonium_pair_cr(seed=2, nseg=3, T=T)
    for m in wl["modes"]:
        m["levels"] = levels
    wl["col_index"] = W.comp_states([levels, levels])
    wl["frame"] = frame
    d = levels
    wl["collapse"] = [{"mode": 0, "L": _lowering(d), "rate": 0.05},
                      {"mode": 1, "L": np.diag(np.arange(d)).astype(complex), "rate": 0.02},
                      {"mode": 1, "L": _lowering(d), "rate": 0.03}]
    return wl


def _transmon(levels=4, T=0.4, frame="interaction"):
    wl = W.transmon_pair(seed=5, T=T)
    for m in wl["modes"]:
        m["levels"] = levels
    wl["col_index"] = W.comp_states([levels, levels])
    wl["frame"] = frame
    wl["collapse"] = [{"mode": 0, "L": _lowering(levels), "rate": 0.1},
                      {"mode": 1, "L": _lowering(levels), "rate": 0.08}]
    return wl


@pytest.mark.parametrize("frame", ["interaction", "lab"])
@pytest.mark.parametrize("make", [_flux_cr, _transmon])
def test_open_density_matrix_matches_oracle(sgctx, make, frame):
    wl = make(frame=frame) if frame == "interaction" else make(T=0.05, frame=frame)
    if frame == "lab":
        wl["dt"] = 0.001
    s = _system(sgctx, wl)
    D = int(np.prod([m["levels"] for m in wl["modes"]]))
    rng = np.random.Generator(np.random.PCG64(4))
    X = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    rho0 = X @ X.conj().T
    rho0 /= np.trace(rho0)
    ref = evolve_density(wl, rho0)
    r64 = s.evolve_open(wl["T"], wl["dt"], rho0, precision="fp64", frame=frame)
    r32 = s.evolve_open(wl["T"], wl["dt"], rho0, precision="mixed", frame=frame)
    assert np.max(np.abs(r64 - ref)) < 1e-10
    assert np.max(np.abs(r32 - ref)) < 1e-5
    assert abs(np.trace(r64) - 1.0) < 1e-12                  # the generator preserves the trace


@pytest.mark.parametrize("make", [_flux_cr, _transmon])
def test_open_gate_fidelity_matches_oracle(sgctx, make):
    wl = make()
    s = _system(sgctx, wl)
    Fa, Fp = gate_fidelity(wl)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        ga, gp = s.gate_fidelity_open(wl["T"], wl["dt"], wl["target"], precision=prec)
        assert abs(ga - Fa) < tol and abs(gp - Fp) < tol, (prec, ga, Fa, gp, Fp)


def test_closed_limit_against_oracle_and_pure_state_fidelity(sgctx):
    # without collapse operators: the oracle's superoperator RK4 (the same map) within
    # 1e-10; the pure-state F_avg within RK4's truncation, since RK4 on vec(rho) and
    # R4 rho R4^dag from RK4 on the states differ at fifth order per step
    wl = _transmon()
    wl["collapse"] = []
    s = _system(sgctx, wl)
    ga, _ = s.gate_fidelity_open(wl["T"], wl["dt"], wl["target"], precision="fp64")
    Fo, _ = gate_fidelity(wl)
    assert abs(ga - Fo) < 1e-10
    Fa, _, _ = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64")
    assert abs(ga - Fa) < 1e-8


def test_amplitude_damping_closed_form_on_the_gpu(sgctx):
    # one 2-level transmon, no drive: rho_11 = e^{-g T} rho_11(0), rho_01 = e^{-g T/2} e^{i E T} rho_01(0)
    wl = W.transmon_pair(seed=1, T=2.0, dt=0.002)
    wl["modes"] = [dict(wl["modes"][0], levels=2)]
    wl["drives"], wl["couplings"] = [], []
    wl["col_index"] = [0, 1]
    g = 0.7
    wl["collapse"] = [{"mode": 0, "L": [[0, 1], [0, 0]], "rate": g}]
    s = _system(sgctx, wl)
    E, _, _ = s.spectrum(0, 2)
    rho0 = 0.5 * np.array([[1, 1], [1, 1]], dtype=complex)
    rho = s.evolve_open(wl["T"], wl["dt"], rho0, precision="fp64")
    assert abs(rho[1, 1] - 0.5 * np.exp(-g * 2.0)) < 1e-12
    assert abs(rho[0, 1] - 0.5 * np.exp(-g * 1.0) * np.exp(1j * (E[1] - E[0]) * 2.0)) < 1e-12


@pytest.mark.parametrize("frame", ["interaction", "lab"])
@pytest.mark.parametrize("make", [_flux_cr, _transmon])
def test_open_pulse_gradient_matches_oracle_adjoint(sgctx, make, frame):
    wl = make(frame=frame) if frame == "interaction" else make(T=0.05, frame=frame)
    if frame == "lab":
        wl["dt"] = 0.001
    s = _system(sgctx, wl)
    Fr, gr = gate_fidelity_pulse_gradient(wl)
    scale = np.max(np.abs(gr))
    F, g = s.gate_fidelity_open_grad(wl["T"], wl["dt"], wl["target"], kind="avg", precision="fp64",
                                     frame=frame, ckpt=4)
    assert abs(F[0] - Fr) < 1e-10
    assert np.max(np.abs(g - gr)) <= 1e-8 * scale, (g, gr)
    F32, g32 = s.gate_fidelity_open_grad(wl["T"], wl["dt"], wl["target"], kind="avg", precision="mixed",
                                         frame=frame, ckpt=4)
    assert abs(F32[0] - Fr) < 1e-5
    assert np.max(np.abs(g32 - gr)) <= 1e-3 * scale


@pytest.mark.parametrize("path", ["slab", "gather"])
def test_open_pulse_gradient_on_the_tiled_and_gather_kernels(sgctx, monkeypatch, path):
    # the adjoint rows of the non-Hermitian generator reach every kernel family
    monkeypatch.setenv("SG_PATH", path)
    wl = _flux_cr()
    s = _system(sgctx, wl)
    Fr, gr = gate_fidelity_pulse_gradient(wl)
    F, g = s.gate_fidelity_open_grad(wl["T"], wl["dt"], wl["target"], kind="avg", precision="fp64", ckpt=3)
    assert abs(F[0] - Fr) < 1e-10
    assert np.max(np.abs(g - gr)) <= 1e-8 * np.max(np.abs(gr))


def test_open_process_fidelity_gradient_matches_central_differences(sgctx):
    wl = _flux_cr()
    s = _system(sgctx, wl)
    F, g = s.gate_fidelity_open_grad(wl["T"], wl["dt"], wl["target"], kind="pro", precision="fp64")
    npul, _ = s.param_counts()
    p0, _ = s.get_params()
    for k in range(npul):
        h = 1e-5 * max(1.0, abs(p0[k]))
        vals = []
        for sgn in (1, -1):
            p = p0.copy()
            p[k] += sgn * h
            s.set_params(pulse=p)
            vals.append(s.gate_fidelity_open(wl["T"], wl["dt"], wl["target"], precision="fp64")[1])
        s.set_params(pulse=p0)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * max(1e-3, np.max(np.abs(g))), (k, g[k], fd)


def _ham_names(wl):
    return [("mode", i, p) for i in range(len(wl["modes"])) for p in ("ej", "ec", "el")] + \
           [("coupling", e, "J") for e in range(len(wl["couplings"]))]


def test_open_hamiltonian_gradient_matches_central_differences(sgctx):
    import copy
    wl = _flux_cr()
    s = _system(sgctx, wl)
    F, gp, gh = s.gate_fidelity_open_grad(wl["T"], wl["dt"], wl["target"], kind="avg", precision="fp64",
                                          ckpt=4, ham=True)
    Fr, gr = gate_fidelity_pulse_gradient(wl)
    assert abs(F[0] - Fr) < 1e-10
    assert np.max(np.abs(gp - gr)) <= 1e-8 * np.max(np.abs(gr))
    scale = np.max(np.abs(gh))
    for idx, (what, k, p) in enumerate(_ham_names(wl)):
        v = wl["modes"][k][p] if what == "mode" else wl["couplings"][k]["J"]
        h = 1e-5 * max(abs(v), 1e-3)
        vals = []
        for sgn in (1, -1):
            w2 = copy.deepcopy(wl)
            if what == "mode":
                w2["modes"][k][p] = v + sgn * h
            else:
                w2["couplings"][k]["J"] = v + sgn * h
            vals.append(gate_fidelity(w2)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(gh[idx] - fd) <= 1e-6 * scale + 1e-9, (what, k, p, gh[idx], fd)
    F32, gp32, gh32 = s.gate_fidelity_open_grad(wl["T"], wl["dt"], wl["target"], kind="avg",
                                                precision="mixed", ckpt=4, ham=True)
    assert np.max(np.abs(gh32 - gh)) <= 1e-3 * scale


def test_open_hamiltonian_gradient_closed_limit(sgctx):
    # without collapse operators the open F_avg and its gradient are the closed ones up
    # to RK4 on vec(rho) against RK4 on the states (fifth order per step)
    wl = _transmon()
    wl["collapse"] = []
    s = _system(sgctx, wl)
    F, gp, gh = s.gate_fidelity_open_grad(wl["T"], wl["dt"], wl["target"], kind="avg", precision="fp64",
                                          ham=True)
    Fc, gpc, ghc = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg",
                                   precision="fp64")
    assert abs(F[0] - Fc[0]) < 1e-8
    assert np.max(np.abs(gp - gpc)) <= 1e-6 * np.max(np.abs(gpc))
    assert np.max(np.abs(gh - ghc)) <= 1e-6 * np.max(np.abs(ghc))
