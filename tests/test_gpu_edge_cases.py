"""Edge cases of the path against the FP64 oracle: one mode, no drives, no
couplings, one RK4 step, one column, the largest level count (8) and mode count
(16), unequal level counts 2 and 8, a zero-amplitude drive, and degenerate
inputs that must be rejected.  FP64: states 1e-10, F 1e-10, gradients 1e-8 of
the largest component; mixed: states 1e-5."""
import copy

import numpy as np
import pytest

from oracle.evolve import (initial_columns, rk4_evolve, rk4_evolve_matrix_free, frame_epilogue,
                           fidelities, adjoint_gradient)
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GHZ, MHZ = W.GHZ, W.MHZ


def _system(sgctx, wl):
    from paper_2406_18155_gb300.api import System
    s = System.from_workload(sgctx, wl)
    s.prepare()
    return s


def _transmon(levels, ej=20.0, ec=0.25):
    return {"kind": "transmon", "ej": ej * GHZ, "ec": ec * GHZ, "ng": 0.0, "ncut": 10, "levels": levels}


def _fluxonium(levels, ej=4.0, ec=1.0, el=1.0):
    return {"kind": "fluxonium", "ej": ej * GHZ, "ec": ec * GHZ, "el": el * GHZ, "phi_ext": np.pi,
            "n_osc": 50, "levels": levels}


def _pwc(mode, op, T, amps, omega_mode):
    return {"mode": mode, "op": op, "env": "pwc", "amps": [a * MHZ for a in amps], "length": T,
            "omega_mode": omega_mode, "phase": 0.0}


def _wl(modes, couplings, drives, T=0.2, dt=0.01, cols=None, seed=0):
    dims = [m["levels"] for m in modes]
    nqb = sum(1 for m in modes if not m.get("coupler"))
    rng = np.random.Generator(np.random.PCG64(seed))
    return {"name": "edge", "modes": modes, "couplings": couplings, "drives": drives, "T": T, "dt": dt,
            "frame": "interaction", "col_index": cols if cols is not None else W.comp_states(dims),
            "target": W.haar_unitary(2 ** nqb, rng), "fid_kind": "avg"}


def _cases():
    T = 0.2
    c = {}
    c["single_mode"] = _wl([_transmon(4)], [], [_pwc(0, "n", T, [30, 20], 0)], cols=[0, 1, 2, 3])
    c["undriven_pair"] = _wl([_fluxonium(3), _fluxonium(3, ej=4.5)],
                             [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": 25 * MHZ}], [])
    c["uncoupled_pair"] = _wl([_transmon(3), _transmon(3, ej=18.0)], [],
                              [_pwc(0, "n", T, [30, 10], 0), _pwc(1, "n", T, [15, 40], 1)])
    one = _wl([_transmon(4), _transmon(4, ej=17.0)],
              [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": 15 * MHZ}],
              [_pwc(0, "n", 0.01, [40], 1)], T=0.01)
    c["one_step"] = one
    col = _wl([_fluxonium(5), _fluxonium(5, ej=3.5)],
              [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": 20 * MHZ}],
              [_pwc(0, "phi", T, [30, 45, 10], 1)])
    col["col_index"] = [col["col_index"][1]]
    col["fid_kind"] = "state"
    c["one_column"] = col
    c["levels8_pair"] = _wl([_transmon(8), _transmon(8, ej=16.0)],
                            [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": 10 * MHZ}],
                            [_pwc(0, "n", T, [20, 30], 0), _pwc(1, "n", T, [35, 5], 1)])
    c["levels_2_and_8"] = _wl([_transmon(2), _fluxonium(8)],
                              [{"a": 0, "op_a": "n", "b": 1, "op_b": "phi", "J": 30 * MHZ}],
                              [_pwc(1, "phi", T, [25, 35], 1)])
    zero = copy.deepcopy(c["undriven_pair"])
    zero["drives"] = [_pwc(0, "phi", T, [0.0, 0.0], 0)]
    c["zero_amplitude_drive"] = zero
    return c


CASES = _cases()


@pytest.fixture
def default_path(monkeypatch):
    monkeypatch.delenv("SG_PATH", raising=False)
    monkeypatch.delenv("SG_SLAB_TMAX", raising=False)


@pytest.mark.parametrize("name", sorted(CASES))
def test_edge_case_states_fidelity_gradient(sgctx, default_path, name):
    wl = CASES[name]
    s = _system(sgctx, wl)
    so = OracleSystem(wl)
    ref = frame_epilogue(so, rk4_evolve(so, initial_columns(so, wl["col_index"])))
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi - ref)) < 1e-10
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi32 - ref)) < 1e-5
    Fa_r, Fs_r, _ = fidelities(so, ref)
    Fa, Fs, _ = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64")
    assert abs(Fs - Fs_r) < 1e-10
    assert (np.isnan(Fa) and np.isnan(Fa_r)) or abs(Fa - Fa_r) < 1e-10
    Fr, gr, _ = adjoint_gradient(wl)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=wl["fid_kind"],
                                precision="fp64", ckpt=3)
    k = 0 if wl["fid_kind"] == "avg" else 1
    assert abs(F[k] - Fr) < 1e-10
    g = np.concatenate([gp, gh])
    assert np.max(np.abs(g - gr)) <= 1e-8 * max(1e-12, np.max(np.abs(gr)))


def test_zero_amplitude_drive_equals_undriven(sgctx, default_path):
    a, b = CASES["undriven_pair"], CASES["zero_amplitude_drive"]
    Fa = _system(sgctx, a).fidelity(a["T"], a["dt"], a["target"], a["col_index"], precision="fp64")
    Fb = _system(sgctx, b).fidelity(b["T"], b["dt"], b["target"], b["col_index"], precision="fp64")
    assert abs(Fa[0] - Fb[0]) < 1e-14 and np.max(np.abs(Fa[2] - Fb[2])) < 1e-14


def test_sixteen_two_level_modes(sgctx, default_path):
    # the largest mode count: D = 2^16, split over several tile passes
    modes = [_transmon(2, ej=15.0 + 0.5 * i) for i in range(16)]
    couplings = [{"a": i, "op_a": "n", "b": i + 1, "op_b": "n", "J": 20 * MHZ} for i in range(15)]
    drives = [_pwc(i, "n", 0.02, [30], i) for i in range(0, 16, 3)]
    wl = {"name": "edge16", "modes": modes, "couplings": couplings, "drives": drives, "T": 0.02,
          "dt": 0.01, "frame": "interaction", "col_index": [0, 12345]}   # evolution only, no target
    s = _system(sgctx, wl)
    so = OracleSystem(wl)
    ref = frame_epilogue(so, rk4_evolve_matrix_free(so, initial_columns(so, wl["col_index"])))
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi - ref)) < 1e-10
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi32 - ref)) < 1e-5


def test_degenerate_inputs_are_rejected(sgctx):
    from paper_2406_18155_gb300.api import System
    from paper_2406_18155_gb300.capi import SGError
    empty = System(sgctx)
    with pytest.raises(SGError):
        empty.prepare()                                       # a system needs modes
    with pytest.raises(SGError):
        empty.evolve(0.1, 0.01, col_index=[0])                # and must be prepared
    wl = CASES["uncoupled_pair"]
    s = _system(sgctx, wl)
    for T, dt in [(0.0, 0.01), (0.1, 0.0), (-0.1, 0.01), (float("nan"), 0.01)]:
        with pytest.raises(SGError):
            s.evolve(T, dt, col_index=[0])
    with pytest.raises(SGError):
        s.evolve(0.1, 0.01, col_index=[])                      # no columns
    with pytest.raises(SGError):
        s.fidelity(0.1, 0.01, wl["target"], [2 * 3 + 2])      # no computational column
