"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances: FP64 path 1e-10 max-abs on every final
amplitude and on F; mixed path |dF| <= 1e-5; gradients per R12."""
import numpy as np
import pytest

import oracle
from oracle.evolve import (initial_columns, rk4_evolve, frame_epilogue, fidelities,
                           adjoint_gradient)
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(params=["onchip", "slab", "gather"])
def path(request, monkeypatch):
    """Kernel family: on-chip (the default where the columns fit in shared memory),
    the tiled HBM slab kernels, or the generic gather kernels."""
    monkeypatch.setenv("SG_PATH", request.param)
    return request.param

GHZ = 2 * np.pi


def _system(sgctx, wl):
    from paper_2406_18155_gb300.api import System
    s = System.from_workload(sgctx, wl)
    s.prepare()
    return s


def _oracle_psi(wl, psi0=None):
    s = OracleSystem(wl)
    p0 = initial_columns(s, wl["col_index"]) if psi0 is None else psi0
    return frame_epilogue(s, rk4_evolve(s, p0))


def _mixed_dims_chain(seed=0, T=0.6, dt=0.01):
    wl = W.fluxonium_chain(seed=seed, nq=3, levels=4, T=T, dt=dt, nseg=3, ring=True)
    wl["modes"][0]["levels"] = 3
    wl["modes"][2]["levels"] = 5
    dims = [3, 4, 5]
    wl["col_index"] = W.comp_states(dims) + [7, 59]       # 8 comp + 2 non-comp columns
    return wl


CASES = {
    "transmon_pair_T2": lambda: W.transmon_pair(seed=3, T=2.0),
    "fluxonium_pair_cr_T1": lambda: W.fluxonium_pair_cr(seed=5, T=1.0),
    "ring3_mixed_dims": lambda: _mixed_dims_chain(seed=2),
    "chain4_l3": lambda: W.fluxonium_chain(seed=7, nq=4, levels=3, T=0.3, dt=0.01, nseg=2),
}


@pytest.mark.parametrize("mode_spec", [
    {"kind": "transmon", "ej": 20 * GHZ, "ec": 0.25 * GHZ, "ng": 0.0, "ncut": 10, "levels": 5},
    {"kind": "transmon", "ej": 15 * GHZ, "ec": 0.3 * GHZ, "ng": 0.2, "ncut": 12, "levels": 4},
    {"kind": "fluxonium", "ej": 4 * GHZ, "ec": 1 * GHZ, "el": 0.9 * GHZ, "phi_ext": np.pi,
     "n_osc": 50, "levels": 5},
    {"kind": "fluxonium", "ej": 3.3 * GHZ, "ec": 1.1 * GHZ, "el": 1.05 * GHZ, "phi_ext": 2.9,
     "n_osc": 64, "levels": 8},
])
def test_spectrum_matches_oracle(sgctx, mode_spec):
    from oracle.subsystems import build_mode
    wl = {"modes": [mode_spec], "couplings": [], "drives": []}
    s = _system(sgctx, wl)
    d = mode_spec["levels"]
    E, n, phi = s.spectrum(0, d)
    ref = build_mode(mode_spec)
    assert np.max(np.abs(E - ref["E"])) < 1e-10
    assert np.max(np.abs(n - ref["ops"]["n"])) < 1e-10
    if mode_spec["kind"] == "fluxonium":
        assert np.max(np.abs(phi - ref["ops"]["phi"])) < 1e-10


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("frame", ["interaction", "lab"])
def test_fp64_evolution_matches_oracle(sgctx, case, frame, path):
    wl = CASES[case]()
    wl["frame"] = frame
    if frame == "lab":
        wl["T"] = round(min(wl["T"], 0.2) / wl["dt"]) * wl["dt"]
        for d in wl["drives"]:
            d["length"] = wl["T"]
    s = _system(sgctx, wl)
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", frame=frame,
                   col_index=wl["col_index"]).cpu().numpy()
    ref = _oracle_psi(wl)
    assert np.max(np.abs(psi - ref)) < 1e-10


@pytest.mark.parametrize("case", sorted(CASES))
def test_fidelity_fp64_and_mixed(sgctx, case, path):
    wl = CASES[case]()
    s = _system(sgctx, wl)
    sysr = OracleSystem(wl)
    ref_psi = _oracle_psi(wl)
    Fa_ref, Fs_ref, Uc_ref = fidelities(sysr, ref_psi)
    Fa, Fs, Uc = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64")
    assert abs(Fs - Fs_ref) < 1e-10
    assert np.max(np.abs(Uc - Uc_ref)) < 1e-10
    if np.isnan(Fa_ref):
        assert np.isnan(Fa)
    else:
        assert abs(Fa - Fa_ref) < 1e-10
    Fa32, Fs32, _ = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="mixed")
    assert abs(Fs32 - Fs_ref) < 1e-5
    if not np.isnan(Fa_ref):
        assert abs(Fa32 - Fa_ref) < 1e-5


def test_evolve_from_arbitrary_states(sgctx):
    import torch
    wl = CASES["ring3_mixed_dims"]()
    s = _system(sgctx, wl)
    D = 60
    psi0 = W.random_columns(D, 5, seed=11)
    dev = torch.from_numpy(psi0.copy()).to("cuda")
    out = s.evolve(wl["T"], wl["dt"], precision="fp64", psi=dev).cpu().numpy()
    assert np.max(np.abs(out - _oracle_psi(wl, psi0))) < 1e-10


@pytest.mark.parametrize("case", ["fluxonium_pair_cr_T1", "transmon_pair_T2", "ring3_mixed_dims"])
def test_gradient_fp64_matches_oracle_adjoint(sgctx, case, path):
    wl = CASES[case]()
    if case == "transmon_pair_T2":
        wl["T"] = 0.5
        for d in wl["drives"]:
            d["length"] = 0.5
    if case == "fluxonium_pair_cr_T1":
        wl["T"] = 0.4
        wl["drives"][0]["length"] = 0.4
    s = _system(sgctx, wl)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                kind=wl["fid_kind"], precision="fp64", ckpt=7)
    Fr, gr, prms = adjoint_gradient(wl)
    g = np.concatenate([gp, gh])
    kind_index = 0 if wl["fid_kind"] == "avg" else 1
    assert abs(F[kind_index] - Fr) < 1e-10
    scale = np.max(np.abs(gr))
    assert np.max(np.abs(g - gr)) <= 1e-8 * scale, (g, gr)


def test_gradient_mixed_matches_oracle(sgctx, path):
    wl = CASES["fluxonium_pair_cr_T1"]()
    s = _system(sgctx, wl)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                kind="avg", precision="mixed")
    Fr, gr, _ = adjoint_gradient(wl)
    g = np.concatenate([gp, gh])
    assert abs(F[0] - Fr) < 1e-5
    assert np.max(np.abs(g - gr)) <= 1e-3 * np.max(np.abs(gr))


def test_invalid_inputs_are_rejected(sgctx):
    from paper_2406_18155_gb300.api import System
    from paper_2406_18155_gb300.capi import SGError, SG_E_INVALID, SG_E_STATE
    wl = W.transmon_pair(seed=0, T=1.0)
    s = System.from_workload(sgctx, wl)
    with pytest.raises(SGError) as e:
        s.evolve(1.0, 0.01, col_index=[0])
    assert e.value.code == SG_E_STATE
    s.prepare()
    with pytest.raises(SGError) as e:
        s.evolve(1.0, 0.003, col_index=[0])           # T/dt not integral
    assert e.value.code == SG_E_INVALID
    with pytest.raises(SGError) as e:
        s.evolve(1.0, 0.01, col_index=[16])           # out of range
    assert e.value.code == SG_E_INVALID
    with pytest.raises(SGError):
        s.add_coupling(0, "phi", 1, "n", 0.1)         # transmon has no phi


@pytest.mark.parametrize("tmax,nq,levels,ring", [(9, 4, 3, False), (27, 4, 3, True), (4, 5, 2, True)])
def test_multipass_slab_matches_oracle(sgctx, monkeypatch, tmax, nq, levels, ring):
    # a small tile budget splits the terms over several mode-group passes
    monkeypatch.setenv("SG_PATH", "slab")
    monkeypatch.setenv("SG_SLAB_TMAX", str(tmax))
    wl = W.fluxonium_chain(seed=tmax, nq=nq, levels=levels, T=0.3, dt=0.01, nseg=3, ring=ring)
    s = _system(sgctx, wl)
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi - _oracle_psi(wl))) < 1e-10
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                precision="fp64", ckpt=5)
    Fr, gr, _ = adjoint_gradient(wl)
    assert abs(F[1] - Fr) < 1e-10
    assert np.max(np.abs(np.concatenate([gp, gh]) - gr)) <= 1e-8 * np.max(np.abs(gr))
    F32, gp32, gh32 = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                      kind="state", precision="mixed", ckpt=5)
    assert abs(F32[1] - Fr) < 1e-5
    assert np.max(np.abs(np.concatenate([gp32, gh32]) - gr)) <= 1e-3 * np.max(np.abs(gr))


def test_two_pass_ring7_against_matrix_free_oracle(sgctx, monkeypatch):
    # D = 4^7 = 16384 > one tile: the ring splits into two overlapping mode groups
    from oracle.evolve import rk4_evolve_matrix_free
    monkeypatch.setenv("SG_PATH", "slab")
    wl = W.fluxonium_chain(seed=9, nq=7, levels=4, T=0.1, dt=0.01, nseg=2, ring=True, ncols=3)
    s = _system(sgctx, wl)
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
    so = OracleSystem(wl)
    ref = frame_epilogue(so, rk4_evolve_matrix_free(so, initial_columns(so, wl["col_index"])))
    assert np.max(np.abs(psi - ref)) < 1e-10
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi32 - ref)) < 1e-5
    # gradient: the slab kernels against the independent gather kernels
    g = {}
    for pth in ("slab", "gather"):
        monkeypatch.setenv("SG_PATH", pth)
        F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                    kind="state", precision="fp64", ckpt=3)
        g[pth] = (F, np.concatenate([gp, gh]))
    assert abs(g["slab"][0][1] - g["gather"][0][1]) < 1e-12
    assert np.max(np.abs(g["slab"][1] - g["gather"][1])) <= 1e-10 * np.max(np.abs(g["gather"][1]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pulse_only_gradient_equals_the_pulse_part(sgctx, path, precision):
    # without a Hamiltonian-gradient buffer the coupling-term cross-densities are
    # skipped; the pulse gradient comes from the driven terms alone and is unchanged
    wl = W.fluxonium_chain(seed=12, nq=4, levels=3, T=0.3, dt=0.01, nseg=3, ring=True)
    s = _system(sgctx, wl)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                precision=precision, ckpt=5)
    F2, gp2, gh2 = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                   precision=precision, ckpt=5, ham=False)
    assert gh2 is None and gh is not None
    assert np.array_equal(F, F2)
    assert np.max(np.abs(gp2 - gp)) <= 1e-14 * np.max(np.abs(gp))
