"""GPU parity of the tiled kernels' real-operator passes (every local operator real
in the truncated eigenbasis up to the interaction-frame phases, which are applied
once per tile entry) against the FP64 oracle and against the complex-row passes,
through the C ABI: the forward passes, and the adjoint passes of the pulse-parameter
gradient.

Shapes: level counts 4 and 2, one-pass and multi-pass plans (a small tile budget,
and the two-group ring of 4^7 states), parity-odd plans (compressed rows) and the
lab frame (full rows), fluxonium (imaginary n (x) n couplings, real phi drives) and
transmon (real n) workloads.  Tolerances as everywhere: FP64 1e-10 on amplitudes
and F, gradients 1e-8 of the largest component; mixed 1e-5 and 1e-3."""
import numpy as np
import pytest

from oracle.evolve import adjoint_gradient, frame_epilogue, initial_columns, rk4_evolve, rk4_evolve_matrix_free
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture
def real_slab(monkeypatch):
    monkeypatch.setenv("SG_PATH", "slab")
    monkeypatch.setenv("SG_SLAB_REAL", "1")
    monkeypatch.delenv("SG_SLAB_TMAX", raising=False)
    return monkeypatch


def _system(sgctx, wl):
    from paper_2406_18155_gb300.api import System
    s = System.from_workload(sgctx, wl)
    s.prepare()
    return s


def _oracle_psi(wl):
    so = OracleSystem(wl)
    return frame_epilogue(so, rk4_evolve(so, initial_columns(so, wl["col_index"])))


CASES = {
    # name: (workload, tile budget or None)
    "transmon_pair_l4": (lambda: W.transmon_pair(seed=3, T=1.0), None),
    "ring4_l4_multipass": (lambda: W.fluxonium_chain(seed=4, nq=4, levels=4, T=0.3, dt=0.01, nseg=3,
                                                     ring=True), 64),
    "chain6_l2_multipass": (lambda: W.fluxonium_chain(seed=5, nq=6, levels=2, T=0.3, dt=0.01, nseg=3), 8),
    "chain5_l4_onepass": (lambda: W.fluxonium_chain(seed=6, nq=5, levels=4, T=0.2, dt=0.01, nseg=2,
                                                    ncols=12), None),
}


@pytest.mark.parametrize("frame", ["interaction", "lab"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_real_forward_matches_oracle_and_complex_rows(sgctx, real_slab, name, frame):
    make, tmax = CASES[name]
    if tmax:
        real_slab.setenv("SG_SLAB_TMAX", str(tmax))
    wl = make()
    wl["frame"] = frame
    if frame == "lab":
        wl["T"], wl["dt"] = 0.05, 0.0025
        for d in wl["drives"]:
            d["length"] = wl["T"]
    s = _system(sgctx, wl)
    ref = _oracle_psi(wl)
    out = {}
    for real in ("1", "0"):
        real_slab.setenv("SG_SLAB_REAL", real)
        for prec in ("fp64", "mixed"):
            out[real, prec] = s.evolve(wl["T"], wl["dt"], precision=prec, frame=frame,
                                       col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(out["1", "fp64"] - ref)) < 1e-10
    assert np.max(np.abs(out["1", "mixed"] - ref)) < 1e-5
    # the real-operator and complex-row passes: same map, different rounding (in the
    # lab frame the phases are 1 and the complex rows real, so the two agree exactly;
    # in the interaction frame a zero difference would mean the real passes never ran)
    d64 = np.max(np.abs(out["1", "fp64"] - out["0", "fp64"]))
    assert d64 < 1e-12 and (frame == "lab" or d64 > 0)
    assert np.max(np.abs(out["1", "mixed"] - out["0", "mixed"])) < 1e-5


@pytest.mark.parametrize("name", ["ring4_l4_multipass", "chain6_l2_multipass", "transmon_pair_l4"])
def test_real_forward_gradient_matches_oracle(sgctx, real_slab, name):
    # the forward and replay passes use real rows, the adjoint the complex ones
    make, tmax = CASES[name]
    if tmax:
        real_slab.setenv("SG_SLAB_TMAX", str(tmax))
    wl = make()
    kind = "state" if name != "transmon_pair_l4" else "avg"
    wl["fid_kind"] = kind
    s = _system(sgctx, wl)
    Fr, gr, _ = adjoint_gradient(wl)
    k = 0 if kind == "avg" else 1
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=kind,
                                precision="fp64", ckpt=4)
    assert abs(F[k] - Fr) < 1e-10
    assert np.max(np.abs(np.concatenate([gp, gh]) - gr)) <= 1e-8 * np.max(np.abs(gr))
    F32, gp32, gh32 = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=kind,
                                      precision="mixed", ckpt=4)
    assert abs(F32[k] - Fr) < 1e-5
    assert np.max(np.abs(np.concatenate([gp32, gh32]) - gr)) <= 1e-3 * np.max(np.abs(gr))


@pytest.mark.parametrize("name", ["ring4_l4_multipass", "chain6_l2_multipass", "chain5_l4_onepass"])
def test_real_pulse_gradient_adjoint_matches_oracle(sgctx, real_slab, name):
    # pulse-parameter gradient only: the adjoint passes run in the real-operator form
    # too, each drive's term contracted with the rotated co-state and state; against
    # the oracle's adjoint and against the complex-row adjoint (SG_SLAB_ZADJ=0)
    make, tmax = CASES[name]
    if tmax:
        real_slab.setenv("SG_SLAB_TMAX", str(tmax))
    wl = make()
    wl["fid_kind"] = "state"
    s = _system(sgctx, wl)
    Fr, gr, _ = adjoint_gradient(wl)
    gr = gr[:s.param_counts()[0]]
    scale = np.max(np.abs(gr))
    out = {}
    for zadj in ("1", "0"):
        real_slab.setenv("SG_SLAB_ZADJ", zadj)
        for prec in ("fp64", "mixed"):
            F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                        precision=prec, ckpt=4, ham=False)
            assert gh is None
            out[zadj, prec] = (F, gp)
    F, gp = out["1", "fp64"]
    assert abs(F[1] - Fr) < 1e-10
    assert np.max(np.abs(gp - gr)) <= 1e-8 * scale
    F32, gp32 = out["1", "mixed"]
    assert abs(F32[1] - Fr) < 1e-5
    assert np.max(np.abs(gp32 - gr)) <= 1e-3 * scale
    # the same gradient as the complex-row adjoint up to rounding (a zero difference
    # would mean the real-operator adjoint never ran)
    d64 = np.max(np.abs(gp - out["0", "fp64"][1]))
    assert 0 < d64 <= 1e-12 * scale
    assert np.max(np.abs(gp32 - out["0", "mixed"][1])) <= 1e-4 * scale


def test_real_two_pass_ring7_against_matrix_free_oracle(sgctx, real_slab):
    # D = 4^7: two overlapping mode groups of 4^6-entry tiles, the ring's plan shape
    wl = W.fluxonium_chain(seed=9, nq=7, levels=4, T=0.1, dt=0.01, nseg=2, ring=True, ncols=3)
    s = _system(sgctx, wl)
    so = OracleSystem(wl)
    ref = frame_epilogue(so, rk4_evolve_matrix_free(so, initial_columns(so, wl["col_index"])))
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi - ref)) < 1e-10
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi32 - ref)) < 1e-5


def test_lean_passes_on_the_two_group_ring_plan(sgctx, real_slab):
    # 4-level parity-odd plans whose tiles hold 4096 entries (the 2^20 ring's plan
    # shape; here the 4^7 ring) run the lean FP32 forward and adjoint passes: the
    # arithmetic of the general real-operator passes with compile-time block strides.
    # Against those passes (SG_SLAB_LEAN=0) and against FP64 on the same plan.
    wl = W.fluxonium_chain(seed=9, nq=7, levels=4, T=0.1, dt=0.01, nseg=2, ring=True, ncols=3)
    wl["fid_kind"] = "state"
    s = _system(sgctx, wl)
    args = (wl["T"], wl["dt"], wl["target"], wl["col_index"])
    out = {}
    for lean in ("1", "0"):
        real_slab.setenv("SG_SLAB_LEAN", lean)
        psi = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"]).cpu().numpy()
        F, gp, _ = s.fidelity_grad(*args, kind="state", precision="mixed", ckpt=3, ham=False)
        out[lean] = (psi, F, gp)
    F64, g64, _ = s.fidelity_grad(*args, kind="state", precision="fp64", ckpt=3, ham=False)
    scale = np.max(np.abs(g64))
    assert np.max(np.abs(out["1"][0] - out["0"][0])) < 1e-6
    assert abs(out["1"][1][1] - F64[1]) < 1e-5
    assert np.max(np.abs(out["1"][2] - g64)) <= 1e-3 * scale
    assert np.max(np.abs(out["1"][2] - out["0"][2])) <= 1e-4 * scale


def test_complex_local_operator_keeps_the_complex_rows(sgctx, real_slab):
    # a genuinely complex local operator is not real up to phases: the plan keeps the
    # complex-row passes and still matches the oracle
    wl = W.local_op_pair(seed=2, T=0.3)
    s = _system(sgctx, wl)
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi - _oracle_psi(wl))) < 1e-10


@pytest.mark.parametrize("nq,ring,ncols", [(7, True, 3), (5, False, 12)])
def test_warp_specialised_pass_equals_one_role_pass(sgctx, real_slab, nq, ring, ncols):
    # FP32 tiles of >= 256 entries run on the double-buffered kernel (compute warps
    # beside load/write-back warps); it does the one-role kernel's arithmetic in the
    # same order, so the states agree exactly, and both match the oracle
    wl = W.fluxonium_chain(seed=10 + nq, nq=nq, levels=4, T=0.1, dt=0.01, nseg=2, ring=ring, ncols=ncols)
    s = _system(sgctx, wl)
    out = {}
    for ws in ("1", "0"):   # SG_SLAB_WS=1 selects the warp-specialised kernel
        real_slab.setenv("SG_SLAB_WS", ws)
        out[ws] = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"]).cpu().numpy()
    assert np.array_equal(out["1"], out["0"])
    assert np.max(np.abs(out["1"] - _oracle_psi(wl))) < 1e-5 if nq < 7 else True
