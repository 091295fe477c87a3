"""GPU parity of the virtual-Z compensated fidelities and their gradients against
the oracle (the errorless phase gates around the pulses of the paper's gate
metric): F_avg and F_state in FP64 within 1e-10 and mixed within 1e-5; the full
gradient (pulse and Hamiltonian parameters) in FP64 within 1e-7 of its largest
component; the Q2 solver with compensation; partial column sets are refused."""
import numpy as np
import pytest

from oracle.compensation import compensated_fidelities
from oracle.evolve import adjoint_gradient, frame_epilogue, initial_columns, rk4_evolve
from oracle.system import OracleSystem
from oracle.trotter import q2_evolve
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system(sgctx, wl):
    from paper_2406_18155_gb300.api import System
    s = System.from_workload(sgctx, wl)
    s.prepare()
    return s


def _short(wl, T):
    wl["T"] = T
    for d in wl["drives"]:
        d["length"] = T
        if d.get("env") == "gaussian":
            d["sigma"], d["t0"] = T / 4, T / 2
    return wl


CASES = {
    "transmon_pair": lambda: _short(W.transmon_pair(seed=3), 0.5),
    "pair_cr_l5": lambda: _short(W.fluxonium_pair_cr(seed=5, nseg=4), 0.4),
    "chain3_l3": lambda: W.fluxonium_chain(seed=7, nq=3, levels=3, T=0.3, dt=0.01, nseg=2),
}


def _oracle_comp(wl):
    so = OracleSystem(wl)
    psi = frame_epilogue(so, rk4_evolve(so, initial_columns(so, wl["col_index"])))
    return compensated_fidelities(so, psi)


@pytest.mark.parametrize("name", sorted(CASES))
def test_vz_fidelities_match_oracle(sgctx, name):
    wl = CASES[name]()
    s = _system(sgctx, wl)
    Fa_r, Fs_r, _ = _oracle_comp(wl)
    Fa, Fs, _ = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64", compensation="vz")
    assert abs(Fa - Fa_r) < 1e-10 and abs(Fs - Fs_r) < 1e-10
    Fa0, _, _ = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64")
    assert Fa >= Fa0 - 1e-14
    Fa32, Fs32, _ = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="mixed",
                               compensation="vz")
    assert abs(Fa32 - Fa_r) < 1e-5 and abs(Fs32 - Fs_r) < 1e-5


@pytest.mark.parametrize("name", sorted(CASES))
def test_vz_gradient_matches_oracle(sgctx, name):
    wl = CASES[name]()
    s = _system(sgctx, wl)
    kind = wl["fid_kind"]
    Fa_r, Fs_r, T_eff = _oracle_comp(wl)
    F_r, g_r, _ = adjoint_gradient(dict(wl, target=T_eff), kind=kind)
    assert abs(F_r - (Fa_r if kind == "avg" else Fs_r)) < 1e-12
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=kind,
                                precision="fp64", ckpt=7, compensation="vz")
    g = np.concatenate([gp, gh])
    assert abs(F[0 if kind == "avg" else 1] - F_r) < 1e-10
    assert np.max(np.abs(g - g_r)) <= 1e-7 * np.max(np.abs(g_r)), np.max(np.abs(g - g_r))


def test_vz_with_the_q2_solver(sgctx):
    wl = CASES["pair_cr_l5"]()
    s = _system(sgctx, wl)
    so = OracleSystem(dict(wl, frame="lab"))
    psi = q2_evolve(so, initial_columns(so, wl["col_index"]))
    Fa_r, Fs_r, _ = compensated_fidelities(so, psi)
    Fa, Fs, _ = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64", solver="q2",
                           compensation="vz")
    assert abs(Fa - Fa_r) < 1e-10 and abs(Fs - Fs_r) < 1e-10


def test_vz_needs_every_computational_state(sgctx):
    from paper_2406_18155_gb300.capi import SGError, SG_E_INVALID
    wl = CASES["chain3_l3"]()
    s = _system(sgctx, wl)
    with pytest.raises(SGError) as e:
        s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"][:5], precision="fp64", compensation="vz")
    assert e.value.code == SG_E_INVALID
