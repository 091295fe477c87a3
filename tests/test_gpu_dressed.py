"""GPU parity of the dressed-basis gate metric (App. C: the computational states
are the idle Hamiltonian's eigenstates) against the oracle: F_avg and F_state in
FP64 within 1e-10 and mixed within 1e-5, the pulse gradient in FP64 within 1e-8
and mixed within 1e-3 of its largest component; unsupported requests refused."""
import numpy as np
import pytest

from oracle.dressed import dressed_fidelities, dressed_pulse_gradient
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


def _transmon_pair():
    wl = _short(W.transmon_pair(seed=3), 0.5)
    wl["col_index"] = W.comp_states([m["levels"] for m in wl["modes"]])
    return wl


CASES = {
    "transmon_pair": _transmon_pair,
    "pair_cr_l5": lambda: _short(W.fluxonium_pair_cr(seed=5, nseg=4), 0.4),
    "chain3_l3": lambda: W.fluxonium_chain(seed=7, nq=3, levels=3, T=0.3, dt=0.01, nseg=2),
    "chain4_l3": lambda: W.fluxonium_chain(seed=9, nq=4, levels=3, T=0.2, dt=0.01, nseg=2),   # D = 81
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_dressed_fidelities_match_oracle(sgctx, name):
    wl = CASES[name]()
    s = _system(sgctx, wl)
    Fa_r, Fs_r, Uc_r = dressed_fidelities(wl)
    Fa, Fs, Uc = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64", basis="dressed")
    assert abs(Fa - Fa_r) < 1e-10 and abs(Fs - Fs_r) < 1e-10
    assert np.max(np.abs(Uc - Uc_r)) < 1e-10
    Fa32, Fs32, _ = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="mixed",
                               basis="dressed")
    assert abs(Fa32 - Fa_r) < 1e-5 and abs(Fs32 - Fs_r) < 1e-5


@pytest.mark.parametrize("name", sorted(CASES))
def test_dressed_pulse_gradient_matches_oracle(sgctx, name):
    wl = CASES[name]()
    s = _system(sgctx, wl)
    kind = wl["fid_kind"]
    F_r, g_r = dressed_pulse_gradient(wl, kind)
    scale = np.max(np.abs(g_r))
    for prec, tol_F, tol_g in (("fp64", 1e-10, 1e-8), ("mixed", 1e-5, 1e-3)):
        F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=kind, precision=prec,
                                    ham=False, ckpt=7, basis="dressed")
        assert gh is None
        assert abs(F[0 if kind == "avg" else 1] - F_r) < tol_F
        assert np.max(np.abs(gp - g_r)) <= tol_g * scale, (prec, np.max(np.abs(gp - g_r)), scale)


def test_dressed_requests_that_are_refused(sgctx):
    from paper_2406_18155_gb300.capi import SGError, SG_E_INVALID, SG_E_UNSUPPORTED
    wl = CASES["pair_cr_l5"]()
    s = _system(sgctx, wl)
    with pytest.raises(SGError) as e:                     # Hamiltonian gradient
        s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg", precision="fp64",
                        basis="dressed")
    assert e.value.code == SG_E_UNSUPPORTED
    with pytest.raises(SGError) as e:                     # a column that is not a computational state
        s.fidelity(wl["T"], wl["dt"], wl["target"], list(wl["col_index"]) + [2], precision="fp64",
                   basis="dressed")
    assert e.value.code == SG_E_INVALID
    big = W.fluxonium_chain(seed=8, nq=5, levels=5, T=0.2, dt=0.01, nseg=2)          # D = 3125 > 1024
    s2 = _system(sgctx, big)
    with pytest.raises(SGError) as e:
        s2.fidelity(big["T"], big["dt"], big["target"], big["col_index"], precision="fp64", basis="dressed")
    assert e.value.code == SG_E_INVALID


def _large(nq, levels, T):
    wl = W.fluxonium_chain(seed=8, nq=nq, levels=levels, T=T, dt=0.01, nseg=2)
    wl["fid_kind"] = "avg"                   # F_state of this target is ~1e-12
    return wl


@pytest.mark.parametrize("nq,levels,T", [(4, 5, 0.1), (5, 4, 0.06)])
def test_dressed_beyond_one_block(sgctx, nq, levels, T):
    """D = 625 and D = 1024 (the largest): the idle Hamiltonian is diagonalised by the
    Jacobi rounds over the whole GPU instead of one block."""
    wl = _large(nq, levels, T)
    s = _system(sgctx, wl)
    Fa_r, Fs_r, Uc_r = dressed_fidelities(wl)
    Fa, Fs, Uc = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64", basis="dressed")
    assert abs(Fa - Fa_r) < 1e-10 and abs(Fs - Fs_r) < 1e-10
    assert np.max(np.abs(Uc - Uc_r)) < 1e-10


def test_dressed_gradient_beyond_one_block(sgctx):
    wl = _large(4, 5, 0.1)
    s = _system(sgctx, wl)
    F_r, g_r = dressed_pulse_gradient(wl, "avg")
    scale = np.max(np.abs(g_r))
    for prec, tol_F, tol_g in (("fp64", 1e-10, 1e-8), ("mixed", 1e-5, 1e-3)):
        F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg", precision=prec,
                                    ham=False, ckpt=7, basis="dressed")
        assert gh is None
        assert abs(F[0] - F_r) < tol_F
        assert np.max(np.abs(gp - g_r)) <= tol_g * scale, (prec, np.max(np.abs(gp - g_r)), scale)


def test_dressed_basis_with_the_q2_solver(sgctx):
    from oracle.dressed import dressed_vectors
    from oracle.evolve import block_fidelity_and_costate, comp_map
    from oracle.system import OracleSystem
    from oracle.trotter import q2_evolve
    wl = CASES["pair_cr_l5"]()
    s = _system(sgctx, wl)
    so = OracleSystem(dict(wl, frame="lab"))
    Vc, _ = dressed_vectors(so)
    _, cols = comp_map(so)
    Uc_r = Vc.conj().T @ q2_evolve(so, Vc[:, cols])
    T = np.asarray(wl["target"], dtype=complex)
    Fa_r, _ = block_fidelity_and_costate(T, Uc_r, cols, "avg")
    Fs_r, _ = block_fidelity_and_costate(T, Uc_r, cols, "state")
    Fa, Fs, Uc = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64", solver="q2",
                            basis="dressed")
    assert abs(Fa - Fa_r) < 1e-10 and abs(Fs - Fs_r) < 1e-10
    assert np.max(np.abs(Uc - Uc_r)) < 1e-10
