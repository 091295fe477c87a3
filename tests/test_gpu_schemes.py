"""GPU parity of the qubit architectures beyond a plain chain (the multipath
coupling of Sec. 3.1 and the coupler schemes of Sec. 4: transmon qubits with a
transmon coupler, fluxoniums with a transmon coupler) against the FP64 oracle:
states, fidelities and gradients, FP64 1e-10 / 1e-8 of the largest gradient
component, mixed 1e-5 / 1e-3."""
import numpy as np
import pytest

from oracle.evolve import initial_columns, rk4_evolve, frame_epilogue, fidelities, adjoint_gradient
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system(sgctx, wl):
    from paper_2406_18155_gb300.api import System
    s = System.from_workload(sgctx, wl)
    s.prepare()
    return s


def _short(wl, T=0.3):
    wl["T"] = T
    for d in wl["drives"]:
        d["length"] = T
    return wl


SCHEMES = {
    "multipath_l4": lambda: _short(W.fluxonium_pair_multipath(seed=4, levels=4, nseg=3)),
    "multipath_l5": lambda: _short(W.fluxonium_pair_multipath(seed=5, levels=5, nseg=3)),
    "ttt_l4": lambda: _short(W.coupler_scheme(seed=6, kind="ttt", nseg=3)),
    "ftf_l4": lambda: _short(W.coupler_scheme(seed=7, kind="ftf", nseg=3)),
    "ftf_l4_3_4": lambda: _short(W.coupler_scheme(seed=8, kind="ftf", nseg=3, levels=(4, 3, 4))),
    "local_ops_l4": lambda: _short(W.local_op_pair(seed=9, levels=4, nseg=3)),
    "local_ops_l3": lambda: _short(W.local_op_pair(seed=10, levels=3, nseg=3)),
}


@pytest.fixture
def default_path(monkeypatch):
    monkeypatch.delenv("SG_PATH", raising=False)
    monkeypatch.delenv("SG_SLAB_TMAX", raising=False)


@pytest.mark.parametrize("name", sorted(SCHEMES))
def test_scheme_states_and_fidelity(sgctx, default_path, name):
    wl = SCHEMES[name]()
    s = _system(sgctx, wl)
    so = OracleSystem(wl)
    ref = frame_epilogue(so, rk4_evolve(so, initial_columns(so, wl["col_index"])))
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi - ref)) < 1e-10
    Fa_r, Fs_r, Uc_r = fidelities(so, ref)
    Fa, Fs, Uc = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64")
    assert Uc.shape == (4, len(wl["col_index"]))            # two qubit modes (+ coupler in level 0)
    assert abs(Fa - Fa_r) < 1e-10 and abs(Fs - Fs_r) < 1e-10
    assert np.max(np.abs(Uc - Uc_r)) < 1e-10
    Fa32, _, _ = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="mixed")
    assert abs(Fa32 - Fa_r) < 1e-5


@pytest.mark.parametrize("name", sorted(SCHEMES))
def test_scheme_gradient(sgctx, default_path, name):
    wl = SCHEMES[name]()
    s = _system(sgctx, wl)
    Fr, gr, _ = adjoint_gradient(wl)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg",
                                precision="fp64", ckpt=7)
    assert abs(F[0] - Fr) < 1e-10
    assert np.max(np.abs(np.concatenate([gp, gh]) - gr)) <= 1e-8 * np.max(np.abs(gr))
    F32, gp32, gh32 = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg",
                                      precision="mixed")
    assert abs(F32[0] - Fr) < 1e-5
    assert np.max(np.abs(np.concatenate([gp32, gh32]) - gr)) <= 1e-3 * np.max(np.abs(gr))


def test_coupler_request_through_the_server(sgctx, default_path):
    # no col_index: the server evolves every computational state (coupler in level 0)
    from paper_2406_18155_gb300.api import Server
    wl = SCHEMES["ftf_l4"]()
    alone = _system(sgctx, wl).fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                             kind="avg", precision="mixed")
    srv = Server(sgctx, mem_budget_bytes=1 << 30, max_slots=2)
    r = srv.wait(srv.submit(_system(sgctx, wl), wl["T"], wl["dt"], wl["target"], None, kind="avg"))
    srv.close()
    assert r["status"] == 0, r["error"]
    assert abs(r["F"][0] - alone[0][0]) <= 1e-12
    assert np.max(np.abs(r["grad_pulse"] - alone[1])) <= 1e-12 * max(1.0, np.max(np.abs(alone[1])))


@pytest.mark.parametrize("path", ["gather", "slab"])
def test_local_ops_on_the_other_kernel_families(sgctx, monkeypatch, path):
    monkeypatch.setenv("SG_PATH", path)
    wl = SCHEMES["local_ops_l4"]()
    s = _system(sgctx, wl)
    Fr, gr, _ = adjoint_gradient(wl)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg",
                                precision="fp64", ckpt=5)
    assert abs(F[0] - Fr) < 1e-10
    assert np.max(np.abs(np.concatenate([gp, gh]) - gr)) <= 1e-8 * np.max(np.abs(gr))


def test_local_op_validation(sgctx):
    from paper_2406_18155_gb300.api import System
    from paper_2406_18155_gb300.capi import SGError, SG_E_INVALID, SG_E_UNSUPPORTED
    s = System(sgctx)
    m = s.add_fluxonium(4 * 6.283, 6.283, 6.283, np.pi, 50, 3)
    bad = np.zeros((3, 3), complex)
    bad[0, 1] = 1.0                                         # not Hermitian
    with pytest.raises(SGError) as e:
        s.add_local_op(m, bad)
    assert e.value.code == SG_E_INVALID
    with pytest.raises(SGError):
        s.add_local_op(m + 1, np.eye(3))                    # no such mode
    for k in range(6):
        assert s.add_local_op(m, np.eye(3) * k) == 2 + k
    with pytest.raises(SGError) as e:
        s.add_local_op(m, np.eye(3))
    assert e.value.code == SG_E_UNSUPPORTED
    with pytest.raises(SGError):
        s.add_coupling(m, 9, m, 0, 0.1)                     # unknown operator id
