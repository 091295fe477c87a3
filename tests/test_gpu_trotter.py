"""GPU parity of the Suzuki-Trotter solvers (Sec. 2.3, App. A: Q1, Q2, Q4, Q4j) against
the oracle's: lab-frame states and fidelities, FP64 within 1e-10, FP32 factors and
state within 1e-5 on short evolutions; the pulse-parameter gradient of Q2, Q4 and
Q4j (discrete adjoint of the product of local factors, Sec. 2.5) against the
oracle's adjoint, FP64 within 1e-9 and FP32 within 2e-4 of the largest component;
unsupported requests are rejected."""
import numpy as np
import pytest

from oracle.evolve import initial_columns, fidelities
from oracle.system import OracleSystem
from oracle.trotter import q2_evolve, q2_pulse_gradient
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
        if d.get("env") == "gaussian":
            d["sigma"], d["t0"] = T / 4, T / 2
    return wl


CASES = {
    "transmon_pair": lambda: _short(W.transmon_pair(seed=2)),                  # 2 modes: one pair factor
    "chain3_l3": lambda: _short(W.fluxonium_chain(seed=3, nq=3, levels=3, nseg=3)),   # odd: last mode alone
    "ring4_l3": lambda: _short(W.fluxonium_chain(seed=4, nq=4, levels=3, nseg=3, ring=True)),
    "pair_cr_l5": lambda: _short(W.fluxonium_pair_cr(seed=5, nseg=4)),
    "ftf_l4": lambda: _short(W.coupler_scheme(seed=6, kind="ftf", nseg=3)),
    "multipath_l4": lambda: _short(W.fluxonium_pair_multipath(seed=7, levels=4, nseg=3)),
    "local_ops_l3": lambda: _short(W.local_op_pair(seed=8, levels=3, nseg=3)),
}


@pytest.fixture
def default_path(monkeypatch):
    monkeypatch.delenv("SG_PATH", raising=False)
    monkeypatch.delenv("SG_SLAB_TMAX", raising=False)


@pytest.mark.parametrize("name", sorted(CASES))
def test_q2_matches_oracle(sgctx, default_path, name):
    wl = CASES[name]()
    s = _system(sgctx, wl)
    so = OracleSystem(dict(wl, frame="lab"))
    ref = q2_evolve(so, initial_columns(so, wl["col_index"]))
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"], solver="q2").cpu().numpy()
    assert np.max(np.abs(psi - ref)) < 1e-10
    Fa_r, Fs_r, Uc_r = fidelities(so, ref)
    Fa, Fs, Uc = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64", solver="q2")
    assert abs(Fs - Fs_r) < 1e-10 and np.max(np.abs(Uc - Uc_r)) < 1e-10
    assert (np.isnan(Fa) and np.isnan(Fa_r)) or abs(Fa - Fa_r) < 1e-10
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"], solver="q2").cpu().numpy()
    assert np.max(np.abs(psi32 - ref)) < 1e-5


@pytest.mark.parametrize("name", ["transmon_pair", "chain3_l3", "ring4_l3", "multipath_l4"])
def test_q1_matches_oracle(sgctx, default_path, name):
    # the first-order product: every term once per step over the full step
    wl = CASES[name]()
    s = _system(sgctx, wl)
    so = OracleSystem(dict(wl, frame="lab"))
    ref = q2_evolve(so, initial_columns(so, wl["col_index"]), scheme="q1")
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"], solver="q1").cpu().numpy()
    assert np.max(np.abs(psi - ref)) < 1e-10
    Fa_r, Fs_r, Uc_r = fidelities(so, ref)
    Fa, Fs, Uc = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64", solver="q1")
    assert abs(Fs - Fs_r) < 1e-10 and np.max(np.abs(Uc - Uc_r)) < 1e-10
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"], solver="q1").cpu().numpy()
    assert np.max(np.abs(psi32 - ref)) < 1e-5
    # Q1 and Q2 are different products of the same factors
    q2 = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"], solver="q2").cpu().numpy()
    assert np.max(np.abs(q2 - psi)) > 1e-8


@pytest.mark.parametrize("name", ["transmon_pair", "ring4_l3", "pair_cr_l5", "local_ops_l3"])
def test_q1_pulse_gradient_matches_oracle(sgctx, default_path, name):
    """The first-order product's pulse gradient: the couplings pulled back in reverse
    order by their full-step factors, then the step's full-step 1-body factors with the
    Frechet derivatives along dt (not dt/2), against the oracle's adjoint."""
    wl = CASES[name]()
    s = _system(sgctx, wl)
    F_r, g_r = q2_pulse_gradient(wl, scheme="q1")
    scale = max(1.0, np.max(np.abs(g_r)))
    for prec, tol_F, tol_g in (("fp64", 1e-10, 1e-9), ("mixed", 1e-5, 2e-4)):
        F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=wl["fid_kind"],
                                    precision=prec, ham=False, solver="q1")
        assert gh is None and gp.shape == g_r.shape
        Fk = F[0] if wl["fid_kind"] == "avg" else F[1]
        assert abs(Fk - F_r) < tol_F, (prec, Fk, F_r)
        assert np.max(np.abs(gp - g_r)) < tol_g * scale, (prec, np.max(np.abs(gp - g_r)), scale)
    # not Q2's gradient: the two products differ at this step
    _, g2 = q2_pulse_gradient(wl, scheme="q2")
    assert np.max(np.abs(g2 - g_r)) > 1e-6 * np.max(np.abs(g_r))


@pytest.mark.parametrize("scheme", ["q1", "q2", "q4", "q4j"])
def test_tiled_products_match_oracle(sgctx, monkeypatch, scheme):
    # beyond the on-chip kernels the products run on the tiles of a two-pass plan: the
    # 4^7 ring (a 4096-entry and a 64-entry group) and, forced by a small tile budget, a
    # 3-level chain of 5 modes
    monkeypatch.delenv("SG_PATH", raising=False)
    monkeypatch.delenv("SG_SLAB_TMAX", raising=False)
    ring = _short(W.fluxonium_chain(seed=11, nq=7, levels=4, nseg=2, ring=True, ncols=3), T=0.1)
    chain = _short(W.fluxonium_chain(seed=12, nq=5, levels=3, nseg=3, ncols=6), T=0.2)
    for wl, env in ((ring, {}), (chain, {"SG_PATH": "slab", "SG_SLAB_TMAX": "27"})):
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        s = _system(sgctx, wl)
        so = OracleSystem(dict(wl, frame="lab"))
        ref = q2_evolve(so, initial_columns(so, wl["col_index"]), scheme=scheme)
        psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"], solver=scheme).cpu().numpy()
        assert np.max(np.abs(psi - ref)) < 1e-10
        psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"],
                         solver=scheme).cpu().numpy()
        assert np.max(np.abs(psi32 - ref)) < 1e-5
        Fa, Fs, Uc = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64", solver=scheme)
        _, Fs_r, Uc_r = fidelities(so, ref)
        assert abs(Fs - Fs_r) < 1e-10 and np.max(np.abs(Uc - Uc_r)) < 1e-10
        for k in env:
            monkeypatch.delenv(k)


def _phase_target(wl):
    """A diagonal target carrying the phases of the evolved columns' diagonal entries, so
    that F_state is near 1 and its gradient is not negligible."""
    from oracle.evolve import comp_map
    so = OracleSystem(dict(wl, frame="lab"))
    psi = q2_evolve(so, initial_columns(so, wl["col_index"]), scheme="q2")
    comp, cols = comp_map(so)
    T = np.eye(len(comp), dtype=complex)
    for s_, j in enumerate(cols):
        if j >= 0:
            u = psi[comp[j], s_]
            T[j, j] = u / abs(u)
    wl = dict(wl, target=T.tolist(), fid_kind="state")
    return wl


@pytest.mark.parametrize("scheme,fuse", [("q1", "1"), ("q2", "1"), ("q4", "1"), ("q4j", "1"), ("q2", "0"),
                                         ("q4j", "0")])
def test_tiled_pulse_gradient_matches_oracle(sgctx, monkeypatch, scheme, fuse):
    """The pulse gradient on the tiles of a two-pass plan: the final states and co-states
    pulled back pass by pass through the inverse and adjoint factors, a cross-density
    contraction after every 1-body half step, against the oracle's adjoint (the 4^7 ring
    and the forced two-pass 3-level chain); one fused launch per pass and sub-step, and
    (SG_Q2_FUSE=0) the segmented pull-back and contraction launches."""
    monkeypatch.delenv("SG_PATH", raising=False)
    monkeypatch.delenv("SG_SLAB_TMAX", raising=False)
    monkeypatch.setenv("SG_Q2_FUSE", fuse)
    ring = _short(W.fluxonium_chain(seed=11, nq=7, levels=4, nseg=2, ring=True, ncols=3), T=0.05)
    chain = _short(W.fluxonium_chain(seed=12, nq=5, levels=3, nseg=3, ncols=6), T=0.1)
    for wl, env in ((ring, {}), (chain, {"SG_PATH": "slab", "SG_SLAB_TMAX": "27"})):
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        wl = _phase_target(wl)
        s = _system(sgctx, wl)
        F_r, g_r = q2_pulse_gradient(wl, kind="state", scheme=scheme)
        assert F_r > 0.5
        scale = np.max(np.abs(g_r))
        for prec, tol_F, tol_g in (("fp64", 1e-10, 1e-9), ("mixed", 1e-5, 2e-4)):
            F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                        precision=prec, ham=False, solver=scheme)
            assert gh is None and gp.shape == g_r.shape
            assert abs(F[1] - F_r) < tol_F, (prec, F[1], F_r)
            assert np.max(np.abs(gp - g_r)) < tol_g * scale, (prec, np.max(np.abs(gp - g_r)), scale)
        for k in env:
            monkeypatch.delenv(k)


def test_q2_rejects_what_it_does_not_run(sgctx, default_path):
    from paper_2406_18155_gb300.capi import SGError, SG_E_UNSUPPORTED
    wl = CASES["transmon_pair"]()
    s = _system(sgctx, wl)
    with pytest.raises(SGError) as e:                       # Hamiltonian gradient: RK4 only
        from paper_2406_18155_gb300.api import evolve_opts
        import ctypes as C
        from paper_2406_18155_gb300.capi import lib
        o, keep = evolve_opts(wl["T"], wl["dt"], "fp64", "interaction", wl["col_index"], solver="q2")
        tg = np.ascontiguousarray(np.asarray(wl["target"], complex).view(np.float64).reshape(-1))
        F, gp, gh = np.zeros(2), np.zeros(8), np.zeros(16)
        p = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        s._chk(lib().sg_fidelity_grad(s.h, C.byref(o), p(tg), 0, p(F), p(gp), p(gh), 0))
    assert e.value.code == SG_E_UNSUPPORTED
    mixed_levels = W.coupler_scheme(seed=9, kind="ftf", nseg=3, levels=(4, 3, 4))
    s2 = _system(sgctx, _short(mixed_levels))
    with pytest.raises(SGError) as e:                       # unequal level counts: not on-chip
        s2.evolve(0.3, 0.01, precision="fp64", col_index=mixed_levels["col_index"], solver="q2")
    assert e.value.code == SG_E_UNSUPPORTED


GRAD_CASES = ["transmon_pair", "chain3_l3", "ring4_l3", "pair_cr_l5", "ftf_l4", "local_ops_l3"]


@pytest.mark.parametrize("name", GRAD_CASES)
def test_q2_pulse_gradient_matches_oracle(sgctx, default_path, name):
    wl = CASES[name]()
    s = _system(sgctx, wl)
    F_r, g_r = q2_pulse_gradient(wl)
    scale = max(1.0, np.max(np.abs(g_r)))
    for prec, tol_F, tol_g in (("fp64", 1e-10, 1e-9), ("mixed", 1e-5, 2e-4)):
        F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=wl["fid_kind"],
                                    precision=prec, ham=False, solver="q2")
        assert gh is None and gp.shape == g_r.shape
        Fk = F[0] if wl["fid_kind"] == "avg" else F[1]
        assert abs(Fk - F_r) < tol_F, (prec, Fk, F_r)
        assert np.max(np.abs(gp - g_r)) < tol_g * scale, (prec, np.max(np.abs(gp - g_r)), scale)


def test_q2_pulse_gradient_longer_evolution(sgctx, default_path):
    """A CR pulse of 4 ns (N = 400 steps, 5 levels per fluxonium, 6 PWC segments):
    the reconstruction of the states by inverse factors stays within the bars."""
    wl = _short(W.fluxonium_pair_cr(seed=11, nseg=6), T=4.0)
    s = _system(sgctx, wl)
    F_r, g_r = q2_pulse_gradient(wl)
    scale = max(1.0, np.max(np.abs(g_r)))
    for prec, tol in (("fp64", 1e-9), ("mixed", 1e-3)):
        F, gp, _ = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=wl["fid_kind"],
                                   precision=prec, ham=False, solver="q2")
        assert np.max(np.abs(gp - g_r)) < tol * scale, (prec, np.max(np.abs(gp - g_r)), scale)


@pytest.mark.parametrize("scheme", ["q4", "q4j"])
@pytest.mark.parametrize("name", ["transmon_pair", "chain3_l3", "pair_cr_l5", "ftf_l4"])
def test_fourth_order_products_match_oracle(sgctx, default_path, name, scheme):
    wl = CASES[name]()
    s = _system(sgctx, wl)
    so = OracleSystem(dict(wl, frame="lab"))
    ref = q2_evolve(so, initial_columns(so, wl["col_index"]), scheme=scheme)
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"], solver=scheme).cpu().numpy()
    assert np.max(np.abs(psi - ref)) < 1e-10
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"], solver=scheme).cpu().numpy()
    assert np.max(np.abs(psi32 - ref)) < 1e-5


@pytest.mark.parametrize("scheme", ["q4", "q4j"])
@pytest.mark.parametrize("name", ["transmon_pair", "ring4_l3", "pair_cr_l5", "local_ops_l3"])
def test_fourth_order_pulse_gradient_matches_oracle(sgctx, default_path, name, scheme):
    # Q4j's complex steps make its factors non-unitary: the states are pulled back by
    # the inverses and the co-states by the adjoints
    wl = CASES[name]()
    s = _system(sgctx, wl)
    F_r, g_r = q2_pulse_gradient(wl, scheme=scheme)
    scale = max(1.0, np.max(np.abs(g_r)))
    for prec, tol_F, tol_g in (("fp64", 1e-10, 1e-9), ("mixed", 1e-5, 2e-4)):
        F, gp, _ = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=wl["fid_kind"],
                                   precision=prec, ham=False, solver=scheme)
        Fk = F[0] if wl["fid_kind"] == "avg" else F[1]
        assert abs(Fk - F_r) < tol_F, (prec, Fk, F_r)
        assert np.max(np.abs(gp - g_r)) < tol_g * scale, (prec, np.max(np.abs(gp - g_r)), scale)


@pytest.mark.parametrize("steps", [1, 3])
@pytest.mark.parametrize("scheme", ["q2", "q4", "q4j"])
def test_edge_cases_single_step_and_no_couplings(sgctx, default_path, steps, scheme):
    # one step (the first and last 1-body rows coincide) and a system without couplings
    # (empty palindrome, no coupling unitaries)
    wl = W.fluxonium_pair_multipath(seed=13, levels=3, nseg=1)
    wl["couplings"] = []
    wl = _short(wl, T=steps * wl["dt"])
    s = _system(sgctx, wl)
    so = OracleSystem(dict(wl, frame="lab"))
    ref = q2_evolve(so, initial_columns(so, wl["col_index"]), scheme=scheme)
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"], solver=scheme).cpu().numpy()
    assert np.max(np.abs(psi - ref)) < 1e-12
    F_r, g_r = q2_pulse_gradient(wl, scheme=scheme)
    F, gp, _ = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=wl["fid_kind"],
                               precision="fp64", ham=False, solver=scheme)
    assert np.max(np.abs(gp - g_r)) < 1e-9 * max(1.0, np.max(np.abs(g_r)))


def test_q2_full_size_chain6_sampled_columns(sgctx, default_path):
    """The 6-fluxonium chain at its full size (D = 4096, all 64 computational columns,
    the on-chip launch of the bench) over 200 steps: two sampled columns against the
    oracle's Q2, FP64 within 1e-10 and mixed within 1e-5."""
    wl = W.fluxonium_chain6(seed=1)
    wl = _short(wl, T=2.0)
    s = _system(sgctx, wl)
    so = OracleSystem(dict(wl, frame="lab"))
    pick = [0, 37]
    ref = q2_evolve(so, initial_columns(so, [wl["col_index"][c] for c in pick]))
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        psi = s.evolve(wl["T"], wl["dt"], precision=prec, col_index=wl["col_index"], solver="q2").cpu().numpy()
        assert psi.shape == (4096, 64)
        assert np.max(np.abs(psi[:, pick] - ref)) < tol, prec
