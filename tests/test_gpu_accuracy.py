"""Accuracy of the mixed-precision path at the step counts the workloads run, against
the FP64 oracle and the FP64 GPU path (through the C ABI).

* Transmon pair (D = 16, N = 10^4) and fluxonium cross-resonance pair (D = 25,
  N = 10^4): the whole horizon against the oracle's stored results
  (`golden/full_horizon.json`), targets the polar factor of the oracle's block so
  that F is close to 1.  FP64: 1e-10 on U_c and F, gradient 1e-7 of its largest
  component (the paper's bound for its adjoint, Sec. 4.3; 10^4 steps of FP64 rounding
  in two summation orders reach ~1e-8).  Mixed: |dF| <= 1e-5, U_c within 1e-5, gradient within 1e-3.
* 6-fluxonium chain (D = 4096, 64 columns, N = 6000): mixed against FP64 on the
  GPU over the whole horizon (F_state with the polar factor of the FP64 block as
  target, every amplitude, the gradient), and two columns against the oracle's
  matrix-free evolution at full N (stored).
* 10-fluxonium ring (D = 2^20, N = 4000), two columns: mixed against FP64 on the
  GPU over the whole horizon, forward and pulse gradient, with the FP64 result's
  normalised computational rows as target (F_state close to 1).

Each test records its measured errors in the assertion message and prints them.
"""
import json
import os

import numpy as np
import pytest

from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_horizon.json")


def _c(a):
    a = np.asarray(a)
    return a[..., 0] + 1j * a[..., 1]


def _gold(name):
    with open(GOLD) as f:
        return json.load(f)["cases"][name]


def _system(sgctx, wl):
    from paper_2406_18155_gb300.api import System
    s = System.from_workload(sgctx, wl)
    s.prepare()
    return s


def _polar(U):
    u, _, vh = np.linalg.svd(U)
    return u @ vh


@pytest.mark.parametrize("name,make", [("transmon_pair", lambda: W.transmon_pair(seed=0)),
                                       ("fluxonium_pair_cr", lambda: W.fluxonium_pair_cr(seed=0))])
def test_pairs_full_horizon_against_oracle(sgctx, name, make):
    g = _gold(name)
    wl = make()
    wl["target"] = _c(g["target"])
    s = _system(sgctx, wl)
    assert int(round(wl["T"] / wl["dt"])) == g["N"] == 10000
    Uref, gref = _c(g["Uc"]), np.array(g["grad_avg"])
    gmax = np.max(np.abs(gref))
    res = {}
    for prec in ("fp64", "mixed"):
        Fa, Fs, U = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision=prec)
        F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg",
                                    precision=prec)
        gg = np.concatenate([gp, gh])
        npul = len(gp)
        res[prec] = {"dU": float(np.max(np.abs(U - Uref))), "dFavg": abs(Fa - g["F_avg"]),
                     "dFstate": abs(Fs - g["F_state"]), "dFgrad": abs(F[0] - g["F_avg"]),
                     "rel_dgrad": float(np.max(np.abs(gg - gref)) / gmax),
                     "rel_dgrad_pulse": float(np.max(np.abs(gp - gref[:npul])) / gmax),
                     "rel_dgrad_ham": float(np.max(np.abs(gh - gref[npul:])) / gmax),
                     "worst_param": g["params"][int(np.argmax(np.abs(gg - gref)))]}
    print(name, "F_avg", g["F_avg"], res)
    assert g["F_avg"] > 0.9
    r = res["fp64"]
    assert r["dU"] < 1e-10 and r["dFavg"] < 1e-10 and r["dFstate"] < 1e-10 and r["dFgrad"] < 1e-10, res
    # 10^4 steps of FP64 in two summation orders: the paper's bound for its own
    # adjoint against automatic differentiation, 1e-7 relative (Sec. 4.3)
    assert r["rel_dgrad"] < 1e-7, res
    r = res["mixed"]
    assert r["dU"] < 1e-5 and r["dFavg"] < 1e-5 and r["dFstate"] < 1e-5 and r["dFgrad"] < 1e-5, res
    assert r["rel_dgrad"] < 1e-3, res


def _block(U, wl):
    """D_c x D_c block with the evolved computational columns at their labels."""
    comp = W.comp_states([m["levels"] for m in wl["modes"]])
    lab = {r: j for j, r in enumerate(comp)}
    B = np.zeros((len(comp), len(comp)), dtype=np.complex128)
    for s, r in enumerate(wl["col_index"]):
        if r in lab:
            B[:, lab[r]] = U[:, s]
    return B


def test_chain6_full_horizon_mixed_against_fp64(sgctx):
    import torch
    wl = W.fluxonium_chain6(seed=0)
    s = _system(sgctx, wl)
    N = int(round(wl["T"] / wl["dt"]))
    assert N == 6000
    psi64 = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"]).cpu().numpy()
    torch.cuda.synchronize()
    comp = W.comp_states([4] * 6)
    target = _polar(_block(psi64[comp, :], wl))
    F64 = s.fidelity(wl["T"], wl["dt"], target, wl["col_index"], precision="fp64")
    F32 = s.fidelity(wl["T"], wl["dt"], target, wl["col_index"], precision="mixed")
    _, g64p, g64h = s.fidelity_grad(wl["T"], wl["dt"], target, wl["col_index"], kind="state", precision="fp64")
    _, g32p, g32h = s.fidelity_grad(wl["T"], wl["dt"], target, wl["col_index"], kind="state", precision="mixed")
    g64, g32 = np.concatenate([g64p, g64h]), np.concatenate([g32p, g32h])
    res = {"dpsi": float(np.max(np.abs(psi32 - psi64))), "F_state": F64[1],
           "dF_state": abs(F32[1] - F64[1]), "rel_dgrad": float(np.max(np.abs(g32 - g64)) / np.max(np.abs(g64)))}
    print("chain6", res)
    assert F64[1] > 0.9
    assert res["dpsi"] < 1e-5 and res["dF_state"] < 1e-5 and res["rel_dgrad"] < 1e-3, res
    # two columns against the oracle's matrix-free evolution over the whole horizon
    gc = _gold("fluxonium_chain6")
    idx = [wl["col_index"].index(r) for r in gc["col_index"]]
    rows = np.array(gc["rows"])
    ref = _c(gc["psi_rows"])
    assert np.max(np.abs(psi64[np.ix_(rows, idx)] - ref)) < 1e-10
    assert np.max(np.abs(psi32[np.ix_(rows, idx)] - ref)) < 1e-5
    assert np.max(np.abs(np.linalg.norm(psi64[:, idx], axis=0) - np.array(gc["norms"]))) < 1e-10


def test_ring10_full_horizon_two_columns_mixed_against_fp64(sgctx):
    wl = W.fluxonium_ring10(seed=0, ncols=2)
    s = _system(sgctx, wl)
    assert int(round(wl["T"] / wl["dt"])) == 4000
    psi64 = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"]).cpu().numpy()
    comp = W.comp_states([4] * 10)
    lab = {r: j for j, r in enumerate(comp)}
    target = np.zeros((len(comp), len(comp)), dtype=np.complex128)
    for sidx, r in enumerate(wl["col_index"]):
        v = psi64[comp, sidx]
        target[:, lab[r]] = v / np.linalg.norm(v)
    F64, g64, _ = s.fidelity_grad(wl["T"], wl["dt"], target, wl["col_index"], kind="state",
                                  precision="fp64", ham=False)
    F32, g32, _ = s.fidelity_grad(wl["T"], wl["dt"], target, wl["col_index"], kind="state",
                                  precision="mixed", ham=False)
    res = {"dpsi": float(np.max(np.abs(psi32 - psi64))), "F_state": F64[1],
           "dF_state": abs(F32[1] - F64[1]), "rel_dgrad": float(np.max(np.abs(g32 - g64)) / np.max(np.abs(g64)))}
    print("ring10", res)
    assert F64[1] > 0.5
    assert res["dpsi"] < 1e-5 and res["dF_state"] < 1e-5 and res["rel_dgrad"] < 1e-3, res
