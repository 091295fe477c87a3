"""GPU parity of the batched dense evolution on the tensor cores (sg_evolve_batch:
tcgen05 TF32 products split 3xTF32, FP32 stage math, float-float state) against
the FP64 oracle, through the C ABI.

* Transmon pairs (D = 16, 16 columns, 4 systems per CTA) and fluxonium
  cross-resonance pairs (D = 25, 4 columns, 2 per CTA), systems of different seeds
  in one batch, a ragged last CTA, both frames: every amplitude within 1e-5 of the
  oracle, as for the other mixed-precision paths.
* The two pairs over their full horizons (10^4 steps): the computational block
  against the oracle's stored result (`golden/full_horizon.json`) within 1e-5, and
  F_avg with the stored polar-factor target within 1e-5.
* Shapes the tensor-core path does not take are refused with SG_E_UNSUPPORTED."""
import json
import os

import numpy as np
import pytest

from oracle.evolve import frame_epilogue, initial_columns, rk4_evolve
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_horizon.json")


def _systems(sgctx, wls):
    from paper_2406_18155_gb300.api import System
    out = []
    for wl in wls:
        s = System.from_workload(sgctx, wl)
        s.prepare()
        out.append(s)
    return out


def _oracle_psi(wl):
    so = OracleSystem(wl)
    return frame_epilogue(so, rk4_evolve(so, initial_columns(so, wl["col_index"])))


@pytest.mark.parametrize("frame", ["interaction", "lab"])
@pytest.mark.parametrize("kind,nsys", [("transmon", 6), ("fluxonium_cr", 3)])
def test_batch_matches_oracle(sgctx, kind, nsys, frame):
    from paper_2406_18155_gb300.api import evolve_batch
    if kind == "transmon":
        T, dt = (1.0, 0.005) if frame == "interaction" else (0.2, 0.001)
        wls = [W.transmon_pair(seed=20 + k, T=T, dt=dt) for k in range(nsys)]
    else:
        T, dt = (1.0, 0.01) if frame == "interaction" else (0.2, 0.002)
        wls = [W.fluxonium_pair_cr(seed=30 + k, T=T, dt=dt) for k in range(nsys)]
    for wl in wls:
        wl["frame"] = frame
    sys_ = _systems(sgctx, wls)
    psi = evolve_batch(sys_, T, dt, wls[0]["col_index"], frame=frame).cpu().numpy()
    for k, wl in enumerate(wls):
        ref = _oracle_psi(wl)
        assert np.max(np.abs(psi[k] - ref)) < 1e-5, (k, np.max(np.abs(psi[k] - ref)))
    # the same systems one at a time on the on-chip kernels (mixed)
    for k, (wl, s) in enumerate(zip(wls, sys_)):
        one = s.evolve(T, dt, precision="mixed", frame=frame, col_index=wl["col_index"]).cpu().numpy()
        assert np.max(np.abs(psi[k] - one)) < 1e-5


@pytest.mark.parametrize("name,make", [("transmon_pair", lambda: W.transmon_pair(seed=0)),
                                       ("fluxonium_pair_cr", lambda: W.fluxonium_pair_cr(seed=0))])
def test_batch_full_horizon_against_stored_oracle(sgctx, name, make):
    from paper_2406_18155_gb300.api import evolve_batch
    with open(GOLD) as f:
        g = json.load(f)["cases"][name]
    wl = make()
    s = _systems(sgctx, [wl])
    psi = evolve_batch(s, wl["T"], wl["dt"], wl["col_index"]).cpu().numpy()[0]
    comp = W.comp_states([m["levels"] for m in wl["modes"]])
    Uc = psi[comp, :]
    Uref = np.asarray(g["Uc"])[..., 0] + 1j * np.asarray(g["Uc"])[..., 1]
    du = np.max(np.abs(Uc - Uref))
    # F_avg with the stored target from the D_c x D_c block
    T = np.asarray(g["target"])[..., 0] + 1j * np.asarray(g["target"])[..., 1]
    lab = {r: j for j, r in enumerate(comp)}
    U = np.zeros_like(T)
    for sidx, r in enumerate(wl["col_index"]):
        if r in lab:
            U[:, lab[r]] = Uc[:, sidx]
    M = T.conj().T @ U
    Dc = T.shape[0]
    F = (np.real(np.trace(M @ M.conj().T)) + abs(np.trace(M)) ** 2) / (Dc * (Dc + 1))
    print(name, "dU", du, "dF", abs(F - g["F_avg"]))
    assert du < 1e-5 and abs(F - g["F_avg"]) < 1e-5


def test_batch_refuses_shapes_it_does_not_take(sgctx):
    from paper_2406_18155_gb300.api import evolve_batch
    from paper_2406_18155_gb300.capi import SGError, SG_E_UNSUPPORTED
    wl = W.fluxonium_chain(seed=1, nq=3, levels=3, T=0.1, dt=0.01, nseg=2)
    s = _systems(sgctx, [wl])
    with pytest.raises(SGError) as e:                   # 5 columns: 2 S not in {8, 16, 32}
        evolve_batch(s, wl["T"], wl["dt"], wl["col_index"][:5])
    assert e.value.code == SG_E_UNSUPPORTED
    wl2 = W.local_op_pair(seed=2, T=0.1)                # a genuinely complex local operator
    s2 = _systems(sgctx, [wl2])
    with pytest.raises(SGError) as e:
        evolve_batch(s2, wl2["T"], wl2["dt"], wl2["col_index"])
    assert e.value.code == SG_E_UNSUPPORTED
