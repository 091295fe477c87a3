"""GPU parity of the on-chip kernels (columns resident in shared memory for the whole
evolution) against the FP64 oracle, and against the tiled HBM kernels.

Shapes cover one CTA holding every column, several CTAs with a ragged last group
(columns past S are zero padding), every level count the kernels take (2..5), both
frames, both fidelity kinds and several checkpoint segment lengths.  Tolerances as
for the other paths: FP64 1e-10 on amplitudes and F, gradients 1e-8 relative to the
largest component; mixed 1e-5 on F and amplitudes, 1e-3 on gradients."""
import numpy as np
import pytest

from oracle.evolve import initial_columns, rk4_evolve, frame_epilogue, adjoint_gradient
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system(sgctx, wl):
    from paper_2406_18155_gb300.api import System
    s = System.from_workload(sgctx, wl)
    s.prepare()
    return s


def _oracle_psi(wl):
    so = OracleSystem(wl)
    return frame_epilogue(so, rk4_evolve(so, initial_columns(so, wl["col_index"])))


def _chain(seed, nq, levels, T=0.2, dt=0.01, ncols=None, ring=False, extra_cols=()):
    wl = W.fluxonium_chain(seed=seed, nq=nq, levels=levels, T=T, dt=dt, nseg=3, ring=ring, ncols=ncols)
    wl["col_index"] = list(wl["col_index"]) + list(extra_cols)
    return wl


SHAPES = {
    # name: (workload, why)
    "pair_l2": lambda: _chain(1, 2, 2),                          # D = 4, one block per column
    "chain3_l3": lambda: _chain(2, 3, 3),                        # D = 27, all 8 columns in one CTA
    "chain4_l4_ragged": lambda: _chain(3, 4, 4, extra_cols=[6, 77, 130, 255, 201]),   # 21 cols, 2 CTAs, 1 pad
    "ring5_l3": lambda: _chain(4, 5, 3, ring=True),              # D = 243, 32 columns over 4 CTAs
    "pair_l5": lambda: _chain(5, 2, 5, extra_cols=[24, 13]),     # D = 25
    "transmon_pair": lambda: W.transmon_pair(seed=6, T=0.5),     # transmons, Gaussian drive
}


@pytest.fixture
def onchip(monkeypatch):
    monkeypatch.delenv("SG_PATH", raising=False)
    monkeypatch.delenv("SG_SLAB_TMAX", raising=False)


@pytest.mark.parametrize("shape", sorted(SHAPES))
@pytest.mark.parametrize("frame", ["interaction", "lab"])
def test_onchip_forward_matches_oracle(sgctx, onchip, shape, frame):
    wl = SHAPES[shape]()
    wl["frame"] = frame
    s = _system(sgctx, wl)
    ref = _oracle_psi(wl)
    psi = s.evolve(wl["T"], wl["dt"], precision="fp64", frame=frame, col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi - ref)) < 1e-10
    psi32 = s.evolve(wl["T"], wl["dt"], precision="mixed", frame=frame, col_index=wl["col_index"]).cpu().numpy()
    assert np.max(np.abs(psi32 - ref)) < 1e-5


@pytest.mark.parametrize("shape", ["pair_l2", "chain3_l3", "chain4_l4_ragged", "ring5_l3", "transmon_pair"])
@pytest.mark.parametrize("ckpt", [1, 4, 0])
def test_onchip_gradient_matches_oracle(sgctx, onchip, shape, ckpt):
    wl = SHAPES[shape]()
    kind = "state" if shape != "transmon_pair" else "avg"
    s = _system(sgctx, wl)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=kind,
                                precision="fp64", ckpt=ckpt)
    wl["fid_kind"] = kind
    Fr, gr, _ = adjoint_gradient(wl)
    k = 0 if kind == "avg" else 1
    assert abs(F[k] - Fr) < 1e-10
    g = np.concatenate([gp, gh])
    assert np.max(np.abs(g - gr)) <= 1e-8 * np.max(np.abs(gr))
    F32, gp32, gh32 = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=kind,
                                      precision="mixed", ckpt=ckpt)
    assert abs(F32[k] - Fr) < 1e-5
    assert np.max(np.abs(np.concatenate([gp32, gh32]) - gr)) <= 1e-3 * np.max(np.abs(gr))


def test_onchip_lab_frame_gradient(sgctx, onchip):
    wl = SHAPES["chain3_l3"]()
    wl["frame"] = "lab"
    wl["T"] = 0.1
    for d in wl["drives"]:
        d["length"] = 0.1
    s = _system(sgctx, wl)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                precision="fp64", frame="lab", ckpt=3)
    Fr, gr, _ = adjoint_gradient(wl)
    assert abs(F[1] - Fr) < 1e-10
    assert np.max(np.abs(np.concatenate([gp, gh]) - gr)) <= 1e-8 * np.max(np.abs(gr))


def test_onchip_agrees_with_tiled_kernels_at_d1024(sgctx, monkeypatch):
    # D = 4^5 = 1024: one column per CTA group of 4; the tiled HBM kernels as the check
    wl = _chain(8, 5, 4, T=0.3, ncols=12)
    s = _system(sgctx, wl)
    out = {}
    for pth in ("onchip", "slab"):
        monkeypatch.setenv("SG_PATH", pth)
        F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                    precision="fp64", ckpt=7)
        psi = s.evolve(wl["T"], wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
        out[pth] = (F[1], np.concatenate([gp, gh]), psi)
    assert abs(out["onchip"][0] - out["slab"][0]) < 1e-12
    assert np.max(np.abs(out["onchip"][2] - out["slab"][2])) < 1e-12
    g = out["slab"][1]
    assert np.max(np.abs(out["onchip"][1] - g)) <= 1e-10 * np.max(np.abs(g))


def test_onchip_largest_tile_mixed(sgctx, onchip, monkeypatch):
    # D = 5^5 = 3125, the largest single-tile shape of the serving mix: mixed
    # precision against the FP64 gather kernels on the same system
    for seed in range(10000):
        wl = W.serving_request(np.random.Generator(np.random.PCG64(seed)))
        if len(wl["modes"]) == 5 and wl["modes"][0]["levels"] == 5:
            break
    wl["T"] = 0.3
    for d in wl["drives"]:
        d["length"] = 0.3
    s = _system(sgctx, wl)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg",
                                precision="mixed")
    monkeypatch.setenv("SG_PATH", "gather")
    Fg, gpg, ghg = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg",
                                   precision="fp64")
    assert abs(F[0] - Fg[0]) < 1e-5
    g = np.concatenate([gpg, ghg])
    assert np.max(np.abs(np.concatenate([gp, gh]) - g)) <= 1e-3 * np.max(np.abs(g))


def test_onchip_d4096_low_words_in_global(sgctx, monkeypatch):
    # D = 4^6 = 4096: the mixed adjoint fits one column per CTA only with the
    # co-state's low words in global memory; checked against the FP64 tiled kernels
    wl = _chain(11, 6, 4, T=0.2, ncols=8)
    s = _system(sgctx, wl)
    monkeypatch.delenv("SG_PATH", raising=False)
    F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                precision="mixed", ckpt=6)
    monkeypatch.setenv("SG_PATH", "slab")
    Fr, gpr, ghr = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                   precision="fp64", ckpt=6)
    assert abs(F[1] - Fr[1]) < 1e-5
    g, gr = np.concatenate([gp, gh]), np.concatenate([gpr, ghr])
    assert np.max(np.abs(g - gr)) <= 1e-3 * np.max(np.abs(gr))
