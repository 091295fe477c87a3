"""sg_evolve_noalloc: the evolution entry point for callers that cannot allocate
device memory during the call (their memory belongs to another allocator, or
they cannot afford cudaMalloc's synchronisation).  It must give the same states
as sg_evolve and as the FP64 oracle, on repeated calls that reuse its fixed scratch
array, and refuse sizes beyond that array.  Kept in a file of its own that pytest
collects last."""
import ctypes

import numpy as np
import pytest

from oracle.evolve import frame_epilogue, initial_columns, rk4_evolve
from oracle.system import OracleSystem
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(sgctx, system, T, dt, prec, cols):
    import torch
    from paper_2406_18155_gb300.api import evolve_opts
    from paper_2406_18155_gb300.capi import check, lib
    D, _ = system.dims()
    psi = torch.empty((D, len(cols)), dtype=torch.complex128, device="cuda")
    o, keep = evolve_opts(T, dt, prec, "interaction", cols)
    check(lib().sg_evolve_noalloc(system.h, ctypes.byref(o), ctypes.c_void_p(psi.data_ptr())),
          sgctx.h)
    return psi.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_noalloc_matches_sg_evolve_on_two_calls(sgctx, prec, tol):
    from paper_2406_18155_gb300.api import System
    wl = W.fluxonium_chain(seed=21, nq=3, levels=4, T=0.5, dt=0.01, nseg=3, ring=True)
    s = System.from_workload(sgctx, wl)
    s.prepare()
    ref = s.evolve(wl["T"], wl["dt"], precision=prec, col_index=wl["col_index"]).cpu().numpy()
    so = OracleSystem(wl)
    orc = frame_epilogue(so, rk4_evolve(so, initial_columns(so, wl["col_index"])))
    for _ in range(2):
        out = _noalloc(sgctx, s, wl["T"], wl["dt"], prec, wl["col_index"])
        assert np.max(np.abs(out - ref)) < tol
        assert np.max(np.abs(out - orc)) < tol


def test_noalloc_rejects_sizes_beyond_its_scratch(sgctx):
    from paper_2406_18155_gb300.api import System
    from paper_2406_18155_gb300.capi import SGError, SG_E_INVALID
    wl = W.fluxonium_ring10(seed=22, T=0.05, ncols=2)
    for d in wl["drives"]:
        d["length"] = wl["T"]
    s = System.from_workload(sgctx, wl)
    s.prepare()
    with pytest.raises(SGError) as e:
        _noalloc(sgctx, s, wl["T"], wl["dt"], "fp64", wl["col_index"])   # 3 slabs of 2^20 x 2 x 16 B
    assert e.value.code == SG_E_INVALID
    assert "MiB" in str(e.value)
