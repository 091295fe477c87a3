"""The on-chip adjoint's bounded mbarrier wait, made to run out on purpose.

A test knob makes CTA 0 skip the bulk copy of its first stage input in every
adjoint launch (SG_TEST_SKIP_BULK=1) and shortens the wait to a few thousand polls
(SG_TEST_WAIT_LIMIT): nothing will ever complete that phase, so the wait gives up,
the CTA issues no further bulk copies and runs to its end, and the call must return
SG_E_TIMEOUT.  No copy is left in flight and no access leaves its buffer, so the
context stays usable: the same solve afterwards gives the result it gave before."""
import numpy as np
import pytest

from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_wait_runs_out_and_reports_timeout(sgctx, monkeypatch, prec):
    from paper_2406_18155_gb300.api import System
    from paper_2406_18155_gb300.capi import SGError, SG_E_TIMEOUT
    monkeypatch.delenv("SG_PATH", raising=False)
    wl = W.fluxonium_chain(seed=31, nq=3, levels=3, T=0.3, dt=0.01, nseg=3)
    s = System.from_workload(sgctx, wl)
    s.prepare()

    def solve():
        return s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                               precision=prec, ckpt=10)
    F0, gp0, gh0 = solve()
    monkeypatch.setenv("SG_TEST_WAIT_LIMIT", "2000")
    monkeypatch.setenv("SG_TEST_SKIP_BULK", "1")
    with pytest.raises(SGError) as e:
        solve()
    assert e.value.code == SG_E_TIMEOUT
    assert "bounded wait" in str(e.value)
    monkeypatch.delenv("SG_TEST_SKIP_BULK")
    monkeypatch.delenv("SG_TEST_WAIT_LIMIT")
    F1, gp1, gh1 = solve()
    assert np.array_equal(F0, F1) and np.array_equal(gp0, gp1) and np.array_equal(gh0, gh1)
