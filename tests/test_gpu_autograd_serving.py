"""torch.autograd.Function against central differences and the oracle adjoint, and
the continuous-batching server: results alone equal results in the mix."""
import numpy as np
import pytest

import oracle
from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system(sgctx, wl):
    from paper_2406_18155_gb300.api import System
    s = System.from_workload(sgctx, wl)
    s.prepare()
    return s


def test_autograd_function_matches_oracle_and_central_differences(sgctx):
    import torch
    from paper_2406_18155_gb300.autograd import fidelity
    wl = W.fluxonium_pair_cr(seed=12, T=0.3)
    s = _system(sgctx, wl)
    p0, h0 = s.get_params()
    pulse = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    ham = torch.tensor(h0, dtype=torch.float64, requires_grad=True)
    args = (wl["T"], wl["dt"], wl["target"], wl["col_index"])
    F = fidelity(s, pulse, ham, *args, kind="avg", precision="fp64")
    (2.0 * F).backward()
    Fr, gr, prms = oracle.adjoint_gradient(wl)
    assert abs(F.item() - Fr) < 1e-10
    g = np.concatenate([pulse.grad.numpy(), ham.grad.numpy()])
    assert np.max(np.abs(g - 2.0 * gr)) <= 1e-8 * np.max(np.abs(gr))
    # central differences through the library (FP64): a pulse amplitude and E_C of mode 0
    th = np.concatenate([p0, h0])
    for idx, h in [(3, 1e-6), (len(p0) + 1, 1e-6)]:
        step = h * max(1.0, abs(th[idx]))
        vals = []
        for sgn in (+1, -1):
            t2 = th.copy()
            t2[idx] += sgn * step
            with torch.no_grad():
                vals.append(fidelity(s, torch.tensor(t2[:len(p0)]), torch.tensor(t2[len(p0):]),
                                     *args, kind="avg", precision="fp64").item())
        fd = (vals[0] - vals[1]) / (2 * step)
        assert abs(fd - gr[idx]) <= 1e-5 * max(abs(gr[idx]), 1e-6), (idx, fd, gr[idx])


def test_server_results_alone_equal_results_in_the_mix(sgctx):
    from paper_2406_18155_gb300.api import Server
    rng = np.random.Generator(np.random.PCG64(5))
    wls = []
    for _ in range(8):
        wl = W.serving_request(rng)
        n = int(round(rng.uniform(0.2, 0.6) / wl["dt"]))
        wl["T"] = n * wl["dt"]
        for d in wl["drives"]:
            d["length"] = wl["T"]
        wls.append(wl)
    alone = []
    for wl in wls:
        s = _system(sgctx, wl)
        alone.append(s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                     kind=wl["fid_kind"], precision="mixed"))
    srv = Server(sgctx, mem_budget_bytes=8 << 30, max_slots=3)
    systems = [_system(sgctx, wl) for wl in wls]
    tickets = [srv.submit(sy, wl["T"], wl["dt"], wl["target"], wl["col_index"],
                          kind=wl["fid_kind"], precision="mixed") for sy, wl in zip(systems, wls)]
    res = [srv.wait(t) for t in tickets]
    for (F, gp, gh), r in zip(alone, res):
        assert r["status"] == 0
        assert (np.isnan(F[0]) and np.isnan(r["F"][0])) or abs(r["F"][0] - F[0]) <= 1e-12
        assert abs(r["F"][1] - F[1]) <= 1e-12
        assert np.max(np.abs(r["grad_pulse"] - gp)) <= 1e-12 * max(1.0, np.max(np.abs(gp)))
        assert np.max(np.abs(r["grad_ham"] - gh)) <= 1e-12 * max(1.0, np.max(np.abs(gh)))
    # continuous batching: later requests started while the first ones were running
    starts = sorted(r["start_s"] for r in res)
    dones = sorted(r["done_s"] for r in res)
    assert starts[1] < dones[0] and starts[2] < dones[0]
    st = srv.stats()
    assert st["completed"] == len(wls) and st["p99_s"] >= st["p50_s"] > 0
    srv.close()


def test_server_packs_same_shape_requests_into_batched_launches(sgctx):
    # one slot packing up to 4 queued requests of one step shape (3 fluxoniums at 3
    # levels; different parameters, pulses and durations) into shared batched
    # on-chip launches, beside requests of other shapes: every result equals the
    # request's solve alone
    from paper_2406_18155_gb300.api import Server
    rng = np.random.Generator(np.random.PCG64(7))
    wls = []
    for i in range(9):
        shape = dict(nq=3, kind="fluxonium", levels=3) if i % 3 != 2 else dict(nq=2, kind="transmon", levels=4)
        wl = W.serving_request(rng, **shape)
        n = int(round(rng.uniform(0.2, 0.6) / wl["dt"]))
        wl["T"] = n * wl["dt"]
        for d in wl["drives"]:
            d["length"] = wl["T"]
        wls.append(wl)
    alone = []
    for wl in wls:
        s = _system(sgctx, wl)
        alone.append(s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                     kind=wl["fid_kind"], precision="mixed"))
    srv = Server(sgctx, mem_budget_bytes=8 << 30, max_slots=1, max_batch=4)
    systems = [_system(sgctx, wl) for wl in wls]
    tickets = [srv.submit(sy, wl["T"], wl["dt"], wl["target"], wl["col_index"],
                          kind=wl["fid_kind"], precision="mixed") for sy, wl in zip(systems, wls)]
    res = [srv.wait(t) for t in tickets]
    for (F, gp, gh), r in zip(alone, res):
        assert r["status"] == 0, r["error"]
        assert abs(r["F"][1] - F[1]) <= 1e-12 and abs(r["F"][0] - F[0]) <= 1e-12
        assert np.max(np.abs(r["grad_pulse"] - gp)) <= 1e-12 * max(1.0, np.max(np.abs(gp)))
        assert np.max(np.abs(r["grad_ham"] - gh)) <= 1e-12 * max(1.0, np.max(np.abs(gh)))
    st = srv.stats()
    assert st["completed"] == len(wls)
    assert st["batches"] >= 1 and st["batched_requests"] >= 2
    assert st["batched_launches"] >= 1 and st["batched_launch_members"] > st["batched_launches"]
    srv.close()


def test_server_concurrent_shapes_sharing_kernels(sgctx):
    # every 3-level request (2..5 modes, both kinds) launches the same kernels with
    # different shared-memory sizes; many run at once, none may fail or change
    from paper_2406_18155_gb300.api import Server
    wls = []
    for seed in range(4000):
        wl = W.serving_request(np.random.Generator(np.random.PCG64(seed)))
        if wl["modes"][0]["levels"] != 3 or any(w["name"] == wl["name"] for w in wls):
            continue
        wl["T"] = 40 * wl["dt"]
        for d in wl["drives"]:
            d["length"] = wl["T"]
        wls.append(wl)
        if len(wls) == 8:
            break
    alone = {}
    for wl in wls:
        s = _system(sgctx, wl)
        alone[wl["name"]] = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                            kind="avg", precision="mixed")
    srv = Server(sgctx, mem_budget_bytes=16 << 30, max_slots=16)
    reqs = [(wl, _system(sgctx, wl)) for wl in wls for _ in range(4)]
    tickets = [srv.submit(sy, wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg")
               for wl, sy in reqs]
    res = [srv.wait(t) for t in tickets]
    srv.close()
    for (wl, _), r in zip(reqs, res):
        assert r["status"] == 0, (wl["name"], r["error"])
        F, gp, gh = alone[wl["name"]]
        assert abs(r["F"][0] - F[0]) <= 1e-12
        assert np.max(np.abs(r["grad_pulse"] - gp)) <= 1e-12 * max(1.0, np.max(np.abs(gp)))


def test_server_admission_and_cancel(sgctx):
    from paper_2406_18155_gb300.api import Server
    from paper_2406_18155_gb300.capi import SGError, SG_E_NOMEM_RETRY
    wl = W.fluxonium_pair_cr(seed=3, T=2.0)
    s = _system(sgctx, wl)
    tiny = Server(sgctx, mem_budget_bytes=1 << 20, max_slots=1)
    with pytest.raises(SGError) as e:
        tiny.submit(s, wl["T"], wl["dt"], wl["target"], wl["col_index"])
    assert e.value.code == SG_E_NOMEM_RETRY
    tiny.close()
    srv = Server(sgctx, mem_budget_bytes=4 << 30, max_slots=1)
    sys2 = [_system(sgctx, wl) for _ in range(4)]
    t = [srv.submit(sy, wl["T"], wl["dt"], wl["target"], wl["col_index"]) for sy in sys2]
    assert srv.cancel(t[-1]) == 0              # still queued behind the single slot
    for x in t[:-1]:
        assert srv.wait(x)["status"] == 0
    assert srv.stats()["cancelled"] == 1
    srv.close()


def test_server_refuses_a_system_already_in_flight(sgctx):
    # a slot runs a request with its own context and may prepare the system, so a
    # system takes one request at a time; after its result it can be submitted again
    from paper_2406_18155_gb300.api import Server
    from paper_2406_18155_gb300.capi import SGError, SG_E_STATE
    wl = W.fluxonium_pair_cr(seed=4, T=2.0)
    s = _system(sgctx, wl)
    srv = Server(sgctx, mem_budget_bytes=4 << 30, max_slots=2)
    t0 = srv.submit(s, wl["T"], wl["dt"], wl["target"], wl["col_index"])
    with pytest.raises(SGError) as e:
        srv.submit(s, wl["T"], wl["dt"], wl["target"], wl["col_index"])
    assert e.value.code == SG_E_STATE
    r0 = srv.wait(t0)
    t1 = srv.submit(s, wl["T"], wl["dt"], wl["target"], wl["col_index"])
    r1 = srv.wait(t1)
    assert r0["status"] == 0 and r1["status"] == 0
    assert r0["F"][0] == r1["F"][0] and np.array_equal(r0["grad_pulse"], r1["grad_pulse"])
    srv.close()
