"""The column-sharded solve through the C ABI (sg_fidelity_grad_sharded): two
processes on one GPU, each evolving half of the columns, exchange their fidelity
sums and gradients over gloo (host-side: no kernel waits on another process), and
must reproduce the unsharded sg_fidelity_grad: FP64 within 1e-12 relative (only
summation orders differ), mixed within 1e-5 in F and 1e-4 of the largest gradient
component (the FP32 per-CTA accumulators group the columns differently)."""
import os
import socket

import numpy as np
import pytest

from paper_2406_18155_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workload(kind):
    if kind == "state":
        return W.fluxonium_chain(seed=41, nq=4, levels=3, T=0.4, dt=0.01, nseg=3, ring=True)
    wl = W.fluxonium_pair_cr(seed=42, T=1.0)
    return wl


def _shard_main(rank, world, port, kind, prec, path, out):
    import torch
    import torch.distributed as dist
    if path:
        os.environ["SG_PATH"] = path
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2406_18155_gb300 import build
    build.build()
    from paper_2406_18155_gb300.api import Context, System
    from paper_2406_18155_gb300.shard import column_block, torch_allreduce
    torch.cuda.set_device(0)
    wl = _workload(kind)
    ctx = Context(0)
    s = System.from_workload(ctx, wl)
    s.prepare()
    a, b = column_block(len(wl["col_index"]), rank, world)
    F, gp, gh = s.fidelity_grad_sharded(wl["T"], wl["dt"], wl["target"], wl["col_index"][a:b],
                                        torch_allreduce(), kind=kind, precision=prec, ckpt=7)
    out.put((rank, F, gp, gh))
    dist.barrier()
    ctx.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind,prec,path", [("state", "fp64", None), ("avg", "fp64", None),
                                            ("state", "mixed", None), ("state", "fp64", "slab")])
def test_two_shards_equal_the_unsharded_solve(sgctx, kind, prec, path, monkeypatch):
    import torch.multiprocessing as mp
    from paper_2406_18155_gb300.api import System
    if path:
        monkeypatch.setenv("SG_PATH", path)
    wl = _workload(kind)
    s = System.from_workload(sgctx, wl)
    s.prepare()
    F1, gp1, gh1 = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind=kind,
                                   precision=prec, ckpt=7)
    g1 = np.concatenate([gp1, gh1])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, kind, prec, path, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=600) for _ in range(2)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    k = 0 if kind == "avg" else 1
    gmax = np.max(np.abs(g1))
    for _, F, gp, gh in res:
        g = np.concatenate([gp, gh])
        if prec == "fp64":
            assert abs(F[k] - F1[k]) < 1e-12
            assert np.max(np.abs(g - g1)) <= 1e-12 * gmax
        else:
            assert abs(F[k] - F1[k]) < 1e-5
            assert np.max(np.abs(g - g1)) <= 1e-4 * gmax
    # both shards return the same totals
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])


def test_sharded_solve_reports_a_failed_allreduce(sgctx):
    from paper_2406_18155_gb300.api import System
    from paper_2406_18155_gb300.capi import SGError, SG_E_STATE
    wl = _workload("state")
    s = System.from_workload(sgctx, wl)
    s.prepare()

    def broken(v):
        raise RuntimeError("peer gone")
    with pytest.raises(SGError) as e:
        s.fidelity_grad_sharded(wl["T"], wl["dt"], wl["target"], wl["col_index"][:4], broken, kind="state",
                                precision="fp64")
    assert e.value.code == SG_E_STATE
    # one shard holding every column with a local sum is the unsharded solve
    F1, gp1, gh1 = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="state",
                                   precision="fp64")
    F2, gp2, gh2 = s.fidelity_grad_sharded(wl["T"], wl["dt"], wl["target"], wl["col_index"], lambda v: v,
                                           kind="state", precision="fp64")
    assert abs(F1[1] - F2[1]) < 1e-13
    assert np.max(np.abs(gp1 - gp2)) <= 1e-12 * np.max(np.abs(gp1))
