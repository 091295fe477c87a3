"""Two CPU ranks (gloo) split the columns of one solve into contiguous blocks; the
overlap terms and the gradient partials are summed over ranks and must equal the
single-process result.  The per-rank engine is the FP64 oracle."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2406_18155_gb300 import workloads as W
from paper_2406_18155_gb300.shard import column_block, allreduce_sum, allreduce_max


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, wl, out):
    from oracle.evolve import (initial_columns, rk4_evolve, frame_epilogue, comp_map,
                               adjoint_from_costate)
    from oracle.system import OracleSystem
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cols = wl["col_index"]
    a, b = column_block(len(cols), rank, world)
    local = dict(wl, col_index=cols[a:b])
    s = OracleSystem(local)
    psiT, hist = rk4_evolve(s, initial_columns(s, local["col_index"]), store=True)
    psi_lab = frame_epilogue(s, psiT)
    comp, labels = comp_map(s)
    T = np.asarray(wl["target"])
    z = sum(np.vdot(T[:, labels[j]], psi_lab[comp, j]) for j in range(b - a) if labels[j] >= 0)
    nc = sum(1 for j in range(b - a) if labels[j] >= 0)
    terms = allreduce_sum(torch.tensor([np.real(z), np.imag(z), float(nc)], dtype=torch.float64))
    zg = complex(terms[0].item(), terms[1].item())
    S = terms[2].item()
    F = abs(zg / S) ** 2
    bar = np.zeros_like(psi_lab)
    for j in range(b - a):
        if labels[j] >= 0:
            bar[comp, j] = (2.0 * zg / S ** 2) * T[:, labels[j]]
    g, _ = adjoint_from_costate(s, hist, psi_lab, bar, s.N)
    g = allreduce_sum(torch.tensor(g, dtype=torch.float64))
    tmax = allreduce_max(1.0 + rank)
    if rank == 0:
        out.put((F, g.numpy(), tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_column_blocks_partition_the_columns():
    for n in (1, 5, 16, 17):
        for w in (1, 2, 3, 8):
            blocks = [column_block(n, r, w) for r in range(w)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (a0, b0), (a1, b1) in zip(blocks, blocks[1:]):
                assert b0 == a1
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def test_two_rank_sharded_solve_equals_single_process():
    from oracle import adjoint_gradient
    wl = W.fluxonium_chain(seed=8, nq=3, levels=3, T=0.2, dt=0.01, nseg=2, ring=True)
    F1, g1, _ = adjoint_gradient(wl)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, wl, q)) for r in range(2)]
    for p in procs:
        p.start()
    F2, g2, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert abs(F1 - F2) < 1e-13
    assert np.max(np.abs(g1 - g2)) < 1e-12 * max(1.0, np.max(np.abs(g1)))
    assert tmax == 2.0
