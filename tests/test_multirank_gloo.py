"""Two CPU ranks (gloo) split the columns of one solve into contiguous blocks; the
overlap sums {Re z, Im z, q, S_c} and the gradient partials are summed over ranks
with the same callback the library's sharded solve uses (shard.torch_allreduce), and
F_state, F_avg and the gradient must equal the single-process result.  The per-rank
engine is the FP64 oracle, so these tests check the sharded formulas themselves:
F_state = |z/S_c|^2, F_avg = (q + |z|^2)/(D_c(D_c+1)), and the co-states built from
the summed z."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2406_18155_gb300 import workloads as W
from paper_2406_18155_gb300.shard import column_block, torch_allreduce, allreduce_max


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, wl, kind, out):
    from oracle.evolve import (initial_columns, rk4_evolve, frame_epilogue, comp_map,
                               adjoint_from_costate)
    from oracle.system import OracleSystem
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    red = torch_allreduce()
    cols = wl["col_index"]
    a, b = column_block(len(cols), rank, world)
    local = dict(wl, col_index=cols[a:b])
    s = OracleSystem(local)
    psiT, hist = rk4_evolve(s, initial_columns(s, local["col_index"]), store=True)
    psi_lab = frame_epilogue(s, psiT)
    comp, labels = comp_map(s)
    T = np.asarray(wl["target"])
    Dc = T.shape[0]
    mine = [j for j in range(b - a) if labels[j] >= 0]
    m = {j: T.conj().T @ psi_lab[comp, j] for j in mine}            # T^dag u_s
    z = sum(m[j][labels[j]] for j in mine)
    q = sum(np.vdot(m[j], m[j]).real for j in mine)
    tot = red(np.array([z.real, z.imag, q, float(len(mine))]))
    zg, qg, S = complex(tot[0], tot[1]), tot[2], tot[3]
    F = abs(zg / S) ** 2 if kind == "state" else (qg + abs(zg) ** 2) / (Dc * (Dc + 1))
    bar = np.zeros_like(psi_lab)
    for j in mine:
        t = T[:, labels[j]]
        if kind == "state":
            bar[comp, j] = (2.0 * zg / S ** 2) * t
        else:
            bar[comp, j] = 2.0 * (T @ m[j] + zg * t) / (Dc * (Dc + 1))
    g, _ = adjoint_from_costate(s, hist, psi_lab, bar, s.N)
    g = red(g)
    tmax = allreduce_max(1.0 + rank)
    if rank == 0:
        out.put((F, g, tmax))
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


@pytest.mark.parametrize("kind", ["state", "avg"])
def test_two_rank_sharded_solve_equals_single_process(kind):
    from oracle import adjoint_gradient
    wl = W.fluxonium_chain(seed=8, nq=3, levels=3, T=0.2, dt=0.01, nseg=2, ring=True)
    if kind == "avg":
        wl["col_index"] = W.comp_states([3, 3, 3])           # every computational state once
        wl["target"] = W.haar_unitary(8, np.random.Generator(np.random.PCG64(3)))
    F1, g1, _ = adjoint_gradient(wl, kind=kind)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, wl, kind, q)) for r in range(2)]
    for p in procs:
        p.start()
    F2, g2, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert abs(F1 - F2) < 1e-13
    assert np.max(np.abs(g1 - g2)) < 1e-12 * max(1.0, np.max(np.abs(g1)))
    assert tmax == 2.0
