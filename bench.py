#!/usr/bin/env python
"""Benchmark of the fidelity + adjoint-gradient solve on one GB300, or on N: by
default N independent replicas with their own seeds (weak scaling, no collective);
with --shard one gate's columns split over the N ranks, which sum their fidelity
terms and gradients over NCCL (strong scaling).

One bench step = one pass of the whole hot path on the workload: subsystem build
and eigensolve, stage tables, forward RK4 of every column with checkpoints,
fidelity, co-state, checkpointed discrete adjoint with fused cross-density
reductions, and the parameter chain.  Metric: state-column RK steps per second of
that solve (S columns x N steps per solve).

    python bench.py [--gpus N [--shard]] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...     # the FP64 CPU oracle as it stands
"""
import argparse
import json
import os

# one hardware work queue per concurrent stream (set before CUDA initialises; the
# package sets the same default)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

from paper_2406_18155_gb300 import workloads as W

METRIC = "state-column RK steps/s (fidelity + adjoint-gradient solve)"
UNIT = "col-steps/s"

WORKLOADS = {
    "fluxonium_ring10": ("10-fluxonium ring, 4 levels (D=1,048,576), 16 computational columns, "
                         "10 drives x 10 PWC segments, T=40 ns, dt=0.01 ns (N=4000)",
                         lambda seed: W.fluxonium_ring10(seed=seed)),
    "fluxonium_chain6": ("6-fluxonium chain, 4 levels (D=4096), 64 columns, 6 drives x 10 PWC "
                         "segments, T=60 ns, dt=0.01 ns (N=6000)",
                         lambda seed: W.fluxonium_chain6(seed=seed)),
    "fluxonium_pair_cr": ("2 fluxoniums, 5 levels (D=25), 4 columns, CR drive 20 PWC segments, "
                          "T=100 ns, dt=0.01 ns (N=10000)",
                          lambda seed: W.fluxonium_pair_cr(seed=seed)),
    "transmon_pair": ("2 transmons, 4 levels (D=16), 16 columns, Gaussian drive, T=50 ns, "
                      "dt=0.005 ns (N=10000)", lambda seed: W.transmon_pair(seed=seed)),
}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# algorithmic bytes per entry of each kernel family
# ----------------------------------------------------------------------------
# Minimal fused two-pass RK4 step on a slab that exceeds one tile (two overlapping
# mode groups per stage), bytes per entry and step: complex64 stages with the
# complex128 state 304, all complex128 448.  The forward stage pass's roofline uses
# this figure, one eighth of it per launch (four stages x two passes).
FWD_STEP_BYTES_TWO_PASS = {8: 304, 16: 448}


def fwd_bytes_per_entry_step(c, npass):
    """Forward RK4 step, bytes per slab entry: c = bytes of a stage value (8 mixed,
    16 FP64); the state psi is complex128 (16)."""
    p = 16
    if npass == 1:
        return (c + p + c + c) + 2 * (c + p + 2 * c + c) + (c + c + 2 * p + c)
    partial_first = 2 * c                      # read y, write kA
    partial_mid = 3 * c                        # read y, kA; write kA
    last_extra = c                             # read kA
    last = (c + p + c + c) + 2 * (c + p + 2 * c + c) + (c + c + 2 * p + c) + 4 * last_extra
    return 4 * (partial_first + (npass - 2) * partial_mid) + last


def adj_bytes_per_entry_step(c, npass):
    """Adjoint step (4 stage passes each reading kbar and y_s), bytes per entry."""
    p = 16
    reads = 2 * c                              # kbar tile, y_s tile per pass
    partial = [reads + c] + [reads + 2 * c] * max(0, npass - 2)
    last_extra = c if npass > 1 else 0
    st3 = reads + last_extra + p + c + c       # read pbar, write Db, Xn
    st21 = reads + last_extra + p + 2 * c + c  # Db read+write
    st0 = reads + last_extra + 2 * p + c + c   # pbar r+w, Db read, Xn
    part = sum(partial) if npass > 1 else 0
    return 4 * part + st3 + 2 * st21 + st0


def store_bytes_per_entry_step(c, npass):
    """Recompute of y2..y4 (3 stage passes, writes only the next stage input)."""
    p = 16
    if npass == 1:
        return 3 * (c + p + c)
    return 3 * (2 * c + (npass - 2) * 3 * c + (c + c + p + c))


def grad_set(args):
    """Gradient set of the configuration: the ring asks for its pulse segments,
    the others for every parameter."""
    if args.grad != "config":
        return args.grad
    return "pulse" if args.workload == "fluxonium_ring10" else "all"


def bench_config(args, wl, desc, world):
    """The workload description printed by both arms (identical by construction)."""
    S = len(wl["col_index"])
    N = int(round(wl["T"] / wl["dt"]))
    D = int(np.prod([m["levels"] for m in wl["modes"]]))
    return {"workload": f"{args.workload}: {desc}", "columns": S, "rk4_steps": N,
            "composite_dim": D, "precision": args.precision,
            "gradient": "pulse parameters" if grad_set(args) == "pulse"
            else "pulse and Hamiltonian parameters",
            "l2": "inputs larger than L2 (slab 128 MiB c64 / 256 MiB c128)"
            if D * S * 8 > 129e6 else "L2-resident working set; no flush",
            "parallelism": (f"one gate's columns sharded over {world} GPUs (NCCL sums of the fidelity terms "
                            "and gradients)" if world > 1 and getattr(args, "shard", False)
                            else f"{world} independent replica(s), one per GPU")}


def _json_num(x):
    """A float for the JSON line; None where it is undefined (NaN)."""
    x = float(x)
    return None if x != x else x


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    if rank == 0 or world > 1:
        from paper_2406_18155_gb300 import build as B
        B.build()
    from paper_2406_18155_gb300.api import Context, System, evolve_opts
    desc, make = WORKLOADS[args.workload]
    shard = world > 1 and args.shard
    wl = make(1000 if shard else 1000 + rank)      # one gate over all ranks, or one replica each
    if args.t_ns > 0:                     # shortened run (profiling captures)
        wl["T"] = round(args.t_ns / wl["dt"]) * wl["dt"]
        for d in wl["drives"]:
            d["length"] = wl["T"]
        desc += f" [shortened to T={wl['T']:.4g} ns]"
    ctx = Context(local)
    sysm = System.from_workload(ctx, wl)
    sysm.prepare()
    S = len(wl["col_index"])
    N = int(round(wl["T"] / wl["dt"]))
    D = int(np.prod([m["levels"] for m in wl["modes"]]))
    prec = args.precision
    stream = torch.cuda.current_stream(local)

    grad = grad_set(args)
    args.grad_set = grad

    if shard:
        # this rank's contiguous block of the gate's columns; the fidelity sums and the
        # gradients are summed over ranks through the library's callback (NCCL)
        from paper_2406_18155_gb300.shard import column_block, torch_allreduce
        c0, c1 = column_block(S, rank, world)
        red = torch_allreduce(device=f"cuda:{local}")

    def one_step(ham=(grad == "all")):
        sysm.prepare()
        if shard:
            return sysm.fidelity_grad_sharded(wl["T"], wl["dt"], wl["target"], wl["col_index"][c0:c1], red,
                                              kind=wl["fid_kind"], precision=prec, ckpt=args.ckpt, ham=ham)
        return sysm.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                  kind=wl["fid_kind"], precision=prec, ckpt=args.ckpt, ham=ham)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # ---- timed region: device time with CUDA events on the library's stream
    os.environ["SG_KTIMING"] = "1"
    clk = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    fam = np.zeros(9)
    fwd_ms, bwd_ms, peak = [], [], 0
    for _ in range(args.steps):
        F, gp, gh = one_step()
        st = sysm.last_stats()
        launches += st["launches"]
        fwd_ms.append(st["forward_ms"])
        bwd_ms.append(st["backward_ms"])
        peak = max(peak, st["peak_bytes"])
        kt = np.zeros(9)
        from paper_2406_18155_gb300.capi import lib
        import ctypes
        lib().sg_kernel_times(sysm.h, kt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 9)
        fam += kt
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    os.environ["SG_KTIMING"] = "0"
    t_s = ev0.elapsed_time(ev1) / 1e3
    if dist:
        tt = torch.tensor([t_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_s = float(tt.item())
    units = S * N * args.steps * (1 if shard else world)
    value = units / t_s

    # ---- end to end through the public call: host target in, host gradients out
    h2d = wl["target"].size * 16 + S * 8 + 8 * sum(len(d.get("amps", [0])) for d in wl["drives"])
    npul, nham = sysm.param_counts()
    d2h = 16 + 8 * (npul + nham)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        one_step()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    if dist:
        tt = torch.tensor([t_e2e], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    e2e_value = S * N * max(1, args.e2e_steps) * (1 if shard else world) / t_e2e

    out = None
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": t_s / args.steps * 1e3, "higher_is_better": True,
               "scaling": "strong" if shard else "weak", "vs_baseline": None,
               "dtype": "c64 stages, c128 state/co-state, f64 reductions" if prec == "mixed" else "c128",
               "data": "synthetic (seeded, shapes and value ranges of the paper's fluxonium workloads)",
               "config": bench_config(args, wl, desc, world),
               "forward_ms": statistics.mean(fwd_ms), "gradient_ms": statistics.mean(bwd_ms),
               "O_t": (statistics.mean(fwd_ms) + statistics.mean(bwd_ms)) / statistics.mean(fwd_ms),
               "peak_library_bytes": peak, "F": [_json_num(F[0]), _json_num(F[1])],
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h)},
               "gpu_launches": int(launches), "clocks": clocks}
        # ---- roofline of the dominant kernel family
        out["roofline"], out["kernel_families"] = roofline(fam, D, S, N, prec, sysm, args)
        if grad == "pulse" and args.full_gradient:
            # the same solve with the Hamiltonian-parameter gradient too (one run, for reference)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            one_step(ham=True)
            torch.cuda.synchronize()
            tf = time.perf_counter() - t0
            st = sysm.last_stats()
            out["full_gradient"] = {"col_steps_per_s": S * N / tf, "forward_ms": st["forward_ms"],
                                    "gradient_ms": st["backward_ms"],
                                    "note": "pulse + Hamiltonian parameters, one untimed-by-events run"}
        # ---- the plain FP64 GPU path on a bounded number of steps
        if args.fp64_steps > 0:
            out["fp64_vs_mixed"] = fp64_comparison(sysm, wl, args.fp64_steps, args.fp64_grad_steps,
                                                   grad == "all", stream)
        if args.q2 and D <= 4096:
            out["q2_vs_rk4"] = q2_comparison(sysm, wl, stream)
        elif args.q2:
            out["q2_vs_rk4"] = q2_tiled_comparison(sysm, wl, stream, args.q2_steps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_sample_steps)
    if rank == 0 and args.serving > 0:
        out["serving"] = serving_bench(ctx, args.serving, args.serving_slots, max_batch=args.serving_batch)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def onchip_shapes(ctx, nsteps, only=None):
    """Per shape class of the serving distribution (kind x modes x levels): one
    fidelity + gradient solve alone on the GPU, mixed precision, T = nsteps dt;
    forward and backward (segment replay + pull-back) device time per RK4 step."""
    from paper_2406_18155_gb300.api import System
    out, seen = [], set()
    for seed in range(20000):
        wl = W.serving_request(np.random.Generator(np.random.PCG64(seed)))
        if wl["name"] in seen or (only and wl["name"] != only):
            continue
        seen.add(wl["name"])
        wl["T"] = nsteps * wl["dt"]
        for d in wl["drives"]:
            d["length"] = wl["T"]
        s = System.from_workload(ctx, wl)
        s.prepare()
        for _ in range(2):
            s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg", precision="mixed")
        st = s.last_stats()
        D = int(np.prod([m["levels"] for m in wl["modes"]]))
        out.append({"shape": wl["name"], "D": D, "columns": len(wl["col_index"]),
                    "forward_us_per_step": round(1e3 * st["forward_ms"] / nsteps, 2),
                    "backward_us_per_step": round(1e3 * st["backward_ms"] / nsteps, 2),
                    "launches": st["launches"]})
        if len(seen) == 24 or only:
            break
    return sorted(out, key=lambda r: (r["D"], r["shape"]))


class UtilSampler:
    """Device utilisation (nvidia-smi utilization.gpu: the fraction of time a kernel was
    running) sampled every 200 ms while a serving stream runs."""

    def __init__(self, device):
        self.device, self.proc, self.vals = device, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", "--query-gpu=utilization.gpu",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            try:
                self.vals.append(float(line.strip()))
            except ValueError:
                pass

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return statistics.mean(self.vals) / 100.0 if self.vals else None


def serving_bench(ctx, n_requests, slots, seed=7, rates=(0.7,), n_saturated=None, max_batch=1):
    """Config 4: requests of 2-5 coupled transmons or fluxoniums at 3-5 levels,
    T ~ U[20, 200] ns, random 10-segment pulses, each a fidelity + gradient solve.
    First n_saturated requests (default 2 x n_requests) submitted at once: the
    saturated throughput is their count over the wall time until the last finishes
    (conservative: it includes the drain, when only the longest requests are left).
    Then, for each rate fraction, a stream of n_requests with Poisson arrivals at
    that fraction of the saturated rate: solves/s, p50/p99 latency (submit -> result)
    and the device utilisation sampled during the stream.  max_batch > 1: each slot
    packs queued same-shape requests into shared batched launches."""
    from paper_2406_18155_gb300.api import Server, System
    rng = np.random.Generator(np.random.PCG64(seed))

    def make(nr):
        out = []
        for _ in range(nr):
            wl = W.serving_request(rng)
            s_ = System.from_workload(ctx, wl)
            out.append((wl, s_))
        return out

    srv = Server(ctx, mem_budget_bytes=120 << 30, max_slots=slots, max_batch=max_batch)
    sat = make(max(4, n_saturated or 2 * n_requests))
    t0 = time.perf_counter()
    tk = [srv.submit(s_, wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg") for wl, s_ in sat]
    sat_res = [srv.wait(t) for t in tk]
    sat_rate = len(sat) / (time.perf_counter() - t0)
    sat_st = srv.stats()
    srv.close()
    del sat
    out = {"saturated_solves_per_s": sat_rate, "saturated_requests": len(sat_res), "slots": slots,
           "max_batch": max_batch, "saturated_errors": int(sum(r["status"] != 0 for r in sat_res)),
           "saturated_packing": {k: sat_st[k] for k in ("batches", "batched_requests", "batched_launches",
                                                          "batched_launch_members")},
           "streams": []}
    for frac in rates:
        srv = Server(ctx, mem_budget_bytes=120 << 30, max_slots=slots, max_batch=max_batch)
        reqs = make(n_requests)
        rate = frac * sat_rate
        gaps = rng.exponential(1.0 / rate, size=len(reqs))
        util = UtilSampler(ctx.device)
        util.start()
        t0 = time.perf_counter()
        tk = []
        next_t = 0.0
        for (wl, s_), g in zip(reqs, gaps):
            next_t += g
            dly = next_t - (time.perf_counter() - t0)
            if dly > 0:
                time.sleep(dly)
            tk.append(srv.submit(s_, wl["T"], wl["dt"], wl["target"], wl["col_index"], kind="avg"))
        res = [srv.wait(t) for t in tk]
        wall = time.perf_counter() - t0
        u = util.stop()
        lat = np.array([r["done_s"] - r["submit_s"] for r in res])
        st_ = srv.stats()
        srv.close()
        steps = np.array([int(round(wl["T"] / wl["dt"])) for wl, _ in reqs])
        out["streams"].append({
            "rate_fraction": frac, "arrival_rate_per_s": rate, "requests": len(reqs),
            "solves_per_s": len(reqs) / wall, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "device_utilisation": u,
            "errors": int(sum(r["status"] != 0 for r in res)), "mean_rk4_steps": float(steps.mean()),
            "packing": {k: st_[k] for k in ("batches", "batched_requests", "batched_launches",
                                            "batched_launch_members")}})
        del reqs
    # the first stream's figures at the top level, as before
    st0 = out["streams"][0]
    out.update({"requests": st0["requests"], "arrival_rate_per_s": st0["arrival_rate_per_s"],
                "solves_per_s": st0["solves_per_s"], "p50_s": st0["p50_s"], "p99_s": st0["p99_s"],
                "errors": st0["errors"], "device_utilisation": st0["device_utilisation"],
                "sample": f"{len(sat_res)} requests submitted at once, then {n_requests} Poisson arrivals of the "
                          f"serving distribution at each of {list(rates)} x the saturated rate (the full stream "
                          "is 10k requests), fidelity + gradient each"})
    return out


def dense_comparison(ctx, nsys, onchip_sys, threads=32):
    """Configs 1-2 shapes (transmon pair D = 16, 16 columns; fluxonium CR pair D = 25,
    4 columns; full horizons, 10^4 steps) as batches of systems of different seeds:
    the tensor-core batch (sg_evolve_batch, 3xTF32) against the on-chip kernels
    (sg_evolve, mixed) for one system alone and for many systems at once (the on-chip
    solves issued from `threads` host threads, each with its own context and stream).
    Device time of the batch launch; wall time of the concurrent on-chip solves."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_2406_18155_gb300.api import Context, System, evolve_batch
    out = {}
    for name, make in (("transmon_pair_d16", lambda sd: W.transmon_pair(seed=sd)),
                       ("fluxonium_pair_cr_d25", lambda sd: W.fluxonium_pair_cr(seed=sd))):
        wls = [make(sd) for sd in range(nsys)]
        S, N = len(wls[0]["col_index"]), int(round(wls[0]["T"] / wls[0]["dt"]))
        sys_ = []
        for wl in wls:
            s_ = System.from_workload(ctx, wl)
            s_.prepare()
            sys_.append(s_)
        r = {"columns": S, "rk4_steps": N}
        for B in (1, nsys):
            evolve_batch(sys_[:B], wls[0]["T"], wls[0]["dt"], wls[0]["col_index"])      # warm
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            evolve_batch(sys_[:B], wls[0]["T"], wls[0]["dt"], wls[0]["col_index"])
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            r[f"tensor_batch_{B}_wall_s"] = wall
            r[f"tensor_batch_{B}_col_steps_per_s"] = B * S * N / wall
        # on-chip, one system alone
        sys_[0].evolve(wls[0]["T"], wls[0]["dt"], precision="mixed", col_index=wls[0]["col_index"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sys_[0].evolve(wls[0]["T"], wls[0]["dt"], precision="mixed", col_index=wls[0]["col_index"])
        torch.cuda.synchronize()
        r["onchip_1_wall_s"] = time.perf_counter() - t0
        r["onchip_1_col_steps_per_s"] = S * N / r["onchip_1_wall_s"]
        # on-chip, many systems at once from several host threads
        M = min(onchip_sys, nsys)
        per = [list(range(k, M, threads)) for k in range(threads)]
        ctxs = [Context(ctx.device, stream=torch.cuda.Stream(ctx.device)) for _ in range(threads)]
        loc = []
        for k in range(threads):
            row = []
            for idx in per[k]:
                s_ = System.from_workload(ctxs[k], wls[idx])
                s_.prepare()
                row.append((s_, wls[idx]))
            loc.append(row)

        def work(k):
            for s_, wl in loc[k]:
                s_.evolve(wl["T"], wl["dt"], precision="mixed", col_index=wl["col_index"])
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, range(threads)))                  # warm
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            list(ex.map(work, range(threads)))
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        r[f"onchip_{M}_concurrent_wall_s"] = wall
        r[f"onchip_{M}_concurrent_col_steps_per_s"] = M * S * N / wall
        r["tensor_over_onchip_throughput"] = r[f"tensor_batch_{nsys}_col_steps_per_s"] / r[
            f"onchip_{M}_concurrent_col_steps_per_s"]
        for c in ctxs:
            c.close()
        out[name] = r
    return out


def slab_passes(D):
    # plans used by the tiled kernels: one pass while a column fits one tile
    # (4096 entries), two overlapping mode groups for the ring beyond that
    return 1 if D <= 4096 else 2


def roofline(fam, D, S, N, prec, sysm, args):
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    src = "of measured" if "hbm_gbs" in peaks else "of fallback"
    c = 8 if prec == "mixed" else 16
    npass = slab_passes(D)
    E = D * S
    fwd_step = FWD_STEP_BYTES_TWO_PASS[c] if npass == 2 else fwd_bytes_per_entry_step(c, npass)
    per_step = {"forward_stage_pass": fwd_step,
                "adjoint_stage_pass": adj_bytes_per_entry_step(c, npass),
                "recompute_stage_pass": store_bytes_per_entry_step(c, npass)}
    launches_per_step = {"forward_stage_pass": 4 * npass, "adjoint_stage_pass": 4 * npass,
                         "recompute_stage_pass": 3 * npass}
    fams = {}
    for k, name in enumerate(["forward_stage_pass", "adjoint_stage_pass", "recompute_stage_pass"]):
        ms, nl, tot = fam[3 * k], fam[3 * k + 1], fam[3 * k + 2]
        if nl <= 0:
            continue
        avg_ms = ms / nl
        bytes_per_launch = per_step[name] * E / launches_per_step[name]
        fams[name] = {"avg_launch_ms": avg_ms, "launches": int(tot),
                      "est_total_ms": avg_ms * tot,
                      "algorithmic_bytes_per_launch": bytes_per_launch,
                      "achieved_gbs": bytes_per_launch / (avg_ms * 1e-3) / 1e9}
    if not fams:
        return None, fams
    dom = max(fams, key=lambda k: fams[k]["est_total_ms"])
    f = fams[dom]
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tf):
        with open(tf) as fh:
            t = json.load(fh)
        key = f"{args.workload}:{prec}:{getattr(args, 'grad_set', 'all')}:{dom}"
        if key in t:
            traffic = t[key]
    return ({"bound": "hbm", "kernel": dom, "achieved": f["achieved_gbs"], "peak": hbm,
             "unit": "GB/s", "frac": f["achieved_gbs"] / hbm, "peak_source": src,
             "traffic": traffic,
             "bytes_per_entry_step": per_step[dom], "launches_per_step": launches_per_step[dom]}, fams)


def _normalised_target(wl, psi):
    """Target whose column for each evolved computational state is that column's
    normalised computational rows in psi: F_state is then close to 1, so a
    difference in F is a difference in infidelity."""
    dims = [m["levels"] for m in wl["modes"]]
    comp = W.comp_states(dims)
    lab = {r: j for j, r in enumerate(comp)}
    T = np.zeros((len(comp), len(comp)), dtype=np.complex128)
    for s_, r in enumerate(wl["col_index"]):
        if r in lab:
            v = psi[comp, s_]
            T[:, lab[r]] = v / max(np.linalg.norm(v), 1e-300)
    return T


def _timed(stream, fn):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1) / 1e3


def fp64_comparison(sysm, wl, nsteps, grad_steps, ham, stream):
    """The plain FP64 GPU path against the mixed one on the same workload and
    columns, device time of the public calls after a warm call:
      forward  - sg_evolve over the first nsteps steps; the mixed result's largest
                 amplitude error against FP64;
      gradient - sg_fidelity_grad over the first grad_steps steps (the
                 configuration's gradient set) with the FP64 forward's normalised
                 computational rows as target (F_state close to 1); |dF| and the
                 gradient error relative to its largest component."""
    S = len(wl["col_index"])
    out = {"steps": nsteps}
    psi = {}
    for prec in ("fp64", "mixed"):
        T = nsteps * wl["dt"]
        sysm.evolve(T, wl["dt"], precision=prec, col_index=wl["col_index"])   # warm
        p, t = _timed(stream, lambda: sysm.evolve(T, wl["dt"], precision=prec, col_index=wl["col_index"]))
        psi[prec] = p.cpu().numpy()
        out[f"{prec}_forward_col_steps_per_s"] = S * nsteps / t
    out["mixed_over_fp64"] = out["mixed_forward_col_steps_per_s"] / out["fp64_forward_col_steps_per_s"]
    out["max_abs_dpsi"] = float(np.max(np.abs(psi["mixed"] - psi["fp64"])))
    if grad_steps > 0:
        Tg = grad_steps * wl["dt"]
        p64 = sysm.evolve(Tg, wl["dt"], precision="fp64", col_index=wl["col_index"]).cpu().numpy()
        target = _normalised_target(wl, p64)
        g = {"steps": grad_steps, "gradient": "pulse and Hamiltonian parameters" if ham else "pulse parameters"}
        res = {}
        for prec in ("fp64", "mixed"):
            call = lambda: sysm.fidelity_grad(Tg, wl["dt"], target, wl["col_index"], kind="state",
                                              precision=prec, ham=ham)
            call()                                                            # warm
            (F, gp, gh), t = _timed(stream, call)
            res[prec] = (F, np.concatenate([gp, gh]) if ham else gp)
            g[f"{prec}_col_steps_per_s"] = S * grad_steps / t
        g["mixed_over_fp64"] = g["mixed_col_steps_per_s"] / g["fp64_col_steps_per_s"]
        g["F_state_fp64"] = float(res["fp64"][0][1])
        g["abs_dF_state"] = abs(float(res["mixed"][0][1]) - float(res["fp64"][0][1]))
        gm = np.max(np.abs(res["fp64"][1]))
        g["rel_dgrad"] = float(np.max(np.abs(res["mixed"][1] - res["fp64"][1])) / max(gm, 1e-300))
        out["gradient"] = g
    return out


def q2_tiled_comparison(sysm, wl, stream, nsteps):
    """The paper's Suzuki-Trotter products on the tiled kernels (slabs beyond the
    on-chip kernels) against RK4 over the first nsteps steps of the workload:
    forward col-steps/s (device time) of RK4 (mixed), Q2 (mixed, FP64) and Q4 (mixed),
    the largest difference of the Q2 and Q4 states from RK4's (each solver's own
    truncation error at the workload's dt), and the pulse-gradient solves of RK4 and
    Q2 (mixed)."""
    import torch
    T = nsteps * wl["dt"]
    out = {"steps": nsteps}
    psi = {}
    for solver, prec in (("rk4", "mixed"), ("q2", "mixed"), ("q2", "fp64"), ("q4", "mixed")):
        kw = dict(precision=prec, col_index=wl["col_index"], solver=solver)
        sysm.evolve(T, wl["dt"], **kw)                                   # warm
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = sysm.evolve(T, wl["dt"], **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        out[f"{solver}_{prec}_forward_col_steps_per_s"] = len(wl["col_index"]) * nsteps / (e0.elapsed_time(e1) / 1e3)
        if prec == "mixed":
            psi[solver] = r.cpu().numpy()
    out["q2_over_rk4_mixed"] = out["q2_mixed_forward_col_steps_per_s"] / out["rk4_mixed_forward_col_steps_per_s"]
    out["max_abs_dpsi_q2_rk4"] = float(np.max(np.abs(psi["q2"] - psi["rk4"])))
    out["max_abs_dpsi_q4_rk4"] = float(np.max(np.abs(psi["q4"] - psi["rk4"])))
    # pulse-gradient solves (fidelity + adjoint) over the same steps: RK4's checkpointed
    # adjoint against Q2's pull-back through inverse factors on the tiles
    for solver in ("rk4", "q2"):
        kw = dict(kind=wl["fid_kind"], precision="mixed", ham=False, solver=solver)
        sysm.fidelity_grad(T, wl["dt"], wl["target"], wl["col_index"], **kw)          # warm
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sysm.fidelity_grad(T, wl["dt"], wl["target"], wl["col_index"], **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        out[f"{solver}_mixed_pulse_gradient_col_steps_per_s"] = len(wl["col_index"]) * nsteps / (e0.elapsed_time(e1) / 1e3)
    return out


def q2_comparison(sysm, wl, stream):
    """The paper's Suzuki-Trotter solvers (Q2, Q4, Q4j) against RK4 on the whole
    workload (single-tile systems only): forward and pulse-gradient col-steps/s of
    each in FP64 and mixed precision (device time), and the fidelity differences at
    the workload's dt."""
    import torch
    out = {}
    for solver in ("rk4", "q2", "q4", "q4j"):
        for prec in ("fp64", "mixed"):
            kw = dict(precision=prec, col_index=wl["col_index"], solver=solver)
            sysm.evolve(wl["T"], wl["dt"], **kw)                          # warm
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sysm.evolve(wl["T"], wl["dt"], **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            out[f"{solver}_{prec}_forward_col_steps_per_s"] = len(wl["col_index"]) * round(wl["T"] / wl["dt"]) / t
    # pulse-parameter gradient solves (fidelity + adjoint), each solver in the frame
    # it runs in; a solve the plan cannot hold is reported as null
    from paper_2406_18155_gb300.capi import SGError
    gq = {}
    for solver in ("rk4", "q2", "q4"):
        for prec in ("fp64", "mixed"):
            kw = dict(kind=wl["fid_kind"], precision=prec, ham=False, solver=solver,
                      frame="lab" if solver == "q2" else wl.get("frame", "interaction"))
            key = f"{solver}_{prec}_pulse_gradient_col_steps_per_s"
            try:
                sysm.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], **kw)   # warm
            except SGError as e:
                out[key] = None
                out[f"{solver}_{prec}_pulse_gradient_unsupported"] = str(e)[:120]
                continue
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, gp, _ = sysm.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"], **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            out[key] = len(wl["col_index"]) * round(wl["T"] / wl["dt"]) / (e0.elapsed_time(e1) / 1e3)
            if prec == "mixed":
                gq[solver] = gp
    for sv in ("q2", "q4"):
        if sv in gq and "rk4" in gq:
            out[f"rel_dgrad_{sv}_vs_rk4_mixed"] = float(np.max(np.abs(gq[sv] - gq["rk4"])) /
                                                        max(1e-300, np.max(np.abs(gq["rk4"]))))
    F = {sv: sysm.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision="fp64", solver=sv)
         for sv in ("rk4", "q2", "q4", "q4j")}
    k = 0 if wl["fid_kind"] == "avg" else 1
    for sv in ("rk4", "q2", "q4", "q4j"):
        out[f"fidelity_{sv}_fp64"] = float(F[sv][k])
    for sv in ("q2", "q4", "q4j"):
        out[f"abs_dF_{sv}_vs_rk4"] = abs(float(F[sv][k]) - float(F["rk4"][k]))
    return out


_W_SYS = None


def _oracle_worker_init(wl):
    """Pool worker: the oracle's system of the workload, built once per process."""
    global _W_SYS
    from oracle.system import OracleSystem
    _W_SYS = OracleSystem(wl)


def _oracle_worker_run(job):
    col, nsteps = job
    from oracle.evolve import initial_columns, rk4_evolve_matrix_free
    rk4_evolve_matrix_free(_W_SYS, initial_columns(_W_SYS, [col]), nsteps=nsteps)
    return col


class OraclePool:
    """The FP64 oracle's matrix-free RK4 forward on the host cores: one spawned
    process per core (numpy.einsum without path optimisation runs on one thread),
    each evolving whole columns of the workload."""

    def __init__(self, wl, cores):
        import multiprocessing as mp
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        self.cores = max(1, cores)
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init,
                                                 initargs=(wl,))
        self.pool.map(_oracle_worker_run, [(wl["col_index"][0], 0)] * self.cores)   # start-up

    def run(self, cols, nsteps):
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker_run, [(c, nsteps) for c in cols], chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(wl, nsteps, repeats=3):
    """The FP64 oracle as it stands on this host, forward part of the step only
    (its adjoint forms dense D x D matrices and cannot run at D = 2^20): the
    matrix-free RK4 of nsteps steps, on one core (one column) and on every core
    (as many columns as cores, at most the workload's), each the best of
    `repeats` runs."""
    from oracle.evolve import initial_columns, rk4_evolve_matrix_free
    from oracle.system import OracleSystem
    s = OracleSystem(wl)
    one = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        rk4_evolve_matrix_free(s, initial_columns(s, wl["col_index"][:1]), nsteps=nsteps)
        one.append(nsteps / (time.perf_counter() - t0))
    cores = min(os.cpu_count() or 1, len(wl["col_index"]))
    pool = OraclePool(wl, cores)
    cols = wl["col_index"][:cores]
    allc = [len(cols) * nsteps / pool.run(cols, nsteps) for _ in range(repeats)]
    pool.close()
    return {"value": max(allc), "unit": UNIT, "cores": cores, "kind": "oracle",
            "one_core": {"value": max(one), "cores": 1},
            "sample": f"forward only: matrix-free FP64 RK4, {nsteps} steps of {len(cols)} of the "
                      f"{len(wl['col_index'])} columns, one process per core; best of {repeats} "
                      f"(one core: 1 column, {max(one):.3g} col-steps/s). The oracle's adjoint forms "
                      "dense D x D matrices and cannot run at this D"}


# ----------------------------------------------------------------------------
# reference arm: the oracle as it stands, on the host cores
# ----------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    desc, make = WORKLOADS[args.workload]
    wl = make(1000)
    cores = min(os.cpu_count() or 1, len(wl["col_index"]))
    pool = OraclePool(wl, cores)
    cols = wl["col_index"][:cores]
    ns = args.ref_sample_steps
    for _ in range(args.warmup):
        pool.run(cols, ns)
    tot = 0.0
    for _ in range(args.steps):
        tot += pool.run(cols, ns)
    pool.close()
    units = len(cols) * ns * args.steps
    v = units / tot
    sample = (f"forward only: matrix-free FP64 RK4, {ns} step(s) of {len(cols)} "
              f"of the {len(wl['col_index'])} columns per step, one process per core; the "
              "oracle's adjoint forms dense D x D matrices and cannot run at this D")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": bench_config(args, wl, desc, world),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fluxonium_ring10", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--ckpt", type=int, default=0)
    ap.add_argument("--shard", action="store_true",
                    help="with N > 1 GPUs: shard one gate's columns over the ranks (strong scaling) "
                         "instead of running one replica per GPU")
    ap.add_argument("--fp64-steps", type=int, default=64,
                    help="forward steps of the FP64-vs-mixed comparison (0: skip)")
    ap.add_argument("--fp64-grad-steps", type=int, default=64,
                    help="steps of the FP64-vs-mixed gradient-solve comparison (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-sample-steps", type=int, default=2,
                    help="RK4 steps per column of the oracle sample beside our line")
    ap.add_argument("--ref-sample-steps", type=int, default=1,
                    help="RK4 steps per column of each reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", type=int, default=64, help="Poisson requests of the serving sample (0: skip); twice as many run saturated first")
    ap.add_argument("--serving-slots", type=int, default=32)
    ap.add_argument("--serving-batch", type=int, default=1,
                    help="per slot, pack up to this many queued same-shape requests into shared launches")
    ap.add_argument("--serving-rates", default="0.7",
                    help="arrival rates as fractions of the saturated rate, comma-separated")
    ap.add_argument("--serving-saturated", type=int, default=0,
                    help="requests of the saturated sample (default 2 x --serving)")
    ap.add_argument("--only-serving", action="store_true", help="print just the serving sample")
    ap.add_argument("--dense", type=int, default=0,
                    help="compare the tensor-core batch with the on-chip kernels on this many systems of the "
                         "config-1 and config-2 shapes and exit")
    ap.add_argument("--dense-onchip", type=int, default=512,
                    help="systems of the concurrent on-chip comparison (with --dense)")
    ap.add_argument("--t-ns", type=float, default=0.0, help="shorten the workload to T ns (profiling)")
    ap.add_argument("--q2", action="store_true",
                    help="also time the Suzuki-Trotter solvers against RK4 (beyond D = 4096: tiled, forward)")
    ap.add_argument("--q2-steps", type=int, default=400,
                    help="steps of the tiled Suzuki-Trotter comparison")
    ap.add_argument("--grad", default="config", choices=["config", "pulse", "all"],
                    help="gradient set: the configuration's (ring: pulse segments), pulse only, or all")
    ap.add_argument("--no-full-gradient", dest="full_gradient", action="store_false",
                    help="skip the reference run with the Hamiltonian gradient too")
    ap.add_argument("--onchip-shapes", type=int, default=0,
                    help="print per-shape on-chip step times over this many RK4 steps and exit")
    ap.add_argument("--shape", default=None, help="with --onchip-shapes: one shape class only")
    args = ap.parse_args()
    if args.onchip_shapes > 0:
        import torch
        from paper_2406_18155_gb300 import build as B
        B.build()
        from paper_2406_18155_gb300.api import Context
        torch.cuda.set_device(0)
        for r in onchip_shapes(Context(0), args.onchip_shapes, args.shape):
            print(json.dumps(r), flush=True)
    elif args.dense > 0:
        import torch
        from paper_2406_18155_gb300 import build as B
        B.build()
        from paper_2406_18155_gb300.api import Context
        torch.cuda.set_device(0)
        print(json.dumps({"dense_tensor_vs_onchip": dense_comparison(Context(0), args.dense, args.dense_onchip)}),
              flush=True)
    elif args.only_serving:
        import torch
        from paper_2406_18155_gb300 import build as B
        B.build()
        from paper_2406_18155_gb300.api import Context
        torch.cuda.set_device(0)
        rates = tuple(float(x) for x in args.serving_rates.split(","))
        print(json.dumps({"serving": serving_bench(Context(0), args.serving, args.serving_slots, rates=rates,
                                                   n_saturated=args.serving_saturated or None,
                                                   max_batch=args.serving_batch)}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
