#!/usr/bin/env python
"""Benchmark of the multiple-double least-squares path on GB300.

Metric: md QR+backsub TFLOPS (paper op counts) at dd/qd/od -- the md operations
of the unblocked Householder least-squares method (QR of [A | b], then back
substitution) converted to double-precision flops with Table 1 of
arXiv 2110.08375, divided by the device time.

Workload (one "step"): the dense least-squares solve m = n = 1024, tile 128
(eight tiles), in double double, quad double and octo double, entries of A and
b ~ U[-1,1) per limb recipe, seed 0.  Inputs are resident in HBM before the
timed region; L2 (129 MB) is flushed between steps by writing a 256 MiB
buffer outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun) every rank solves its own replica of the workload (the
single solve does not shard); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "md QR+backsub TFLOPS (paper op counts) at dd/qd/od"
PREC_NAMES = {2: "dd", 4: "qd", 8: "od"}
TOL = {2: 1e-24, 4: 1e-55, 8: 1e-112}   # relative error of x against the oracle
FP64_PEAK_TOPS = 2 * 152 * 2.07e9 / 1e12   # FP64 pipe: 2 instructions/clk/SM x 152 SMs x 2.07 GHz
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the
# dominant kernel (profiles/gemm_kernel_od_trailing_n1024.md): 60.3 MB + 7.0 MB
TRAFFIC_BYTES = 67.24e6
TRAFFIC_LAUNCH = ("gemm_kernel<8, ViewDenseT, ViewDense>, X = W^T C of tile 0 beyond the next tile's columns "
                  "(128 x 769, K 1024 in four chunks): algorithmic 65.1e6 bytes")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mdls", choices=["mdls", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--tile", type=int, default=128)
    ap.add_argument("--precs", default="2,4,8")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-modes", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--no-backsub", action="store_true")
    ap.add_argument("--no-config0", action="store_true")
    ap.add_argument("--no-qr", action="store_true")
    ap.add_argument("--no-modes-large", action="store_true")
    ap.add_argument("--no-complex", action="store_true")
    ap.add_argument("--no-toeplitz", action="store_true")
    ap.add_argument("--bs-n", type=int, default=17920, help="size of the back-substitution entry")
    ap.add_argument("--bs-tile", type=int, default=128)
    ap.add_argument("--only-backsub", action="store_true",
                    help="time only the back-substitution entry (a small case for profiling)")
    ap.add_argument("--bs-sweep", action="store_true",
                    help="add the back-substitution grid: quad double, n x tile")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "mdls" else "gloo"
        if args.impl == "mdls":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples (every 200 ms) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(self.rows), "reasons": reasons}


def workload_flops(precs, n):
    from paper_2110_08375_gb300 import opcount
    return {p: opcount.lstsq_table1_flops(p, n, n) for p in precs}


# md mul-add pairs of the paper's blocked QR at m = n, tile 128, back-solved
# from its own timings and TFLOPS figures (context only: the algorithmic
# count of the unblocked method, used for `value`, is about (4/3) n^3 mul-add
# pairs, 14-17x fewer).
PAPER_QR_PAIRS = {512: 2.55e9, 1024: 2.395e10, 1536: 7.48e10, 2048: 1.70e11}


def paper_equivalent(precs, n, per_prec_ms, steps):
    """TFLOPS in the paper's own counting (QR mul-add pairs x Table-1 add+mul
    flops / time of the least-squares solve), for comparison with its tables
    only."""
    if n not in PAPER_QR_PAIRS:
        return None
    from paper_2110_08375_gb300 import opcount
    out = {"note": "paper-equivalent op count (back-solved from the paper's timings), context only"}
    for p in precs:
        sig = opcount.TABLE1_SIGMA[p]
        out[PREC_NAMES[p]] = PAPER_QR_PAIRS[n] * (sig["add"] + sig["mul"]) / (per_prec_ms[p] / steps / 1e3) / 1e12
    return out


def cpu_baseline(n_sample: int, precs, seed: int = 0, single_core: bool = True) -> dict:
    """The oracle (plain C, OpenMP) on a bounded sample of the workload: the
    leading n_sample x n_sample block of each precision's A and the leading
    n_sample entries of b, solved in every precision."""
    import oracle
    import synth
    from paper_2110_08375_gb300 import opcount
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    flops = 0
    t0 = time.perf_counter()
    for p in precs:
        A, b = synth.lstsq_problem(p, 1024, 1024, seed=seed, tag="cfg1")
        As = A[:, :n_sample, :n_sample].copy()
        bs = b[:, :n_sample].copy()
        oracle.lstsq(As, bs)
        flops += opcount.lstsq_table1_flops(p, n_sample, n_sample)
    dt = time.perf_counter() - t0
    out = {"value": flops / dt / 1e12, "unit": "TFLOPS", "cores": cores, "kind": "oracle",
           "sample": f"lstsq of the leading {n_sample}x{n_sample} block of the n=1024 inputs, "
                     f"precisions {','.join(PREC_NAMES[p] for p in precs)}; {dt:.1f} s",
           "seconds": dt}
    if not single_core:
        return out
    # the same oracle on one core, on a smaller block (its time grows as n^3)
    n1 = max(16, n_sample * 5 // 14)
    oracle.set_threads(1)
    flops1 = 0
    t1 = time.perf_counter()
    for p in precs:
        A, b = synth.lstsq_problem(p, 1024, 1024, seed=seed, tag="cfg1")
        oracle.lstsq(A[:, :n1, :n1].copy(), b[:, :n1].copy())
        flops1 += opcount.lstsq_table1_flops(p, n1, n1)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    out["single_core"] = {"value": flops1 / dt1 / 1e12, "unit": "TFLOPS", "cores": 1,
                          "sample": f"lstsq of the leading {n1}x{n1} block, same precisions; {dt1:.1f} s"}
    return out


def run_reference(args):
    rank, world, _ = dist_setup(args)
    precs = [int(x) for x in args.precs.split(",")]
    if rank != 0:
        barrier(world)
        return
    n_sample = 256
    for _ in range(args.warmup):
        cpu_baseline(n_sample, precs, single_core=False)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        r = cpu_baseline(n_sample, precs, single_core=False)
        vals.append(r["value"])
        secs += r["seconds"]
    value = statistics.mean(vals)
    cb = dict(r)
    cb["value"] = value
    cb.pop("seconds", None)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"lstsq sample {n_sample}x{n_sample} of m=n={args.n}, dd/qd/od, seed 0",
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "TFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    barrier(world)


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2110_08375_gb300 as mdls
    import synth
    from paper_2110_08375_gb300 import opcount

    rank, world, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    precs = [int(x) for x in args.precs.split(",")]
    n, t = args.n, args.tile
    stream = torch.cuda.current_stream()
    if args.only_backsub:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        res = run_backsub(args, dev, stream, flush, n=args.bs_n, t=args.bs_tile, sweep=False)
        if rank == 0:
            print(json.dumps({"backsub": res}), flush=True)
        barrier(world)
        return

    host = {}
    data = {}
    for p in precs:
        A, b = synth.lstsq_problem(p, n, n, seed=0, tag="cfg1")
        host[p] = (torch.from_numpy(A).pin_memory(), torch.from_numpy(b).pin_memory())
        Ad, bd = host[p][0].to(dev), host[p][1].to(dev)
        xd = torch.zeros((p, n), dtype=torch.float64, device=dev)
        ws = mdls.workspace(mdls.mdls_lstsq_workspace(p, n, n, t), dev)
        data[p] = (Ad, bd, xd, ws)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        for p in precs:
            Ad, bd, xd, ws = data[p]
            mdls.mdls_lstsq(Ad, bd, xd, tile=t, ws=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for p in precs:
        st = mdls.mdls_read_status(data[p][3])
        if st != 0:
            raise RuntimeError(f"device status {mdls.status_string(st)} for p={p}")

    # timed region: K steps, L2 flushed before each (outside the events)
    mdls.mdls_profile_enable(True)
    mdls.mdls_profile_read()
    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(precs) + 1)] for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        for k, p in enumerate(precs):
            Ad, bd, xd, ws = data[p]
            mdls.mdls_lstsq(Ad, bd, xd, tile=t, ws=ws)
            ev[i][k + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    stages = mdls.mdls_profile_read()
    mdls.mdls_profile_enable(False)
    per_prec_ms = {p: sum(ev[i][k].elapsed_time(ev[i][k + 1]) for i in range(args.steps))
                   for k, p in enumerate(precs)}
    total_ms = sum(ev[i][0].elapsed_time(ev[i][-1]) for i in range(args.steps))
    total_ms = max_over_ranks(total_ms, world)
    fl = workload_flops(precs, n)
    step_flops = sum(fl.values())
    value = world * step_flops * args.steps / (total_ms / 1e3) / 1e12

    # roofline of the dominant stage (trailing-update md GEMMs, FP64 ALU bound)
    trail_ms = stages["trailing"][0]
    trail_ops = sum(opcount.trailing_md_fmas(n, n, t, extra_cols=1) * opcount.gemm_fma_cost(p)
                    for p in precs) * args.steps
    dominant = max(stages, key=lambda k: stages[k][0])
    achieved = trail_ops / (trail_ms / 1e3) / 1e12 if trail_ms > 0 else None
    roofline = {"bound": "alu", "kernel": "gemm_kernel (trailing update C += Y (W^T C))",
                "achieved": achieved, "peak": FP64_PEAK_TOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TOPS if achieved else None,
                "traffic": TRAFFIC_BYTES if n == 1024 and t == 128 else None,
                "traffic_launch": TRAFFIC_LAUNCH,
                "op": "one FP64 instruction (DADD, DMUL or DFMA each occupy one FP64 pipe slot)",
                "peak_source": "FP64 pipe issue rate 2/clk/SM (ncu peak_sustained) x 152 SMs x 2.07 GHz",
                "dominant_stage": dominant}
    # the same FP64 pipe over the whole step: the next tile's WY products run
    # beside the trailing update, so the stage's own events include time the
    # two share; here the FP64 instructions of both kinds of products over the
    # step's wall time
    step_ops = sum((opcount.trailing_md_fmas(n, n, t, extra_cols=1) + opcount.wy_md_fmas(n, n, t, extra_cols=1))
                   * opcount.gemm_fma_cost(p) for p in precs) * args.steps
    step_rate = step_ops / (total_ms / 1e3) / 1e12
    roofline["whole_step"] = {"achieved": step_rate, "frac": step_rate / FP64_PEAK_TOPS,
                              "work": "FP64 instructions of the trailing-update and WY products of every "
                                      "precision, over the step's wall time (panels, T and back "
                                      "substitution earn nothing)"}

    checks = {}
    for p in precs:
        xref = cached_oracle(f"lstsq_n{n}_p{p}", *[h.numpy() for h in host[p]]) if t == 128 else None
        if xref is None:
            checks[PREC_NAMES[p]] = "no cached oracle answer for these inputs"
        else:
            e2, ei = md_errors(data[p][2].cpu().numpy(), xref)
            checks[PREC_NAMES[p]] = {"rel_2norm": e2, "max_entry": ei, "tolerance": TOL[p],
                                     "ok": e2 < TOL[p] and ei < TOL[p]}

    out = {"metric": METRIC, "value": value, "unit": "TFLOPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"least squares m=n={n}, tile {t} ({-(-n // t)} tiles), "
                                  f"{'+'.join(PREC_NAMES[p] for p in precs)}, seed 0",
                      "l2": "flushed before every timed step (256 MiB write, outside the events)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "clocks": clocks,
           "gpu_launches": int(sum(v[1] for v in stages.values())),
           "roofline": roofline,
           "per_prec": {PREC_NAMES[p]: {"ms": per_prec_ms[p] / args.steps,
                                        "tflops": fl[p] / (per_prec_ms[p] / args.steps / 1e3) / 1e12}
                        for p in precs},
           "vs_oracle": checks,
           "paper_equivalent": paper_equivalent(precs, n, per_prec_ms, args.steps),
           "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()}}

    # end to end through the public API with host buffers: H2D of A and b, the
    # solve, D2H of x, every step
    if not args.no_e2e:
        xs_host = {p: torch.empty((p, n), dtype=torch.float64).pin_memory() for p in precs}
        h2d = sum(host[p][0].numel() * 8 + host[p][1].numel() * 8 for p in precs)
        d2h = sum(xs_host[p].numel() * 8 for p in precs)

        def e2e_step():
            for p in precs:
                Ad, bd, xd, ws = data[p]
                Ad.copy_(host[p][0], non_blocking=True)
                bd.copy_(host[p][1], non_blocking=True)
                mdls.mdls_lstsq(Ad, bd, xd, tile=t, ws=ws)
                xs_host[p].copy_(xd, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0.record(stream)
            e2e_step()
            e1.record(stream)
            torch.cuda.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        e2e_ms = max_over_ranks(e2e_ms, world)
        out["e2e"] = {"value": world * step_flops * args.steps / (e2e_ms / 1e3) / 1e12, "unit": "TFLOPS",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "ms_per_step": e2e_ms / args.steps}
        # the e2e answers match the device-resident answers
        for p in precs:
            assert torch.equal(xs_host[p], data[p][2].cpu())

    # precision modes on the same workload: split (tensor-core WY products) and
    # refine (dd factorisation + refinement); each timed like the main loop and
    # compared with the oracle's cached answer (relative 2-norm error)
    if not args.no_modes:
        modes = {}
        for mname, mcode, plist in (("split", mdls.MODE_SPLIT, precs),
                                    ("refine", mdls.MODE_REFINE, [p for p in precs if p > 2])):
            res = {}
            for p in plist:
                Ad, bd, _, _ = data[p]
                xm = torch.zeros((p, n), dtype=torch.float64, device=dev)
                wsm = mdls.workspace(mdls.mdls_lstsq_workspace(p, n, n, t, mcode), dev)
                mdls.mdls_lstsq(Ad, bd, xm, tile=t, mode=mcode, ws=wsm)
                torch.cuda.synchronize()
                st = mdls.mdls_read_status(wsm)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                ms = 0.0
                mdls.mdls_profile_enable(True)
                mdls.mdls_profile_read()
                for _ in range(args.steps):
                    flush.zero_()
                    e0.record(stream)
                    mdls.mdls_lstsq(Ad, bd, xm, tile=t, mode=mcode, ws=wsm)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                mstages = mdls.mdls_profile_read()
                mdls.mdls_profile_enable(False)
                ms /= args.steps
                xref = cached_oracle(f"lstsq_n{n}_p{p}", *[h.numpy() for h in host[p]]) if t == 128 else None
                err = md_errors(xm.cpu().numpy(), xref)[0] if xref is not None else None
                res[PREC_NAMES[p]] = {"ms": ms, "speedup_vs_plain": (per_prec_ms[p] / args.steps) / ms,
                                      "table1_tflops": fl[p] / (ms / 1e3) / 1e12,
                                      "rel_err_vs_oracle": err, "status": st,
                                      "stages_ms": {k2: round(v2[0] / args.steps, 3) for k2, v2 in mstages.items()
                                                    if v2[0] > 0}}
                del wsm
            modes[mname] = res
        out["modes"] = modes
        # each mode over the whole step (the same workload and accuracy
        # tolerances as `value`; refine covers qd and od only)
        out["modes_total"] = {}
        for mname, res in modes.items():
            plist = [p for p in precs if PREC_NAMES[p] in res]
            ms = sum(res[PREC_NAMES[p]]["ms"] for p in plist)
            if ms > 0:
                out["modes_total"][mname] = {
                    "precisions": "+".join(PREC_NAMES[p] for p in plist), "ms_per_step": ms,
                    "value": sum(fl[p] for p in plist) / (ms / 1e3) / 1e12, "unit": "TFLOPS"}

    # batched: the mixed workload (n ~ log-uniform [32, 512], m = n + U{0..n},
    # half dd, half qd) solved by one graph launch, against a loop of single
    # mdls_lstsq calls (default tile, one reused workspace) on the same stream
    if not args.no_batched:
        out["batched"] = run_batched(args, dev, stream, flush)
    if not args.no_backsub:
        out["backsub_qd_17920"] = run_backsub(args, dev, stream, flush, n=args.bs_n, t=args.bs_tile)
    if args.bs_sweep:
        out["backsub_sweep_qd"] = run_backsub_sweep(args, dev, stream, flush)
    if not args.no_config0:
        out["lstsq_dd_256"] = run_config0(args, dev, stream, flush)
    if not args.no_qr:
        out["qr_with_q_1024"] = run_qr_with_q(args, dev, stream, flush, precs)
    if not args.no_modes_large:
        out["modes_4096x2048"] = run_modes_large(args, dev, stream, flush)
    if not args.no_complex:
        out["complex"] = run_complex(args, dev, stream, flush)
    if not args.no_toeplitz:
        out["toeplitz"] = run_toeplitz(args, dev, stream, flush)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(448, precs)
        out["cpu_baseline"].pop("seconds", None)
    if rank == 0:
        print(json.dumps(out), flush=True)
    barrier(world)


def run_batched(args, dev, stream, flush):
    import torch

    import paper_2110_08375_gb300 as mdls
    import synth
    shapes = synth.batched_shapes(args.batch, seed=0)
    probs = []
    for i, (m, n, p) in enumerate(shapes):
        A, b = synth.batched_problem(i, m, n, p, seed=0)
        probs.append((torch.from_numpy(A).to(dev), torch.from_numpy(b).to(dev),
                      torch.zeros((p, n), dtype=torch.float64, device=dev)))
    t0 = time.perf_counter()
    plan = mdls.mdls_batched_plan(probs, autotune=True)
    plan_s = time.perf_counter() - t0
    plan.launch(stream)
    torch.cuda.synchronize()
    status = plan.status()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    graph_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        plan.launch(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        graph_ms += e0.elapsed_time(e1)
    graph_ms /= args.steps
    batched_x = [x.clone() for (_, _, x) in probs]
    # loop of single solves
    need = max(mdls.mdls_lstsq_workspace(p, m, n, 0) for (m, n, p) in shapes)
    ws = mdls.workspace(need, dev)
    def loop():
        for (A, b_, x) in probs:
            mdls.mdls_lstsq(A, b_, x, tile=0, ws=ws)
    loop()
    torch.cuda.synchronize()
    flush.zero_()
    e0.record(stream)
    loop()
    e1.record(stream)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1)
    # the same loop in split mode (the mode the tuner may pick for the graph)
    need_s = max(mdls.mdls_lstsq_workspace(p, m, n, 0, mdls.MODE_SPLIT) for (m, n, p) in shapes)
    ws_s = mdls.workspace(need_s, dev)
    xs_split = [torch.zeros_like(x) for (_, _, x) in probs]

    def loop_split():
        for (A, b_, _), xs in zip(probs, xs_split):
            mdls.mdls_lstsq(A, b_, xs, tile=0, mode=mdls.MODE_SPLIT, ws=ws_s)
    loop_split()
    torch.cuda.synchronize()
    flush.zero_()
    e0.record(stream)
    loop_split()
    e1.record(stream)
    torch.cuda.synchronize()
    loop_split_ms = e0.elapsed_time(e1)
    del ws_s
    worst = 0.0
    for xb, (_, _, x) in zip(batched_x, probs):
        d = (xb - x).sum(dim=0).abs().max().item() / max(x[0].abs().max().item(), 1e-300)
        worst = max(worst, d)
    tiles = plan.tiles()
    modes = plan.modes()
    res = {"problems": len(shapes), "solves_per_s": len(shapes) / (graph_ms / 1e3),
           "loop_solves_per_s": len(shapes) / (loop_ms / 1e3), "speedup_vs_loop": loop_ms / graph_ms,
           "loop_split_solves_per_s": len(shapes) / (loop_split_ms / 1e3),
           "speedup_vs_split_loop": loop_split_ms / graph_ms,
           "graph_ms": graph_ms, "loop_ms": loop_ms, "plan_s_with_autotune": plan_s,
           "max_rel_diff_batched_vs_loop": worst, "nonzero_status": sum(1 for s in status if s != 0),
           "tiles_used": sorted(set(tiles)),
           "modes_used": {"plain": sum(1 for m in modes if m == mdls.MODE_PLAIN),
                          "split": sum(1 for m in modes if m == mdls.MODE_SPLIT)}}
    plan.destroy()
    return res


def md_errors(x, ref):
    """(relative 2-norm error, largest entry error / largest |ref|) of md
    vectors x and ref of shape (p, n): each entry's difference is the sum of
    the 2p limbs, formed exactly and rounded once by math.fsum."""
    import math
    import numpy as np
    d = np.array([math.fsum(list(x[:, i]) + [-v for v in ref[:, i]]) for i in range(ref.shape[1])])
    nr = float(np.linalg.norm(ref[0]))
    mr = float(np.max(np.abs(ref[0])))
    return float(np.linalg.norm(d)) / nr, float(np.max(np.abs(d))) / mr


def cached_oracle(name, *inputs):
    """The oracle's answer stored by tests/golden/make_oracle_cache.py for the
    given inputs (None when absent or computed from other inputs)."""
    import hashlib
    import numpy as np
    f = os.path.join(ROOT, "tests", "golden", "oracle_cache", name + ".npz")
    if not os.path.exists(f):
        return None
    z = np.load(f)
    h = hashlib.sha256()
    for a in inputs:
        a = np.ascontiguousarray(a)
        h.update(str(a.shape).encode())
        h.update(memoryview(a).cast("B"))
    return z["x"] if h.hexdigest() == str(z["input_sha256"]) else None


def run_backsub(args, dev, stream, flush, p=4, n=17920, t=128, sweep=True):
    """Back substitution alone (Algorithm 1): quad double, n = 17920, tile 128
    (140 tiles).  R upper triangular with diagonal U[1,2], strict upper part
    U[-1,1)/n, lower limbs x_l = x_(l-1) 2^-54 U[-1,1); y U[-1,1): the seeded
    inputs of synth.upper_triangular_fast, the same ones the parity test
    checks, and the solution is compared with the oracle's cached answer."""
    import torch

    import paper_2110_08375_gb300 as mdls
    import synth
    from paper_2110_08375_gb300 import opcount
    t0 = time.perf_counter()
    Rh, yh = synth.upper_triangular_fast(p, n, seed=0)
    xref = cached_oracle(f"backsub_n{n}_p{p}", Rh, yh)
    R = torch.from_numpy(Rh).to(dev)
    del Rh
    y = torch.from_numpy(yh).to(dev)
    gen_s = time.perf_counter() - t0
    x = torch.zeros((p, n), dtype=torch.float64, device=dev)
    ws = mdls.workspace(mdls.mdls_backsub_workspace(p, n, t), dev)
    for _ in range(2):
        mdls.mdls_backsub(R, y, x, tile=t, ws=ws)
    torch.cuda.synchronize()
    status = mdls.mdls_read_status(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms = []
    mdls.mdls_profile_enable(True)
    mdls.mdls_profile_read()
    for _ in range(max(args.steps, 3)):
        flush.zero_()
        e0.record(stream)
        mdls.mdls_backsub(R, y, x, tile=t, ws=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    stages = mdls.mdls_profile_read()
    mdls.mdls_profile_enable(False)
    k = len(ms)
    med = statistics.median(ms)
    # the paper's tile study (its back-substitution experiments vary the tile
    # size at fixed n): the same solve with other tiles, same resident R
    tiles_ms = {t: med}
    for t2 in ((32, 64, 256) if sweep else ()):
        ws2 = mdls.workspace(mdls.mdls_backsub_workspace(p, n, t2), dev)
        x2 = torch.zeros_like(x)
        mdls.mdls_backsub(R, y, x2, tile=t2, ws=ws2)
        torch.cuda.synchronize()
        ms2 = []
        for _ in range(3):
            flush.zero_()
            e0.record(stream)
            mdls.mdls_backsub(R, y, x2, tile=t2, ws=ws2)
            e1.record(stream)
            torch.cuda.synchronize()
            ms2.append(e0.elapsed_time(e1))
        tiles_ms[t2] = statistics.median(ms2)
        del ws2
    flops = opcount.table1_flops(p, opcount.backsub_counts(n))
    # the paper's count for Algorithm 1 also credits the tile inversions
    # (t^3/2 mul-add pairs per tile): context only
    sig = opcount.TABLE1_SIGMA[p]
    ntiles = -(-n // t)
    paper_pairs = ntiles * t ** 3 / 2 + n * (n - 1) / 2
    rbytes = n * (n + 1) // 2 * 8 * p
    del R
    torch.cuda.empty_cache()
    check = {"vs_oracle": "no cached oracle answer for these inputs"}
    if xref is not None:
        e2, ei = md_errors(x.cpu().numpy(), xref)
        check = {"vs_oracle_rel_2norm": e2, "vs_oracle_max_entry": ei, "tolerance": 1e-55,
                 "ok": e2 < 1e-55 and ei < 1e-55}
    return {"workload": f"qd back substitution n={n}, tile {t} ({-(-n // t)} tiles), R resident in HBM, "
                        "L2 flushed before each solve",
            "inputs_s": round(gen_s, 1), "check": check,
            "ms": med, "table1_tflops": flops / (med / 1e3) / 1e12,
            "paper_equivalent_tflops": paper_pairs * (sig["add"] + sig["mul"]) / (med / 1e3) / 1e12,
            "hbm_gbs_upper_triangle": rbytes / (med / 1e3) / 1e9, "status": status,
            "tile_sweep_ms": {str(k2): round(v2, 3) for k2, v2 in sorted(tiles_ms.items())},
            "stages_ms": {kk: round(v[0] / k, 3) for kk, v in stages.items() if v[0] > 0}}


def _timed(stream, flush, fn, reps):
    """Median CUDA-event time (ms) of fn() over reps calls, L2 flushed before each."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(reps):
        flush.zero_()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def run_config0(args, dev, stream, flush, n=256, t=32):
    """Least squares m = n = 256, tile 32 (eight tiles), double double: the
    small dense workload, kernel time with inputs resident and end to end
    (pinned host A, b in, x out, every solve)."""
    import torch

    import paper_2110_08375_gb300 as mdls
    import synth
    from paper_2110_08375_gb300 import opcount
    p = 2
    A, b = synth.lstsq_problem(p, n, n, seed=0, tag="cfg0")
    Ah, bh = torch.from_numpy(A).pin_memory(), torch.from_numpy(b).pin_memory()
    Ad, bd = Ah.to(dev), bh.to(dev)
    xd = torch.zeros((p, n), dtype=torch.float64, device=dev)
    xh = torch.empty((p, n), dtype=torch.float64).pin_memory()
    ws = mdls.workspace(mdls.mdls_lstsq_workspace(p, n, n, t), dev)
    for _ in range(3):
        mdls.mdls_lstsq(Ad, bd, xd, tile=t, ws=ws)
    torch.cuda.synchronize()
    st = mdls.mdls_read_status(ws)
    reps = max(args.steps, 5)
    ms = _timed(stream, flush, lambda: mdls.mdls_lstsq(Ad, bd, xd, tile=t, ws=ws), reps)

    def e2e():
        Ad.copy_(Ah, non_blocking=True)
        bd.copy_(bh, non_blocking=True)
        mdls.mdls_lstsq(Ad, bd, xd, tile=t, ws=ws)
        xh.copy_(xd, non_blocking=True)
    e2e_ms = _timed(stream, flush, e2e, reps)
    fl = opcount.lstsq_table1_flops(p, n, n)
    return {"workload": f"dd least squares m=n={n}, tile {t} (8 tiles), seed 0", "status": st,
            "ms": ms, "table1_tflops": fl / (ms / 1e3) / 1e12, "e2e_ms": e2e_ms,
            "e2e_table1_tflops": fl / (e2e_ms / 1e3) / 1e12}


# The paper's V100 kernel times for QR of 1024 x 1024 with 8 tiles of 128
# (context only: another GPU, CAMPARY-generated kernels, its own op counts)
PAPER_V100_QR_1024_MS = {2: 451.5, 4: 3167.0, 8: 11754.6}


def run_qr_with_q(args, dev, stream, flush, precs, n=1024, t=128):
    """Blocked Householder QR with Q formed (Algorithm 2's full output,
    m = n = 1024, tile 128) in every precision: the paper-comparable QR."""
    import torch

    import paper_2110_08375_gb300 as mdls
    import synth
    from paper_2110_08375_gb300 import opcount
    out = {"workload": f"QR with Q, m=n={n}, tile {t} (8 tiles), A as in the least-squares step, seed 0"}
    for p in precs:
        A, _ = synth.lstsq_problem(p, n, n, seed=0, tag="cfg1")
        A0 = torch.from_numpy(A).to(dev)
        Ad = A0.clone()
        Qd = torch.zeros((p, n, n), dtype=torch.float64, device=dev)
        ws = mdls.workspace(mdls.mdls_qr_workspace(p, n, n, t, True), dev)

        def run():
            Ad.copy_(A0)
            mdls.mdls_qr(Ad, Qd, tile=t, ws=ws)
        run()
        torch.cuda.synchronize()
        st = mdls.mdls_read_status(ws)
        reps = 3 if p < 8 else 2
        ms = _timed(stream, flush, run, reps)
        # the copy of A (n^2 p doubles) inside the timed call is under 0.1 ms
        fl = opcount.table1_flops(p, opcount.qr_counts(n, n, want_q=True))
        out[PREC_NAMES[p]] = {"ms": ms, "table1_tflops": fl / (ms / 1e3) / 1e12, "status": st,
                              "paper_v100_kernel_ms": PAPER_V100_QR_1024_MS[p]}
        del Ad, Qd, ws, A0
    torch.cuda.empty_cache()
    return out


def run_modes_large(args, dev, stream, flush, m=4096, n=2048, t=128):
    """Precision modes at m = 4096, n = 2048, tile 128, kappa = 1e6 in quad and
    octo double: A = U diag(sigma) V^T with exactly orthogonal Walsh-Hadamard
    factors, x* ~ U[-1,1) and b = A x* formed exactly (synth.modes_problem),
    so x* is the exact solution; each mode's time and its error against x*."""
    import torch

    import paper_2110_08375_gb300 as mdls
    import synth
    from paper_2110_08375_gb300 import opcount
    out = {"workload": f"least squares m={m}, n={n}, tile {t}, kappa 1e6, consistent b = A x* (exact)"}
    for p in (4, 8):
        pr = synth.modes_problem(p, m, n, 1e6, seed=0, consistent=True)
        Ad, bd = torch.from_numpy(pr["A"]).to(dev), torch.from_numpy(pr["b"]).to(dev)
        fl = opcount.lstsq_table1_flops(p, m, n)
        res = {}
        for name, mode in (("plain", mdls.MODE_PLAIN), ("split", mdls.MODE_SPLIT), ("refine", mdls.MODE_REFINE)):
            xd = torch.zeros((p, n), dtype=torch.float64, device=dev)
            ws = mdls.workspace(mdls.mdls_lstsq_workspace(p, m, n, t, mode), dev)
            run = lambda: mdls.mdls_lstsq(Ad, bd, xd, tile=t, mode=mode, ws=ws)  # noqa: E731
            if name != "plain":
                run()                      # the plain od solve takes seconds: timed once, cold
            ms = _timed(stream, flush, run, 1 if name == "plain" else 2)
            st = mdls.mdls_read_status(ws)
            e2, ei = md_errors(xd.cpu().numpy(), pr["xstar"])
            res[name] = {"ms": ms, "table1_tflops": fl / (ms / 1e3) / 1e12, "rel_err_vs_exact": e2,
                         "max_entry_err": ei, "status": st}
            del ws
        for name in ("split", "refine"):
            res[name]["speedup_vs_plain"] = res["plain"]["ms"] / res[name]["ms"]
            res[name]["equal_accuracy"] = res[name]["rel_err_vs_exact"] <= max(10 * res["plain"]["rel_err_vs_exact"],
                                                                               TOL[p])
        out[PREC_NAMES[p]] = res
        del Ad, bd
    torch.cuda.empty_cache()
    return out


def run_backsub_sweep(args, dev, stream, flush, p=4, nmax=20480):
    """The paper's back-substitution study on GB300 (its experiments vary
    the tile size and the number of tiles at fixed precision): quad double,
    n in {2560, 5120, 10240, 17920, 20480} x tile in {32, 64, 128, 256}, the
    leading n x n block of one seeded upper triangular R (diagonal U[1,2],
    strict upper part U[-1,1)/nmax), drawn on the device with torch's
    generator (timing only: these solves are not compared with the oracle;
    the n = 17920 entry above is).  Median of three solves, L2 flushed."""
    import torch

    import paper_2110_08375_gb300 as mdls
    from paper_2110_08375_gb300 import opcount
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    R = torch.empty((p, nmax, nmax), dtype=torch.float64, device=dev)   # [limb][col][row]
    R[0].uniform_(-1.0, 1.0, generator=g).div_(nmax)
    R[0].diagonal().uniform_(1.0, 2.0, generator=g)
    for l in range(1, p):
        R[l].uniform_(-1.0, 1.0, generator=g).mul_(R[l - 1]).mul_(2.0 ** -54)
    for l in range(p):
        R[l].copy_(torch.tril(R[l]))
    y = torch.empty((p, nmax), dtype=torch.float64, device=dev)
    y[0].uniform_(-1.0, 1.0, generator=g)
    for l in range(1, p):
        y[l].uniform_(-1.0, 1.0, generator=g).mul_(y[l - 1]).mul_(2.0 ** -54)
    out = {}
    for n in (2560, 5120, 10240, 17920, 20480):
        Rv = R.as_strided((p, n, n), (nmax * nmax, nmax, 1))   # leading n x n block, ld = nmax
        yv = y[:, :n]
        row = {}
        for t in (32, 64, 128, 256):
            x = torch.zeros((p, n), dtype=torch.float64, device=dev)
            ws = mdls.workspace(mdls.mdls_backsub_workspace(p, n, t), dev)
            mdls.mdls_backsub(Rv, yv, x, tile=t, ws=ws)
            torch.cuda.synchronize()
            ms = _timed(stream, flush, lambda: mdls.mdls_backsub(Rv, yv, x, tile=t, ws=ws), 3)
            row[str(t)] = {"ms": round(ms, 3), "status": mdls.mdls_read_status(ws),
                           "table1_tflops": round(opcount.table1_flops(p, opcount.backsub_counts(n)) / (ms / 1e3) / 1e12, 3)}
            del ws
        out[str(n)] = row
    del R
    torch.cuda.empty_cache()
    return out


# The paper's V100 times for complex double-double QR of 512 x 512 ("all
# kernels", ms) at 16 x 32, 8 x 64, 4 x 128 and 2 x 256 tiles: context only.
PAPER_V100_ZQR_DD_512_MS = {32: 97.4, 64: 227.4, 128: 238.5, 256: 420.8}


def run_complex(args, dev, stream, flush):
    """Complex multiple doubles (real and imaginary planes): the paper's
    complex double-double QR of 512 x 512 with Q formed at four tile sizes,
    and complex least squares m = n = 512, tile 128, in dd, qd and od with
    each solution's error against the oracle's cached answer when present.
    Entries of A and b: real and imaginary parts ~ U[-1,1) in every limb
    recipe, seed 0."""
    import torch

    import paper_2110_08375_gb300 as mdls
    import synth
    from paper_2110_08375_gb300 import opcount
    out = {}
    n = 512
    A_re, _ = synth.lstsq_problem(2, n, n, seed=0, tag="cplx/re")
    A_im, _ = synth.lstsq_problem(2, n, n, seed=0, tag="cplx/im")
    A0r, A0i = torch.from_numpy(A_re).to(dev), torch.from_numpy(A_im).to(dev)
    qr = {}
    for t in (32, 64, 128, 256):
        Ar, Ai = A0r.clone(), A0i.clone()
        Qr = torch.zeros((2, n, n), dtype=torch.float64, device=dev)
        Qi = torch.zeros_like(Qr)
        ws = mdls.workspace(mdls.lib().mdls_zqr_workspace(2, n, n, t, 1), dev)

        def run():
            Ar.copy_(A0r)
            Ai.copy_(A0i)
            mdls.mdls_zqr(Ar, Ai, Qr, Qi, tile=t, ws=ws)
        run()
        torch.cuda.synchronize()
        ms = _timed(stream, flush, run, 3)
        qr[str(t)] = {"ms": round(ms, 3), "status": mdls.mdls_read_status(ws),
                      "table1_tflops": round(opcount.zqr_table1_flops(2, n, n) / (ms / 1e3) / 1e12, 3),
                      "paper_v100_kernel_ms": PAPER_V100_ZQR_DD_512_MS[t]}
        del ws, Qr, Qi
    out["zqr_dd_512_with_q"] = qr
    ls = {}
    for p in (2, 4, 8):
        Ar, br = synth.lstsq_problem(p, n, n, seed=0, tag="cplx/ls/re")
        Ai, bi = synth.lstsq_problem(p, n, n, seed=0, tag="cplx/ls/im")
        d = [torch.from_numpy(v).to(dev) for v in (Ar, Ai, br, bi)]
        xr = torch.zeros((p, n), dtype=torch.float64, device=dev)
        xi = torch.zeros_like(xr)
        ws = mdls.workspace(mdls.lib().mdls_zlstsq_workspace(p, n, n, 128), dev)
        run = lambda: mdls.mdls_zlstsq(d[0], d[1], d[2], d[3], xr, xi, tile=128, ws=ws)  # noqa: E731
        run()
        torch.cuda.synchronize()
        ms = _timed(stream, flush, run, 3)
        entry = {"ms": round(ms, 3), "status": mdls.mdls_read_status(ws),
                 "table1_tflops": round(opcount.zlstsq_table1_flops(p, n, n) / (ms / 1e3) / 1e12, 3)}
        ref = cached_oracle(f"zlstsq_n512_p{p}", Ar, Ai, br, bi)
        if ref is not None:
            import numpy as np
            xh = np.concatenate([xr.cpu().numpy(), xi.cpu().numpy()], axis=1)
            e2, ei = md_errors(xh, ref)
            entry.update({"vs_oracle_rel_2norm": e2, "vs_oracle_max_entry": ei, "ok": e2 < TOL[p] and ei < TOL[p]})
        ls[PREC_NAMES[p]] = entry
        del ws
    out["zlstsq_512_tile128"] = ls
    torch.cuda.empty_cache()
    return out


def run_toeplitz(args, dev, stream, flush, n=512, d=8, t=128):
    """Lower triangular block-Toeplitz solve of a power-series Newton step:
    J(t) x(t) = b(t) mod t^9 with nine 512 x 512 blocks (entries ~ U[-1,1)
    per limb recipe, seed 0), tile 128, in dd, qd and od: one QR of J_0,
    then nine block solves."""
    import numpy as np
    import torch

    import paper_2110_08375_gb300 as mdls
    import synth
    from paper_2110_08375_gb300 import opcount
    out = {"workload": f"block-Toeplitz J(t) x(t) = b(t) mod t^{d + 1}, {d + 1} blocks of {n} x {n}, tile {t}"}
    for p in (2, 4, 8):
        J = np.stack([synth.md_matrix(p, n, n, 0, f"toebench/J{i}") for i in range(d + 1)], axis=1)
        b = np.stack([synth.md_vector(p, n, 0, f"toebench/b{k}") for k in range(d + 1)], axis=1)
        Jd = torch.from_numpy(np.ascontiguousarray(J)).to(dev)
        bd = torch.from_numpy(np.ascontiguousarray(b)).to(dev)
        x = torch.zeros((p, d + 1, n), dtype=torch.float64, device=dev)
        ws = mdls.workspace(mdls.lib().mdls_toeplitz_lstsq_workspace(p, n, n, t), dev)
        run = lambda: mdls.mdls_toeplitz_lstsq(Jd, bd, x, tile=t, ws=ws)  # noqa: E731
        run()
        torch.cuda.synchronize()
        ms = _timed(stream, flush, run, 3)
        fl = opcount.table1_flops(p, opcount.toeplitz_counts(n, n, d))
        out[PREC_NAMES[p]] = {"ms": round(ms, 3), "status": mdls.mdls_read_status(ws),
                              "table1_tflops": round(fl / (ms / 1e3) / 1e12, 3)}
        del ws, Jd, bd
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
