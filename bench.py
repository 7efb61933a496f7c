#!/usr/bin/env python
"""Benchmark: PR+MAR solves per second on the 24x24 grid Ising workload.

One step = one PR + MAR solve (forward contraction of the whole tree, log Z,
adjoint sweep, all 576 single-variable marginals) of the 24x24 grid binary
MRF (576 spins, 1104 couplings exp(J s_i s_j) with J ~ N(0,1), 576 fields
exp(h s_i) with h ~ N(0, 0.5), seed 20240524), in TF32 tensor-core GEMMs with
FP32 storage and power-of-two rescaling (FP64 log-scale bookkeeping), on the
library's greedy contraction tree with its absorption chains re-associated
(tn_reassociate).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun); every rank solves its own replica
(the path has no exchange step at one evidence set), value = solves of all
ranks / max time over ranks ("scaling": "weak").

--impl reference times the CPU FP64 oracle (bucket elimination) on the host
cores on a bounded sample: the elimination of a prefix of the row-sweep
order, scaled to a full PR by the symbolic work ratio and to PR+MAR by the
factor 3 of the paper's Corollary on reverse-mode cost.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "grid24x24 Ising PR+MAR"
METRIC = "PR+MAR solves/sec (24x24 grid Ising, TF32 contraction)"
UNIT = "solves/s"


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum,
# averaged over one step's launches of the kernel class) from the ncu capture
# summarised in profiles/absorb_streaming_grid24_tf32.md, valid only while the
# kernel sources hash to the values recorded with it.
TRAFFIC = {
    "absorb": {"bytes_per_launch": 6.124e6, "launches": 272,
               "sources": {"paper_2405_14060_gb300/csrc/stream_impl.cuh":
                           "03c7fe364243eef912e2ecd26c66b9ef81d20048b2117b87e2a1627fb842541a",
                           "paper_2405_14060_gb300/csrc/stream.cuh":
                           "0989adeb8b5a666f5824bedad209aca1f20b4f69416d16dabec4b4ee84b65512"}},
}


def _traffic(kernel):
    import hashlib
    t = TRAFFIC.get(kernel)
    if not t:
        return None
    for path, digest in t["sources"].items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return t["bytes_per_launch"]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def _workload():
    from paper_2405_14060_gb300 import synth
    return synth.workload(2)


def run_reference(args):
    """CPU FP64 oracle on the host cores, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    w = _workload()
    order = np.arange(w.model.nvars)          # row sweep: width-24 buckets
    nelim = int(os.environ.get("TN_ORACLE_PREFIX", "96"))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        wp, wf = oracle.ve_pr_prefix(w.model, order, nelim)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt * wf / wp * 3.0)   # full PR, then PR+MAR = 3 x PR
    t = float(np.mean(times))
    value = 1.0 / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "order": "row sweep (bucket elimination)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"bucket elimination of the first {nelim} of 576 variables "
                                   "of the row-sweep order, scaled by the symbolic work ratio "
                                   "to a full PR and x3 to PR+MAR"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _fp64_torch_baseline(model, l, r):
    """Plain PyTorch float64 contraction along the same tree (torch.einsum per
    node, max-normalised with the log kept on the side), forward + autograd
    backward for the marginals: the 'plain FP64 GPU contraction'."""
    import torch
    leaves = [list(map(int, s)) for s in model.scopes] + [[v] for v in range(model.nvars)]
    from collections import Counter
    total = Counter()
    for L in leaves:
        total.update(L)
    dev = "cuda"
    base = [torch.tensor(t, dtype=torch.float64, device=dev).reshape([2] * len(s))
            for s, t in zip(model.scopes, model.tables)]
    unity = [torch.ones(2, dtype=torch.float64, device=dev, requires_grad=True)
             for _ in range(model.nvars)]
    labels = [list(L) for L in leaves]
    cnt = [Counter(L) for L in leaves]
    letters = {}

    def let(v):
        if v not in letters:
            letters[v] = chr(ord("a") + len(letters)) if len(letters) < 26 else \
                chr(ord("A") + len(letters) - 26)
        return letters[v]
    plan = []
    for a, b in zip(l, r):
        c = cnt[a] + cnt[b]
        keep = [v for v in dict.fromkeys(labels[a] + labels[b]) if c[v] < total[v]]
        cnt.append(Counter({v: c[v] for v in keep}))
        labels.append(keep)
        plan.append((int(a), int(b), keep))

    def run():
        ts = list(base) + list(unity)
        logs = 0.0
        for a, b, keep in plan:
            letters.clear()
            eq = ("".join(let(v) for v in labels[a]) + "," + "".join(let(v) for v in labels[b]) +
                  "->" + "".join(let(v) for v in keep))
            c = torch.einsum(eq, ts[a], ts[b])
            m = c.detach().max()
            logs = logs + torch.log(m)
            ts.append(c / m)
        z = ts[-1].reshape(())
        lz = torch.log(z) + logs
        lz.backward()
        return lz
    for u in unity:
        u.grad = None
    run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 2
    for _ in range(reps):
        for u in unity:
            u.grad = None
        lz = run()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps, float(lz.detach())


def _task_extras():
    """Throughput of the tropical tasks on their workload (a second or two):
    MAP and MMAP on the 300-variable banded Bayesian network with 20% of the
    variables observed.  Device time from the library's CUDA events, wall
    time through the host-pointer C ABI.  The batched and sliced workloads
    take minutes and are timed by their parity tests instead."""
    from paper_2405_14060_gb300 import synth, tn
    out = {}
    w3 = synth.workload(3)
    M = tn.Model.from_synth(w3.model)

    def timed(fn, reps):
        fn()
        t0 = time.perf_counter()
        dev = 0.0
        for _ in range(reps):
            fn()
            dev += M.last_device_ms()
        return (time.perf_counter() - t0) / reps, dev / reps

    wall, dev = timed(lambda: M.map(w3.evid, prec="fp32"), 20)
    out["map_bn300_fp32"] = {"solves_per_s": 1.0 / wall, "device_ms": dev,
                             "config": "300 vars, 60 observed, greedy tree, max-plus FP32"}
    wall, dev = timed(lambda: M.mmap(w3.query, w3.evid, prec="fp32"), 10)
    out["mmap_bn300_fp32"] = {"solves_per_s": 1.0 / wall, "device_ms": dev,
                              "config": f"{len(w3.query)} query vars, sum phase then max-plus"}
    return out


def aggregate_ranks(ms_local, steps, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` replicas: every rank solved `steps`
    problems; the job's time is the slowest rank's (max over ranks)."""
    ms = ms_local
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1e3)


def run_ours(args):
    import torch
    from paper_2405_14060_gb300 import tn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = _workload()
    m = w.model
    M = tn.Model.from_synth(m)
    # greedy order, then runs of absorption steps re-associated
    tree = M.reassociate(*M.optimize_order(0))
    M.set_order(*tree)
    prec = args.prec
    stats = M.tree_stats(1, "fp32")
    ncard = int(m.card.sum())
    evid = torch.full((1, m.nvars), -1, dtype=torch.int32, device="cuda")
    logz = torch.zeros(1, dtype=torch.float64, device="cuda")
    marg = torch.zeros(1, ncard, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream

    def step():
        M.mar_dev(evid, logz, marg, prec=prec, stream=sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches = M.last_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        # the timed region is what `ncu --profile-from-start off` captures
        torch.cuda.profiler.start()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    ms, value = aggregate_ranks(e0.elapsed_time(e1), args.steps, world, dist, "cuda")

    # end to end through the host-pointer C ABI: H2D evidence, D2H log Z + marginals
    ev_h = np.full((1, m.nvars), -1, np.int32)
    M.mar(ev_h, prec=prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne2e = max(3, args.steps // 2)
    for _ in range(ne2e):
        lz_h, marg_h = M.mar(ev_h, prec=prec)
    t_e2e = (time.perf_counter() - t0) / ne2e
    e2e = {"value": world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(ev_h.nbytes),
           "d2h_bytes_per_step": int(lz_h.nbytes + marg_h.nbytes)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # accuracy against the library's own FP64 path on the same tree
    lz64, marg64 = M.mar(prec="fp64")
    fp64_ms = M.last_device_ms()
    acc = {"logz": float(lz_h[0]), "logz_fp64": float(lz64[0]),
           "dlogz_abs": float(abs(lz_h[0] - lz64[0])),
           "dlogz_rel": float(abs(lz_h[0] - lz64[0]) / abs(lz64[0])),
           "max_marg_err": float(np.max(np.abs(marg_h - marg64)))}

    # roofline of the dominant kernel class
    peaks, peak_src = _peaks()
    prof = M.profile("mar", prec=prec, reps=3)
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, d = dom
    if name in ("tcgemm",):
        ratio = {"tf32": 1.1 / 2.25, "bf16": 1.0}[prec]
        peak = peaks["bf16_tflops"] * ratio
        ach = d["flops"] / (d["ms"] / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None}
    else:
        peak = peaks["hbm_gbs"]
        ach = d["bytes"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": _traffic(name),
                "traffic_unit": "bytes per launch (ncu DRAM read + write)",
                "algorithmic_bytes_per_launch": d["bytes"] / max(1.0, d["launches"])}
    roof.update({"kernel": name, "launches_per_step": d["launches"],
                 "ms_per_step": d["ms"], "peak_source": peak_src})
    prof_out = {k: {"ms": round(v["ms"], 4), "launches": int(v["launches"]),
                    "gflop": round(v["flops"] / 1e9, 3), "gbytes": round(v["bytes"] / 1e9, 4)}
                for k, v in prof.items()}

    # plain FP64 GPU contraction baselines
    fp64 = {"own_fp64_ms": fp64_ms}
    if not args.skip_torch_fp64:
        try:
            t_torch, lz_torch = _fp64_torch_baseline(m, *tree)
            fp64.update({"torch_einsum_fp64_ms": t_torch * 1e3, "torch_einsum_logz": lz_torch})
        except Exception as e:  # baseline only: report, do not fail the bench
            fp64["torch_einsum_fp64_error"] = str(e)[:200]
    best64 = min(v for k, v in fp64.items() if k.endswith("_ms"))
    fp64["x_vs_fp64"] = best64 / (ms / args.steps)

    # CPU oracle baseline on a bounded sample (one rank only)
    cpu = None
    if not args.skip_cpu_baseline:
        import oracle
        order = np.arange(m.nvars)
        nelim = int(os.environ.get("TN_ORACLE_PREFIX", "96"))
        t0 = time.perf_counter()
        wp, wf = oracle.ve_pr_prefix(m, order, nelim)
        dt = time.perf_counter() - t0
        t_full = dt * wf / wp * 3.0
        cpu = {"value": 1.0 / t_full, "unit": UNIT, "cores": oracle.num_threads(),
               "kind": "oracle",
               "sample": f"bucket elimination (FP64) of the first {nelim} of 576 variables of "
                         f"the row-sweep order ({dt:.1f} s), scaled by the symbolic work ratio "
                         f"{wf / wp:.2f} to a full PR and x3 to PR+MAR"}

    tasks = None
    if not args.skip_tasks:
        try:
            tasks = _task_extras()
        except Exception as e:  # reported, never fails the bench line
            tasks = {"error": str(e)[:200]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": prec, "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": prec, "order": "greedy + re-associated absorption chains",
                   "tree": {"tc_log2": round(stats["tc"], 3), "sc_log2": stats["sc"],
                            "rw_log2": round(stats["rw"], 3)},
                   "l2": "no flush: working set per step > 5 GB of tensor traffic >> 129 MB L2",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(launches * args.steps), "clocks": clk.summary(),
        "accuracy": acc, "fp64_baseline": fp64, "profile": prof_out, "tasks": tasks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tf32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-torch-fp64", action="store_true")
    ap.add_argument("--skip-tasks", action="store_true",
                    help="skip the MAP / MMAP throughput extras")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2405_14060_gb300 import build
        build.build()
        run_ours(args)


if __name__ == "__main__":
    main()
