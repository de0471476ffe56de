#!/usr/bin/env python3
"""Benchmark of the batched-einsum engine.

Workload (one "step"): the DG local-gradient functional batched einsum on a
P4 tetrahedral mesh -- b = 3 einsums 'rij,er,ej->ei' (one per derivative
direction x) sharing the derivative matrices D (3 x 35 x 35), with per-row
geometric factors G[e, r, x] and the field u = sin(a) * b fused into the
operand load; E = 262144 elements, FP64, synthetic N(0,1) data.  A step runs
the whole hot path through the C ABI: parse -> canonicalize -> lookup in the
tuning database -> evaluate on the GPU.

  value  : algorithmic GB/s over all ranks (operands read once, outputs
           written once, per step), inputs already resident in HBM
  e2e    : same metric through be_execute_host with pinned host buffers
           (host -> device copies of the inputs and device -> host copies of
           the results inside the timed region)
  roofline: the dominant kernel, achieved vs peak, from CUDA events on the
           launching stream

``--impl reference`` times the CPU oracle (plain FP64 loops, all host
cores) on a bounded sample of the same workload instead.
Multi-GPU: the path shards by replicas (each rank evaluates its own batch).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "batched-einsum GB/s & TFLOP/s vs roofline; served einsums/s, p50/p99 latency"
E_FULL, NDOF, DIM = 262144, 35, 3


def algorithmic(E, ndof=NDOF, dim=DIM):
    """Bytes (each operand read once, each output written once) and flops
    (hoisted: t = D u once per element, then G t per row, plus the producer
    multiply; sin counted as 0) of one DG-gradient step."""
    byts = 8 * (2 * E * ndof + E * dim * dim + dim * ndof * ndof + dim * E * ndof)
    flops = E * (2 * dim * ndof * ndof + 2 * dim * dim * ndof + ndof)
    return byts, flops


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "source": "fallback"}
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        peaks.update({k: d[k] for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained") if k in d})
        peaks["source"] = "measured"
    return peaks


# FP64 vector-pipe peak of B300 (nominal 1.25 TFLOP/s dense FP64): the bound
# of the FP64-pipe variant of the element kernel.
FP64_PEAK_TFLOPS = 1.25
# FP32 pipe of B300 from unit counts and clock: 148 SMs x 128 FP32 lanes x
# 2 flops (FMA) x 2.032 GHz: the bound of the double-float element kernel.
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# FP32 flops the double-float kernel spends per element on its compensated
# dot products: 15 per term (1 mul + 3 fma + 8 add, FMA counted twice) over
# 3*35*35 + 3*3*35 terms, plus 3 per normalisation of 2*105 results (the
# sine and the conversions are not counted, so this is a lower bound)
DF_FLOPS_PER_ELEMENT = 15 * (3 * 35 * 35 + 3 * 3 * 35) + 3 * 2 * 105
# bf16 MMA flops the tensor-core variant issues per element: per column
# block of 32 and K-slice of 16, u's digit q = 0..5 times D's digit planes
# p = 0..min(5, 6 - q) in one MMA of N = 32 (number of planes): 6 + 6 + 5 +
# 4 + 3 + 2 = 26 planes (832 columns); 3 K-slices, 4 column blocks, x 2
TC_MMA_FLOPS_PER_ELEMENT = 2 * 16 * 3 * 4 * 32 * (6 + 6 + 5 + 4 + 3 + 2)
# headers whose code is compiled into each kernel: the committed profile of a
# kernel stays valid only while the kernel source and these hash as recorded
KERNEL_HEADERS = {"kernels_element_tc.cu": ["df_math.cuh", "tc_common.cuh", "exec.hpp"],
                  "kernels_element_df.cu": ["df_math.cuh", "exec.hpp"],
                  "kernels_element.cu": ["exec.hpp"],
                  "kernels_dense.cu": ["dense.hpp", "tc_common.cuh"],
                  "kernels_persistent.cu": ["generic_eval.cuh", "exec.hpp"]}


def source_hash(source):
    """sha256 (first 16 hex digits) of a kernel source file followed by the
    headers compiled into it."""
    d = os.path.join(ROOT, "paper_2601_12220_b300", "csrc")
    h = hashlib.sha256()
    for f in [source] + KERNEL_HEADERS.get(source, []):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


_PIPE = {}


def pipe_peaks(be):
    """Measured FP64 and FP32 pipe peaks of this device (TFLOP/s, be_peak_probe:
    FMA chains in registers), measured once per process; the rooflines of the
    FP64 and FP32 / double-float paths use these, with the nominal figures
    (FP64 1.25 TFLOP/s; FP32 148 SMs x 128 lanes x 2 x 2.032 GHz) beside them."""
    if not _PIPE:
        _PIPE["fp64"] = be.peak_probe("fp64")
        _PIPE["fp32"] = be.peak_probe("fp32")
        _PIPE["source"] = "measured (be_peak_probe: FMA chains, best of 5)"
        _PIPE["nominal_fp64"] = FP64_PEAK_TFLOPS
        _PIPE["nominal_fp32"] = FP32_PEAK_TFLOPS
    return _PIPE


def kernel_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary of ``kernel``,
    valid only while the kernel source hashes to the value recorded there."""
    src = os.path.join(ROOT, "paper_2601_12220_b300", "csrc", kernel["source"])
    summ = os.path.join(ROOT, "profiles", kernel["profile"])
    if not (os.path.exists(src) and os.path.exists(summ)):
        return None
    h = source_hash(kernel["source"])
    got = {}
    for line in open(summ):
        if ":" in line:
            k, v = line.split(":", 1)
            got[k.strip().lstrip("-* ").strip()] = v.strip()
    if got.get("source_sha256_16") != h:
        return None
    try:
        return float(got["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(pg, per_rank_ms, units_per_rank, device=None):
    """Whole-job numbers of a replica run: the step time is the MAX over ranks
    (every rank waited at a barrier before and after its timed region) and
    the value counts the units of all ranks.  pg is torch.distributed or None."""
    import torch
    world = pg.get_world_size() if pg else 1
    t = torch.tensor([float(x) for x in per_rank_ms], dtype=torch.float64, device=device)
    if pg:
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
    ms = t.tolist()
    return ms, world * units_per_rank / (ms[0] * 1e-3)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_baseline(E_sample, reps=1, data=None):
    """The oracle as it stands, on E_sample elements of the same workload."""
    from oracle import evaluate as ev
    D, G, a, b = data if data is not None else W.dg_gradient(E=E_sample)
    text = W.dg_gradient_spec(E=E_sample)
    threads = ev.set_threads(cpu_cores())
    t = time.perf_counter()
    for _ in range(reps):
        ev.evaluate(text, dict(D=D, G=G, a=a, b=b))
    dt = (time.perf_counter() - t) / reps
    byts, _ = algorithmic(E_sample)
    return {"value": byts / dt / 1e9, "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": f"DG gradient with E={E_sample} of {E_FULL} elements (all outputs, FP64 nested loops), "
                      f"{reps} pass(es), {dt:.2f} s per pass"}


def run_reference(args):
    world, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    E_s = args.ref_sample
    data = W.dg_gradient(E=E_s)
    for _ in range(args.warmup):
        oracle_baseline(E_s, data=data)
    t = time.perf_counter()
    for _ in range(args.steps):
        cb = oracle_baseline(E_s, data=data)
    dt = (time.perf_counter() - t) / args.steps
    byts, flops = algorithmic(E_s)
    value = byts / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"dg_gradient_p4 (CPU oracle on E={E_s} per step)", "E": E_s,
                       "ndof": NDOF, "b": DIM, "producer": "sin(a)*b", "parallelism": "none (host cores)"},
            "cpu_baseline": {**cb, "value": value},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "tflops": flops / dt / 1e12}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_2601_12220_b300 as be

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    E = args.elements
    D, G, a, b = W.dg_gradient(E=E)
    host = dict(D=D, G=G, a=a, b=b)
    bufs = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    outs = [torch.empty((E, NDOF), dtype=torch.float64, device=dev) for _ in range(DIM)]
    text = W.dg_gradient_spec(E=E)
    ctx = be.Context(None, device=local)
    stream = torch.cuda.current_stream(dev)
    byts, flops = algorithmic(E)

    strat = be.plan_strategy(ctx, be.Einsum(text))
    kid = be.KERNEL_ELEMENT if strat == be.STRAT_ELEMENT else be.KERNEL_GENERIC

    forced = be.make_config(be.STRAT_ELEMENT, (0, 0, args.element_variant)) if args.element_variant else None

    def step():
        e = be.Einsum(text)                       # parse
        c = e.canonicalize()                      # normal form
        hit = ctx.lookup(c, be.PREC_FP64)         # tuning database
        cfg = forced or (hit[0] if hit else None)
        be.execute(ctx, e, bufs, outs, cfg=cfg, precision=be.PREC_FP64, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ctx.set_timing(True)
    with Clocks(local) as clk:
        t0.record(stream)
        for k in range(args.steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
    ctx.set_timing(False)
    if pg:
        pg.barrier()
    ms = t0.elapsed_time(t1) / args.steps
    n_launch, k_total = ctx.timing(kid)
    kms = k_total / max(1, n_launch)
    launches_per_step = n_launch / args.steps
    (ms, kms), value = aggregate(pg, [ms, kms], byts / 1e9, device=dev)

    # end to end through the public API with pinned host buffers
    pinned = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in host.items()}
    host_outs = [torch.empty((E, NDOF), dtype=torch.float64).pin_memory().numpy() for _ in range(DIM)]
    e_host = be.Einsum(text)
    for _ in range(max(1, args.warmup)):
        be.execute_host(ctx, e_host, pinned, host_outs, cfg=forced, stream=stream)
    if pg:
        pg.barrier()
    t = time.perf_counter()
    for _ in range(args.steps):
        e2 = be.Einsum(text)
        c2 = e2.canonicalize()
        hit = ctx.lookup(c2, be.PREC_FP64)
        be.execute_host(ctx, e2, pinned, host_outs, cfg=forced or (hit[0] if hit else None), stream=stream)
    e2e_s = (time.perf_counter() - t) / args.steps
    if pg:
        tt = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        e2e_s = tt.item()
    h2d = sum(v.nbytes for v in host.values())
    d2h = sum(o.nbytes for o in host_outs)

    peaks = load_peaks()
    # the default for this shape is the tensor-core variant (3)
    variant = args.element_variant or 3
    kernel = {1: {"name": "element_kernel", "source": "kernels_element.cu", "profile": "element_kernel_dg_p4.md"},
              2: {"name": "element_df_kernel", "source": "kernels_element_df.cu",
                  "profile": "element_df_kernel_dg_p4.md"},
              3: {"name": "element_tc_kernel", "source": "kernels_element_tc.cu",
                  "profile": "element_tc_kernel_dg_p4.md"}}[variant]
    ach_gb = byts / (kms * 1e-3) / 1e9
    traffic = kernel_traffic(kernel)
    hbm = {"achieved": ach_gb, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach_gb / peaks["hbm_gbs"],
           "peak_source": peaks["source"]}
    if variant == 3:                  # tensor cores: the path's roofline is HBM
        mma_tf = TC_MMA_FLOPS_PER_ELEMENT * E / (kms * 1e-3) / 1e12
        roofline = {"kernel": kernel["name"], "bound": "hbm", "achieved": ach_gb, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": ach_gb / peaks["hbm_gbs"], "peak_source": peaks["source"],
                    "traffic": traffic, "algorithmic_bytes": byts,
                    "tensor": {"achieved": mma_tf, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                               "frac": mma_tf / peaks["bf16_tflops"],
                               "counts": f"bf16 digit-product MMA flops issued ({TC_MMA_FLOPS_PER_ELEMENT} per element)"}}
    else:
        if variant == 1:              # FP64 pipe
            pp = pipe_peaks(be)
            ach_tf, peak, src = flops / (kms * 1e-3) / 1e12, pp["fp64"], pp["source"]
            what = "algorithmic FP64 flops"
        else:                         # double-float on the FP32 pipe
            ach_tf = DF_FLOPS_PER_ELEMENT * E / (kms * 1e-3) / 1e12
            pp = pipe_peaks(be)
            peak, src = pp["fp32"], pp["source"]
            what = f"FP32 flops of the compensated dot products ({DF_FLOPS_PER_ELEMENT} per element)"
        roofline = {"kernel": kernel["name"], "bound": "alu", "achieved": ach_tf, "peak": peak,
                    "unit": "TFLOP/s", "frac": ach_tf / peak, "counts": what,
                    "peak_source": src, "traffic": traffic, "algorithmic_bytes": byts, "hbm": hbm}
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"dg_gradient_p4: b=3 'rij,er,ej->ei', D 3x35x35 shared, G[E,3,3] sliced per row, "
                                   f"u=sin(a)*b fused, E={E}", "E": E, "ndof": NDOF, "b": DIM,
                       "global_batch": world * E, "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 ({byts / 1e6:.0f} MB per step), no flush",
                       "strategy": {1: "generic", 2: "element"}.get(strat, str(strat)),
                       "element_variant": {1: "fp64 pipe", 2: "double-float", 3: "tensor cores"}[variant]},
            "tflops": world * flops / (ms * 1e-3) / 1e12, "kernel_ms": kms,
            "roofline": roofline,
            "e2e": {"value": world * byts / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3},
            "clocks": clk.summary(), "gpu_launches": int(round(args.steps * launches_per_step))}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(args.cpu_sample)
    return line
    if pg:
        pg.destroy_process_group()


# ---------------------------------------------------------------- FEM action

def back_to_back_ms(torch, be, ctx, text, bufs, outs, stream, steps, cfg=None, precision=None):
    """Device time per launch of one parsed einsum's execute, back to back:
    the executes are queued behind a bounded spin kernel while the host
    submits them, and one event pair brackets all of them (on an idle GPU a
    per-launch event pair would also count the host's submission).  Returns
    (ms per launch, host seconds per execute)."""
    e = be.Einsum(text)
    kw = {} if precision is None else {"precision": precision}
    hit = ctx.lookup(e.canonicalize(), **kw)
    cfg = cfg or (hit[0] if hit else None)
    be.execute(ctx, e, bufs, outs, cfg=cfg, stream=stream, **kw)
    torch.cuda.synchronize()
    hs = []
    for _ in range(10):
        h0 = time.perf_counter()
        be.execute(ctx, e, bufs, outs, cfg=cfg, stream=stream, **kw)
        hs.append(time.perf_counter() - h0)
    host_s = float(np.median(hs))                       # host time per execute
    torch.cuda.synchronize()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # spin for 4x the host's submission time of all the launches (20 ms to 1 s)
    torch.cuda._sleep(int(2.0e9 * min(1.0, max(20e-3, 4.0 * host_s * steps))))
    k0.record(stream)
    for _ in range(steps):
        be.execute(ctx, e, bufs, outs, cfg=cfg, stream=stream, **kw)
    k1.record(stream)
    torch.cuda.synchronize()
    return k0.elapsed_time(k1) / steps, host_s


def run_fem(args):
    """FEM action 'ij,ej->ei', b = 4 rows sharing D (4 x 4), E = 4096: time per
    batched einsum through be_execute and as a CUDA-graph replay of a batch,
    plus canonicalization of 200 copies under random renames, row and
    operand permutations (latency p50 / p99 and one key for all)."""
    import torch
    import paper_2601_12220_b300 as be

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    E = args.fem_e
    peaks = load_peaks()
    D, us = W.fem_action(E=E)
    host = {"D": D, **{f"u{k}": u for k, u in enumerate(us)}}
    bufs = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    outs = [torch.empty((E, 4), dtype=torch.float64, device=dev) for _ in range(4)]
    text = W.fem_action_spec(E=E)
    ctx = be.Context(None, device=local)
    stream = torch.cuda.current_stream(dev)
    byts = 8.0 * (sum(v.size for v in host.values()) + 4 * E * 4)

    def step():
        e = be.Einsum(text)
        c = e.canonicalize()
        hit = ctx.lookup(c)
        be.execute(ctx, e, bufs, outs, cfg=hit[0] if hit else None, stream=stream)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    steps = max(args.steps, 100)
    with Clocks(local) as clk:
        ms = timed(step, steps)
    # kernel time per launch, back to back (the step's host work left out)
    kms_b2b, host_s = back_to_back_ms(torch, be, ctx, text, bufs, outs, stream, steps)
    n_k, t_k = steps, kms_b2b * steps
    batch = be.Batch(ctx, [(be.Einsum(text), bufs, outs)])
    ms_graph = timed(lambda: batch.run(stream), steps)
    # canonicalization of 200 relabeled copies
    ins, out = ["ij", "ej"], "ei"
    rows = [["D", f"u{k}"] for k in range(4)]
    g = W.rng(1, 77)
    lat, keys = [], set()
    for _ in range(200):
        r = W.relabel(out, ins, rows, g)
        lens = {r.rename["i"]: 4, r.rename["j"]: 4, r.rename["e"]: E}
        decl = {}
        for row in r.rows:
            for q, a in enumerate(row):
                decl[a] = ",".join(str(lens[c]) for c in r.ins[q])
        t = (f"{','.join(r.ins)}->{r.out} | " + " | ".join(",".join(x) for x in r.rows) + " ; " +
             " ; ".join(f"{a}:f64[{sh}]" for a, sh in decl.items()))
        e = be.Einsum(t)
        a0 = time.perf_counter()
        c = e.canonicalize()
        lat.append(time.perf_counter() - a0)
        keys.add(c.key)
    lat = np.sort(np.asarray(lat)) * 1e6
    line = {"metric": METRIC, "value": world * 1e3 / ms, "unit": "batched einsums/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"fem_action: b=4 'ij,ej->ei', D 4x4 shared, E={E}, U[-1,1]",
                       "parallelism": f"replicas x{world}",
                       "l2": f"inputs in L2 ({byts / 2**20:.1f} MB)" if byts < 100e6
                       else f"inputs larger than L2 ({byts / 1e9:.2f} GB per step), no flush"},
            "einsums_per_s": world * 4e3 / ms, "gb_s": world * byts / (ms * 1e-3) / 1e9,
            "kernel_ms": t_k / max(1, n_k), "execute_host_us": host_s * 1e6,
            "roofline": {"kernel": "element kernel", "bound": "hbm",
                         "achieved": byts / (t_k / max(1, n_k) * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": byts / (t_k / max(1, n_k) * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "peak_source": peaks["source"],
                         "timing": f"CUDA events around {steps} back-to-back launches queued behind a spin kernel",
                         "traffic": None},
            "graph_replay": {"ms_per_step": ms_graph, "batched_einsums_per_s": world * 1e3 / ms_graph},
            "canonicalize_200_copies": {"p50_us": float(lat[len(lat) // 2]), "p99_us": float(lat[int(0.99 * len(lat))]),
                                        "distinct_keys": len(keys), "key": sorted(keys)[0]},
            "clocks": clk.summary(), "gpu_launches": n_k}
    return line


# ------------------------------------------- DG divergence and face mass

def run_stacked(args):
    """DG local divergence 'xre,rij,xej->ei' (select producer over x) or
    face mass 'fe,ifj,fej->ei', b rows sharing the operator, on the element
    strategy's stacked form; the same einsum on the generic loop-nest
    kernel is timed beside it."""
    import torch
    import paper_2601_12220_b300 as be

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    E, order, rows = args.stacked_elements, args.order, args.rows
    N = W.tet_dofs(order)
    if args.workload == "dg_divergence":
        D, data = W.dg_divergence(E=E, order=order, rows=rows)
        host = W.dg_divergence_arrays(D, data)
        text = W.dg_divergence_spec(E=E, order=order, rows=rows)
        X, S, NJ0 = 3, 3, N
        desc = f"dg_divergence_p{order}: b={rows} 'xre,rij,xej->ei', D 3x{N}x{N} shared, F selects u/v/w by x, E={E}"
    else:
        M, data = W.face_mass(E=E, order=order, rows=rows)
        host = W.face_mass_arrays(M, data)
        text = W.face_mass_spec(E=E, order=order, rows=rows)
        X, S, NJ0 = 1, 4, W.tri_dofs(order)
        desc = f"face_mass_p{order}: b={rows} 'fe,ifj,fej->ei', M {N}x4x{NJ0} shared, E={E}"
    K = S * NJ0
    bufs = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    outs = [torch.empty((E, N), dtype=torch.float64, device=dev) for _ in range(rows)]
    ctx = be.Context(None, device=local)
    stream = torch.cuda.current_stream(dev)
    byts = 8.0 * sum(v.size for k, v in host.items()) + 8.0 * rows * E * N
    # FP32 flops of the double-float kernel: 15 per compensated term over the
    # contraction (N x K) and the production of v (K x X), per row
    df_flops = 15.0 * rows * E * (N * K + K * X)
    strat = be.plan_strategy(ctx, be.Einsum(text))
    # the element variant: double-float by default for the stacked form;
    # --element-variant 3 runs the tensor-core kernel (contractions of up to
    # 64 values: every face mass, the divergence up to P3)
    variant = args.element_variant or 2
    forced = be.make_config(be.STRAT_ELEMENT, (0, 0, args.element_variant)) if args.element_variant else None
    # bf16 MMA flops the tensor-core kernel issues per element and row: per
    # K-slice of 16 and column block of 32, u's six digits against D's
    # planes p <= 6 - q (26 planes of 32 columns)
    ncb = (N + 31) // 32
    tc_mma_flops = 2.0 * 16 * ((K + 15) // 16) * ncb * 32 * 26 * E * rows

    def step(cfg=None):
        e = be.Einsum(text)
        c = e.canonicalize()
        hit = ctx.lookup(c, be.PREC_FP64)
        be.execute(ctx, e, bufs, outs, cfg=cfg or forced or (hit[0] if hit else None), precision=be.PREC_FP64,
                   stream=stream)

    def timed(cfg, steps):
        for _ in range(args.warmup):
            step(cfg)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            step(cfg)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    with Clocks(local) as clk:
        ms = timed(None, args.steps)
    n_launch = args.steps                     # one element-kernel launch per step
    # kernel time per launch, back to back (the step's host work left out)
    kms, _ = back_to_back_ms(torch, be, ctx, text, bufs, outs, stream, max(20, args.steps), cfg=forced,
                             precision=be.PREC_FP64)
    gen_ms = timed(be.make_config(be.STRAT_GENERIC), max(3, args.steps // 4))
    peaks = load_peaks()
    ach_tf = df_flops / (kms * 1e-3) / 1e12
    ach_gb = byts / (kms * 1e-3) / 1e9
    if variant == 3:
        ach_mma = tc_mma_flops / (kms * 1e-3) / 1e12
        roof = {"kernel": "element_tc_kernel (stacked form)", "bound": "hbm", "achieved": ach_gb,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach_gb / peaks["hbm_gbs"],
                "peak_source": peaks["source"], "traffic": None, "algorithmic_bytes": byts,
                "timing": "CUDA events around back-to-back launches queued behind a spin kernel",
                "tensor": {"achieved": ach_mma, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                           "frac": ach_mma / peaks["bf16_tflops"],
                           "counts": "bf16 digit-product MMA flops issued (26 planes of 32 columns per K-slice and "
                                     "column block)"}}
    else:
        roof = {"kernel": "element_df_kernel" if variant == 2 else "element_kernel", "bound": "alu",
                "achieved": ach_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach_tf / FP32_PEAK_TFLOPS,
                "timing": "CUDA events around back-to-back launches queued behind a spin kernel",
                "counts": "FP32 flops of the compensated terms (15 per term, contraction and production)",
                "peak_source": "FP32 pipe from unit counts and clock: 148 SMs x 128 lanes x 2 x 2.032 GHz",
                "traffic": None, "algorithmic_bytes": byts,
                "hbm": {"achieved": ach_gb, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": ach_gb / peaks["hbm_gbs"], "peak_source": peaks["source"]}}
    line = {"metric": METRIC, "value": world * byts / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "E": E, "order": order, "b": rows, "K": K,
                       "parallelism": f"replicas x{world}", "l2": f"{byts / 1e6:.0f} MB per step, no flush",
                       "strategy": {1: "generic", 2: "element"}.get(strat, str(strat)),
                       "element_variant": {1: "fp64 pipe", 2: "double-float", 3: "tensor cores"}[variant]
                                          + " (stacked form)"},
            "kernel_ms": kms,
            "roofline": roof,
            "generic": {"ms_per_step": gen_ms, "value": world * byts / (gen_ms * 1e-3) / 1e9,
                        "speedup_of_element": gen_ms / ms},
            "clocks": clk.summary(), "gpu_launches": n_launch}
    return line


# ---------------------------------------------------------------- workload 3

V_FULL, O_FULL, B_CHEM = 128, 32, 4
SPLIT_PRODUCTS = 6             # BF16 tensor products per output term of the split GEMM (three parts per operand)
SPLIT_DTYPE = "f64 (split: 3 BF16 parts per operand, 6 tensor products, FP32 accumulation, FP32-pair drains)"


def chem_device_inputs(torch, dev, v, o, seed=1003):
    """The dense workload's operands drawn on the device (torch's Philox
    generator, seeded): A_k[a,b,e,f] = N(0,1) exp(-(|a-e|+|b-f|)/8), k < 4,
    and the shared T[e,f,i,j] = N(0,1) exp(-(|e-i|+|f-j|)/8) -- the shapes
    and decay of the workload without 8.6 GB of host generation and copy."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    ia = torch.arange(v, device=dev, dtype=torch.float64)
    io = torch.arange(o, device=dev, dtype=torch.float64)
    wv = torch.exp(-(ia[:, None] - ia[None, :]).abs() / 8.0)          # [a, e]
    wo = torch.exp(-(ia[:, None] - io[None, :]).abs() / 8.0)          # [e, i]
    bufs = {}
    for k in range(B_CHEM):
        A = torch.randn((v, v, v, v), generator=g, device=dev, dtype=torch.float64)
        A *= wv[:, None, :, None]
        A *= wv[None, :, None, :]
        bufs[f"A{k}"] = A
    T = torch.randn((v, v, o, o), generator=g, device=dev, dtype=torch.float64)
    T *= wo[:, None, :, None] * wo[None, :, None, :]
    bufs["T"] = T
    return bufs


def chem_sampled_error(torch, bufs, outs, v, o, n=256, seed=7):
    """Componentwise error of sampled outputs (a, b, i, j) of every row
    against an FP64 dot product of the same operands (numpy), relative to
    the absolute contraction S = sum |A| |T|: max and median."""
    rng = np.random.default_rng(seed)
    T = bufs["T"].reshape(v * v, o * o)
    rel = []
    for k in range(len(outs)):
        A = bufs[f"A{k}"].reshape(v * v, v * v)
        C = outs[k].reshape(v * v, o * o)
        m = rng.integers(0, v * v, n)
        c = rng.integers(0, o * o, n)
        a = A[torch.as_tensor(m, device=A.device)].cpu().numpy()
        t = T[:, torch.as_tensor(c, device=T.device)].cpu().numpy()
        got = C[torch.as_tensor(m, device=C.device), torch.as_tensor(c, device=C.device)].cpu().numpy()
        ref = np.einsum("nk,kn->n", a, t)
        S = np.einsum("nk,kn->n", np.abs(a), np.abs(t))
        rel.append(np.abs(got - ref) / S)
    rel = np.concatenate(rel)
    return {"max_over_S": float(rel.max()), "median_over_S": float(np.median(rel)), "samples": int(rel.size),
            "tolerance": 1e-6, "reference": "FP64 dot products of the sampled rows and columns (numpy)"}


def run_chem(args):
    """Dense cluster contraction 'abef,efij->abij' (v=128, o=32, b=4) on the
    split-precision tensor-core path."""
    import torch
    import paper_2601_12220_b300 as be

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    v, o = args.chem_v, args.chem_o
    bufs = chem_device_inputs(torch, dev, v, o)
    outs = [torch.empty((v, v, o, o), dtype=torch.float64, device=dev) for _ in range(B_CHEM)]
    text = W.chem_dense_spec(v=v, o=o)
    ctx = be.Context(None, device=local)
    stream = torch.cuda.current_stream(dev)
    M, N, K = v * v, o * o, v * v
    useful = B_CHEM * 2.0 * M * N * K
    byts = 8.0 * (B_CHEM * M * K + K * N + B_CHEM * M * N)
    pad = lambda x, t: (x + t - 1) // t * t
    issued = B_CHEM * SPLIT_PRODUCTS * 2.0 * pad(M, 128) * pad(N, 128) * pad(K, 64)

    def step():
        e = be.Einsum(text)
        c = e.canonicalize()
        hit = ctx.lookup(c, be.PREC_SPLIT)
        be.execute(ctx, e, bufs, outs, cfg=hit[0] if hit else None, precision=be.PREC_SPLIT, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.set_timing(True)
    with Clocks(local) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
    ctx.set_timing(False)
    assert ctx.status() == be.OK
    err = chem_sampled_error(torch, bufs, outs, v, o)
    ms = t0.elapsed_time(t1) / args.steps
    n_g, t_g = ctx.timing(be.KERNEL_DENSE_GEMM)
    n_s, t_s = ctx.timing(be.KERNEL_SPLIT)
    gemm_ms = t_g / max(1, n_g)
    peaks = load_peaks()
    bf16_peak = peaks["bf16_tflops"]
    per_launch_useful = useful / B_CHEM
    ach = per_launch_useful / (gemm_ms * 1e-3) / 1e12
    ach_issued = issued / B_CHEM / (gemm_ms * 1e-3) / 1e12
    line = {"metric": METRIC, "value": world * useful / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": SPLIT_DTYPE,
            "data": "synthetic",
            "config": {"workload": f"chem_dense: b={B_CHEM} 'abef,efij->abij', v={v}, o={o}, efij shared, "
                                   "entries N(0,1)*exp(-gap/8) (drawn on the device)", "parallelism": "replicas",
                       "l2": f"inputs larger than L2 ({byts / 1e9:.1f} GB per step)"},
            "gb_s": world * byts / (ms * 1e-3) / 1e9,
            "kernels": {"gemm_split_kernel_ms": gemm_ms, "gemm_launches": n_g,
                        "split_ms_per_step": t_s / args.steps, "split_launches": n_s},
            "roofline": {"kernel": "gemm_split_kernel", "bound": "tensor", "achieved": ach, "peak": bf16_peak,
                         "unit": "TFLOP/s", "frac": ach / bf16_peak,
                         "achieved_issued": ach_issued, "frac_issued": ach_issued / bf16_peak,
                         "counts": f"achieved: useful FP64-equivalent flops (2 M N K); issued: the {SPLIT_PRODUCTS} BF16 "
                                   "products on the padded tile grid",
                         "peak_source": f"measured bf16 burst ({peaks['source']})",
                         "traffic": kernel_traffic({"source": "kernels_dense.cu",
                                                    "profile": "gemm_split_kernel_chem.md"})},
            "error_vs_fp64": err,
            "clocks": clk.summary(), "gpu_launches": n_g + n_s}
    return line


def run_affine(args):
    """TCCG-shaped contraction 'abcd,cdef->abef' (every extent args.affine_n)
    with affine producers (alpha1 A + beta1)(alpha2 B + beta2) fused into the
    split-precision tensor-core path; the plain contraction is timed beside it."""
    import torch
    import paper_2601_12220_b300 as be

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.affine_n
    g = W.rng(8, 0)
    A = g.standard_normal((n, n, n, n))
    B = W.rng(8, 1).standard_normal((n, n, n, n))
    bufs = {"A": torch.from_numpy(A).to(dev), "B": torch.from_numpy(B).to(dev)}
    out = [torch.empty((n, n, n, n), dtype=torch.float64, device=dev)]
    decl = f"A:f64[{n},{n},{n},{n}] ; B:f64[{n},{n},{n},{n}]"
    text = (f"abcd,cdef->abef | P,Q ; {decl} ; P(a,b,c,d) := $a1*A[a,b,c,d]+$b1 ; "
            f"Q(c,d,e,f) := $a2*B[c,d,e,f]+$b2")
    plain = f"abcd,cdef->abef | A,B ; {decl}"
    sc = (0.5, -1.25, 2.0, 0.75)
    ctx = be.Context(None, device=local)
    stream = torch.cuda.current_stream(dev)
    M = N = K = n * n
    useful = 2.0 * M * N * K
    byts = 8.0 * (M * K + K * N + M * N)
    pad = lambda x, t: (x + t - 1) // t * t
    issued = SPLIT_PRODUCTS * 2.0 * pad(M, 128) * pad(N, 128) * pad(K, 64)

    def timed(t, scalars, steps):
        def step():
            e = be.Einsum(t)
            c = e.canonicalize()
            hit = ctx.lookup(c, be.PREC_SPLIT)
            be.execute(ctx, e, bufs, out, cfg=hit[0] if hit else None, precision=be.PREC_SPLIT, scalars=scalars,
                       stream=stream)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    strat = be.plan_strategy(ctx, be.Einsum(text), precision=be.PREC_SPLIT)
    ctx.set_timing(True)
    with Clocks(local) as clk:
        ms = timed(text, sc, args.steps)
    ctx.set_timing(False)
    assert ctx.status() == be.OK
    n_g, t_g = ctx.timing(be.KERNEL_DENSE_GEMM)
    n_s, t_s = ctx.timing(be.KERNEL_SPLIT)
    gemm_ms = t_g / max(1, n_g)
    # componentwise error of sampled outputs of the affine contraction (its
    # result is in `out` after the timed steps; the plain run follows)
    rs = np.random.default_rng(11)
    mi, ni = rs.integers(0, M, 256), rs.integers(0, N, 256)
    Pm = sc[0] * A.reshape(M, K)[mi] + sc[1]
    Qn = sc[2] * B.reshape(K, N)[:, ni] + sc[3]
    got = out[0].reshape(M, N)[torch.as_tensor(mi, device=dev), torch.as_tensor(ni, device=dev)].cpu().numpy()
    ref = np.einsum("nk,kn->n", Pm, Qn)
    S = np.einsum("nk,kn->n", np.abs(Pm), np.abs(Qn))
    rel = np.abs(got - ref) / S
    err = {"max_over_S": float(rel.max()), "median_over_S": float(np.median(rel)), "samples": int(rel.size),
           "tolerance": 1e-6, "reference": "FP64 dot products of the sampled rows and columns (numpy)"}
    plain_ms = timed(plain, (), args.steps)
    peaks = load_peaks()
    bf16_peak = peaks["bf16_tflops"]
    ach = useful / (gemm_ms * 1e-3) / 1e12
    ach_issued = issued / (gemm_ms * 1e-3) / 1e12
    line = {"metric": METRIC, "value": world * useful / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": SPLIT_DTYPE,
            "data": "synthetic",
            "config": {"workload": f"dense_affine: 'abcd,cdef->abef', extents {n}, operands "
                                   "(0.5 A - 1.25), (2 B + 0.75) as runtime-scalar affine producers, N(0,1)",
                       "M": M, "N": N, "K": K, "parallelism": "replicas",
                       "strategy": {1: "generic", 3: "dense split"}.get(strat, str(strat)),
                       "l2": f"inputs larger than L2 ({byts / 1e9:.2f} GB per step)"},
            "kernels": {"gemm_split_kernel_ms": gemm_ms, "split_ms_per_step": t_s / args.steps},
            "plain": {"ms_per_step": plain_ms, "value": world * useful / (plain_ms * 1e-3) / 1e12},
            "roofline": {"kernel": "gemm_split_kernel", "bound": "tensor", "achieved": ach, "peak": bf16_peak,
                         "unit": "TFLOP/s", "frac": ach / bf16_peak, "achieved_issued": ach_issued,
                         "frac_issued": ach_issued / bf16_peak,
                         "peak_source": f"measured bf16 burst ({peaks['source']})", "traffic": None},
            "error_vs_fp64": err,
            "clocks": clk.summary(), "gpu_launches": n_g + n_s}
    return line


# ---------------------------------------------------------------- workload 4

def factored_macs(out, ins, lens, min_gain=1.5):
    """Multiply-adds of one row under the order of steps the batched executor
    picks (fewest multiply-adds over all orders of two-operand contractions
    and of one-operand sums of an operand's own letters) when it cuts the
    loop nest's (volume x (operands - 1)) at least min_gain times and the
    notation has 2 to 5 operands; None otherwise (the row then runs its loop
    nest)."""
    import itertools
    if not 2 <= len(ins) <= 5:
        return None
    vol = lambda letters: math.prod(lens[c] for c in letters)
    all_l = set(out).union(*[set(x) for x in ins])
    direct = vol(all_l) * (len(ins) - 1)
    best = [direct / min_gain]
    found = [False]

    def rec(slots, cost):
        if len(slots) == 1:
            if cost < best[0]:
                best[0], found[0] = cost, True
            return
        for a in range(len(slots)):
            rest = set(out).union(*[slots[k] for k in range(len(slots)) if k != a])
            keep = slots[a] & rest
            c = cost + vol(slots[a])
            if keep != slots[a] and c < best[0]:
                rec(slots[:a] + [keep] + slots[a + 1:], c)
        for a, b in itertools.combinations(range(len(slots)), 2):
            rest = set(out).union(*[slots[k] for k in range(len(slots)) if k not in (a, b)])
            both = slots[a] | slots[b]
            c = cost + vol(both)
            if c < best[0]:
                rec([slots[k] for k in range(len(slots)) if k not in (a, b)] + [both & rest], c)

    rec([set(x) for x in ins], 0.0)
    return best[0] if found[0] else None


def run_mix(args):
    """Uneven batch: N instances drawn from twelve notations of the paper, each
    under a random rename / row / operand permutation, lengths round(2^U(3,12))
    capped, f64 or f32, b in 1..4 -- evaluated by one persistent launch (CUDA
    graph replay) and, for comparison, by one be_execute launch per instance."""
    import torch
    import paper_2601_12220_b300 as be

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g = W.rng(4, 0)
    items, insts, byts, n_rows = [], [], 0, 0
    fl64, fl32 = 0.0, 0.0          # loop-nest flops of the f64 and f32 instances
    for _ in range(args.mix_n):
        inst = W.mix_instance(g, max_operand=1 << args.mix_operand_log2, max_flops=1 << args.mix_flops_log2)
        f = len(inst.rows) * W._flops(inst.out, inst.ins, inst.lens)
        if "64" in str(inst.dtype):
            fl64 += f
        else:
            fl32 += f
        arrs = W.instance_arrays(inst, g)
        e = be.Einsum(W.instance_spec(inst))
        dt = torch.float64 if e.out_dtype == be.F64 else torch.float32
        bufs = {k: torch.from_numpy(v).to(dev) for k, v in arrs.items()}
        outs = [torch.empty(e.out_shape, dtype=dt, device=dev) for _ in range(e.b)]
        items.append((e, bufs, outs))
        insts.append(inst)
        byts += sum(v.nbytes for v in arrs.values()) + sum(o.numel() * o.element_size() for o in outs)
        n_rows += e.b
    ctx = be.Context(None, device=local)
    stream = torch.cuda.current_stream(dev)
    # strategy policy: element-shaped FP64 instances on the element strategy;
    # FP64 GEMM-form instances of >= 2^mix_split_log2 multiply-adds on the
    # split-precision tensor cores (held to 1e-6 S) unless --mix-no-split
    policy = be.make_config(tile=(0, 0, 0, args.mix_split_log2), split=0 if args.mix_no_split else 1)
    t_plan = time.perf_counter()
    batch = be.Batch(ctx, items, policy)
    t_plan = time.perf_counter() - t_plan
    info = batch.info()
    kinds = batch.kinds()
    # per-instance bound: HBM for element instances, the BF16 tensor pipe for
    # split instances (3 products), the FP64 / FP32 pipe for generic ones
    peaks0 = load_peaks()
    bf16 = peaks0["bf16_tflops"] * 1e12
    pipe_s = {"hbm": 0.0, "tensor": 0.0, "fp64": 0.0, "fp32": 0.0}
    gen_work = {"fp64": 0.0, "fp32": 0.0}   # flops of the generic instances' evaluations
    n_fac_expected = 0
    for (e, bufs, outs), inst in zip(items, insts):
        f = len(inst.rows) * W._flops(inst.out, inst.ins, inst.lens)
        nbytes = sum(t.numel() * t.element_size() for t in bufs.values()) + \
            sum(o.numel() * o.element_size() for o in outs)
        if be.plan_strategy(ctx, e) == be.STRAT_ELEMENT:
            pipe_s["hbm"] += nbytes / (peaks0["hbm_gbs"] * 1e9)
        elif (not args.mix_no_split and "64" in str(inst.dtype) and f / 2 >= 2 ** args.mix_split_log2 and
              be.plan_strategy(ctx, e, precision=be.PREC_SPLIT) == be.STRAT_DENSE_SPLIT):
            pipe_s["tensor"] += SPLIT_PRODUCTS * f / bf16
        else:
            # generic: the work of the evaluation the batch runs (a factored
            # instance's pairwise steps, else its loop nest)
            fm = factored_macs(inst.out, inst.ins, inst.lens)
            if fm is not None:
                f = len(inst.rows) * 2.0 * fm
                n_fac_expected += 1
            pipe = "fp64" if "64" in str(inst.dtype) else "fp32"
            pipe_s[pipe] += f / (pipe_peaks(be)[pipe] * 1e12)
            gen_work[pipe] += f

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b2.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b2) / steps

    def per_instance():
        for e, bufs, outs in items:
            be.execute(ctx, e, bufs, outs, stream=stream)

    ctx.set_timing(True)
    with Clocks(local) as clk:
        ms_batch = timed(lambda: batch.run(stream), args.steps, args.warmup)
    ctx.set_timing(False)
    n_k, t_k = ctx.timing(be.KERNEL_PERSISTENT)
    assert ctx.status() == be.OK
    ms_single = timed(per_instance, max(1, args.steps // 2), 1)
    generic_only = be.Batch(ctx, items, be.make_config(stage_mask=1))
    ms_generic = timed(lambda: generic_only.run(stream), max(1, args.steps // 2), 1)
    generic_only.close()
    # the same policy with every generic instance on its loop nest (no factoring)
    unfactored = be.Batch(ctx, items, be.make_config(tile=(0, 0, 0, args.mix_split_log2),
                                                      split=0 if args.mix_no_split else 1, stage_mask=2))
    ms_unfactored = timed(lambda: unfactored.run(stream), max(1, args.steps // 2), 1)
    unfactored.close()
    fac = batch.factored()
    peaks = load_peaks()
    kms = t_k / max(1, n_k)
    g64, g32 = gen_work["fp64"], gen_work["fp32"]
    line = {"metric": METRIC, "value": world * args.mix_n / (ms_batch * 1e-3), "unit": "einsums/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32 mix",
            "data": "synthetic",
            "config": {"workload": f"uneven_mix: {args.mix_n} instances of 12 notations, lengths round(2^U(3,12)), "
                                   f"operands <= 2^{args.mix_operand_log2}, flops <= 2^{args.mix_flops_log2}",
                       "rows": n_rows, "tiles": info["tiles"], "plan_s": t_plan, "parallelism": "replicas"},
            "rows_per_s": world * n_rows / (ms_batch * 1e-3),
            "instances_per_strategy": kinds,
            "one_launch_per_einsum": {"ms_per_step": ms_single, "einsums_per_s": args.mix_n / (ms_single * 1e-3)},
            "speedup_vs_one_launch_per_einsum": ms_single / ms_batch,
            "all_generic_batch": {"ms_per_step": ms_generic, "einsums_per_s": args.mix_n / (ms_generic * 1e-3)},
            "factored": dict(fac, unfactored_batch={"ms_per_step": ms_unfactored,
                                                    "einsums_per_s": args.mix_n / (ms_unfactored * 1e-3)}),
            "per_pipe_bound_ms": {k: v * 1e3 for k, v in pipe_s.items()},
            "roofline_per_instance_pipe": {
                "bound_ms": max(pipe_s.values()) * 1e3, "serial_bound_ms": sum(pipe_s.values()) * 1e3,
                "frac": max(pipe_s.values()) / (ms_batch * 1e-3),
                "frac_serial": sum(pipe_s.values()) / (ms_batch * 1e-3),
                "factored_instances_counted": n_fac_expected,
                "counts": "each instance at its own pipe's peak: element instances' bytes at measured HBM, split "
                          "instances' issued BF16 flops (6 products) at the measured bf16 rate, generic f64 / f32 "
                          "instances' flops at the measured FP64 / FP32 rates (a factored instance's pairwise steps, "
                          "2 x multiply-adds; else its loop nest, 2 x volume x (operands - 1)); bound = the busiest "
                          "pipe (pipes overlap), serial = their sum"},
            "gb_s": world * byts / (ms_batch * 1e-3) / 1e9,
            "roofline": {"kernel": "persistent_kernel", "bound": "alu",
                         "achieved": (g64 + g32) / (kms * 1e-3) / 1e12,
                         "peak": (g64 + g32) / (g64 / (pipe_peaks(be)["fp64"] * 1e12) + g32 / (pipe_peaks(be)["fp32"] * 1e12)) / 1e12,
                         "unit": "TFLOP/s",
                         "frac": (g64 / (pipe_peaks(be)["fp64"] * 1e12) + g32 / (pipe_peaks(be)["fp32"] * 1e12)) / (kms * 1e-3),
                         "counts": "flops of the generic instances' evaluations (factored pairwise steps, else the loop "
                                   "nest), over the whole batch run (its graph: persistent launches and the element and "
                                   "split branches beside them); peak: the time at the measured FP64 rate for the f64 "
                                   "instances plus the measured FP32 rate for the f32 ones",
                         "loop_nest_flops": fl64 + fl32,
                         "traffic": None, "algorithmic_bytes": byts,
                         "hbm": {"achieved": byts / (kms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": byts / (kms * 1e-3) / 1e9 / peaks["hbm_gbs"]}},
            "clocks": clk.summary(), "gpu_launches": n_k}
    return line


# ---------------------------------------------------------------- workload 5

def run_serving(args):
    """Poisson request stream through the serving loop: 80 % requests drawn
    from the uneven mix (lengths 8..512), 10 % FEM-action and 10 % DG-gradient
    shaped requests (E = 4096 so the stream is servable), operands resident
    on the device.  Reports einsums/s and p50/p99 latency, and the same
    arrival sequence served one launch per einsum (a single FIFO server
    whose per-request times are measured, with queueing replayed)."""
    import torch
    import paper_2601_12220_b300 as be

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g = W.rng(5, 1)
    templates = []
    for k in range(args.serve_templates):
        kind = g.random()
        if kind < 0.1:
            D, us = W.fem_action(E=4096)
            e = be.Einsum(W.fem_action_spec(E=4096))
            host = {"D": D, **{f"u{q}": u for q, u in enumerate(us)}}
        elif kind < 0.2:
            D, G, a, b = W.dg_gradient(E=4096)
            e = be.Einsum(W.dg_gradient_spec(E=4096))
            host = dict(D=D, G=G, a=a, b=b)
        else:
            inst = W.mix_instance(g, lo_exp=3.0, hi_exp=9.0, max_operand=1 << 20, max_flops=1 << 24)
            e = be.Einsum(W.instance_spec(inst))
            host = W.instance_arrays(inst, g)
        dt = torch.float64 if e.out_dtype == be.F64 else torch.float32
        bufs = {a: torch.from_numpy(v).to(dev) for a, v in host.items()}
        outs = [torch.empty(e.out_shape, dtype=dt, device=dev) for _ in range(e.b)]
        templates.append((e, bufs, outs))
    ctx = be.Context(None, device=local, hbm_budget=64 << 30)
    srv = be.Server(ctx, n_streams=args.serve_streams, hbm_budget=64 << 30)
    prepared = [srv.prepare(*t) for t in templates]
    arrivals = W.poisson_arrivals(args.serve_rate, args.serve_seconds)
    pick = W.rng(5, 2).integers(0, len(templates), size=len(arrivals))
    # warm-up: every template once
    for p in prepared:
        srv.submit(p)
    srv.drain(60.0)
    srv.reset_stats()

    def serve(arr, pk):
        t0 = time.perf_counter()
        for t, k in zip(arr, pk):
            while time.perf_counter() - t0 < t:
                pass
            srv.submit(prepared[k])
        submitted = time.perf_counter() - t0
        srv.drain(300.0)
        return submitted

    with Clocks(local) as clk:
        serve(arrivals, pick)
    st = srv.stats()
    # arrival-rate sweep: the same template mix at each offered rate, to
    # the rate where throughput stops following the offer (saturation)
    sweep = []
    for r in (float(x) for x in args.serve_sweep.split(",") if x.strip()):
        arr = W.poisson_arrivals(r, args.serve_sweep_seconds, seed_offset=3)
        pk = W.rng(5, 4).integers(0, len(templates), size=len(arr))
        srv.reset_stats()
        sub = serve(arr, pk)
        s2 = srv.stats()
        sweep.append({"offered_per_s": r, "submitted_per_s": len(arr) / max(sub, 1e-9),
                      "einsums_per_s": s2["throughput"], "latency_p50_ms": s2["p50_s"] * 1e3,
                      "latency_p99_ms": s2["p99_s"] * 1e3, "completed": s2["completed"],
                      "failed": s2["failed"], "max_inflight": s2["max_inflight"]})
    # one launch per einsum, same sequence: measured service times, FIFO replay
    service = np.zeros(len(templates))
    for k, (e, bufs, outs) in enumerate(templates):
        be.execute(ctx, e, bufs, outs)
        torch.cuda.synchronize()
        a = time.perf_counter()
        for _ in range(3):
            be.execute(ctx, e, bufs, outs)
            torch.cuda.synchronize()
        service[k] = (time.perf_counter() - a) / 3
    fin, lat = 0.0, []
    for t, k in zip(arrivals, pick):
        fin = max(fin, t) + service[k]
        lat.append(fin - t)
    lat = np.sort(np.asarray(lat))
    single_rate = len(arrivals) / (fin - arrivals[0])
    # kernel launches of the served sequence: each template's count (the same
    # on every execution), summed over the requests
    kinds = (be.KERNEL_ELEMENT, be.KERNEL_GENERIC, be.KERNEL_DENSE_GEMM, be.KERNEL_SPLIT, be.KERNEL_PERSISTENT)
    per_template = np.zeros(len(templates), dtype=np.int64)
    ctx.set_timing(True)
    for k, (e, bufs, outs) in enumerate(templates):
        be.execute(ctx, e, bufs, outs)
        torch.cuda.synchronize()
        per_template[k] = sum(ctx.timing(kd)[0] for kd in kinds)
    ctx.set_timing(False)
    launches = int(per_template[pick].sum())
    line = {"metric": METRIC, "value": world * st["throughput"], "unit": "einsums/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": 1e3 / max(st["throughput"], 1e-9), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32 mix", "data": "synthetic",
            "config": {"workload": f"serving: Poisson {args.serve_rate:.0f}/s for {args.serve_seconds} s, "
                                   f"{len(templates)} resident request templates (80 % uneven mix 8..512, "
                                   "10 % FEM action E=4096, 10 % DG gradient E=4096)",
                       "streams": args.serve_streams, "hbm_budget_gb": 64, "requests": len(arrivals),
                       "parallelism": "replicas"},
            "latency_p50_ms": st["p50_s"] * 1e3, "latency_p99_ms": st["p99_s"] * 1e3,
            "completed": st["completed"], "failed": st["failed"], "max_inflight": st["max_inflight"],
            "peak_inflight_bytes": st["peak_bytes"],
            "one_launch_per_einsum": {"einsums_per_s": single_rate,
                                      "latency_p50_ms": float(lat[len(lat) // 2]) * 1e3,
                                      "latency_p99_ms": float(lat[int(0.99 * (len(lat) - 1))]) * 1e3},
            "clocks": clk.summary(), "gpu_launches": launches}
    if sweep:
        line["rate_sweep"] = sweep
    srv.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--elements", type=int, default=E_FULL)
    ap.add_argument("--cpu-sample", type=int, default=E_FULL)
    ap.add_argument("--ref-sample", type=int, default=32768)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--element-variant", type=int, default=0,
                    help="element kernel: 0 the default (tensor cores where the shape allows, else "
                         "double-float), 1 FP64 pipe, 2 double-float, 3 tensor cores")
    ap.add_argument("--workload", default="dg_gradient",
                    choices=["dg_gradient", "chem_dense", "uneven_mix", "serving", "dg_divergence", "face_mass",
                             "dense_affine", "fem_action"])
    ap.add_argument("--affine-n", type=int, default=64, help="every extent of the dense_affine contraction")
    ap.add_argument("--order", type=int, default=4, help="polynomial order of dg_divergence / face_mass")
    ap.add_argument("--rows", type=int, default=1, help="einsums b of dg_divergence / face_mass")
    ap.add_argument("--stacked-elements", type=int, default=100000)
    ap.add_argument("--fem-e", type=int, default=4096, help="elements of the fem_action workload")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-sweep", default="",
                    help="comma-separated offered rates (requests/s) served after the main run, e.g. 5000,20000,80000")
    ap.add_argument("--serve-sweep-seconds", type=float, default=3.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-templates", type=int, default=256)
    ap.add_argument("--serve-streams", type=int, default=8)
    ap.add_argument("--mix-n", type=int, default=512)
    ap.add_argument("--mix-split-log2", type=int, default=23,
                    help="FP64 GEMM-form mix instances of at least 2^this multiply-adds take the split path")
    ap.add_argument("--mix-no-split", action="store_true",
                    help="keep FP64 GEMM-form mix instances on the FP64 generic path")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload only: skip the sub-objects of the other configurations")
    ap.add_argument("--mix-operand-log2", type=int, default=22)
    ap.add_argument("--mix-flops-log2", type=int, default=26)
    ap.add_argument("--chem-v", type=int, default=V_FULL)
    ap.add_argument("--chem-o", type=int, default=O_FULL)
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    if args.workload == "chem_dense":
        line = run_chem(args)
    elif args.workload == "uneven_mix":
        line = run_mix(args)
    elif args.workload == "serving":
        line = run_serving(args)
    elif args.workload in ("dg_divergence", "face_mass"):
        line = run_stacked(args)
    elif args.workload == "dense_affine":
        line = run_affine(args)
    elif args.workload == "fem_action":
        line = run_fem(args)
    else:
        line = run_ours(args)
        if line.get("n_gpus", 1) == 1 and not args.no_configs:
            line["configs"] = other_configs(args)
            import paper_2601_12220_b300 as be
            line["measured_pipe_peaks_tflops"] = pipe_peaks(be)
    if rank == 0:
        print(json.dumps(line), flush=True)


def other_configs(args):
    """The other configurations of the benchmark, one sub-object each (1 GPU,
    short runs): FEM action with canonicalization of 200 copies, the dense
    split-precision contraction with its error, the 512-instance uneven mix
    (batched vs one launch per einsum) and the serving loop (3 s Poisson
    stream at 20 k requests/s)."""
    import copy

    def sub(fn, **kw):
        a = copy.copy(args)
        for k, v in kw.items():
            setattr(a, k, v)
        t = time.perf_counter()
        try:
            d = fn(a)
        except Exception as exc:                       # reported, never hidden
            return {"error": f"{type(exc).__name__}: {exc}"}
        d.pop("metric", None)
        d["wall_s"] = time.perf_counter() - t
        return d

    return {
        "fem_action_b4_E4096": sub(run_fem, steps=100, warmup=5),
        "chem_dense_v128_o32_b4": sub(run_chem, steps=5, warmup=3),
        "uneven_mix_512": sub(run_mix, steps=6, warmup=3),
        "serving_poisson_20k": sub(run_serving, serve_seconds=3.0, serve_sweep=""),
        # the rows built beyond the five configurations, on the same run
        "dg_divergence_p4_b1": sub(run_stacked, workload="dg_divergence", order=4, rows=1, steps=10, warmup=3,
                                   element_variant=0),
        "face_mass_p4_b1": sub(run_stacked, workload="face_mass", order=4, rows=1, steps=10, warmup=3,
                               element_variant=0),
        "dense_affine_n96": sub(run_affine, affine_n=96, steps=5, warmup=3),
    }


if __name__ == "__main__":
    main()
