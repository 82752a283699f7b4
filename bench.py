#!/usr/bin/env python
"""Benchmark of one hdiff + vadv step (GT4Py paper, Sec. 3.1 benchmark
stencils) at 256x256x80 in FP64, through libgtb's C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gtb|reference]

A step is one pass of the whole hot path over one batch: hdiff (Laplacian,
limited fluxes, update) on one input set and vadv (coefficients, forward
elimination, back substitution) on another, co-scheduled in one launch
(gtb_step); the same step as two separate launches is timed beside it.
Prints ONE JSON line (rank 0).

* value: domain points per second (Mpoints/s) of whole steps, inputs resident
  in HBM, device time from CUDA events on the launching stream, max over ranks.
  Three input sets of ~380 MB each (> the 126 MB L2) rotate between steps.
* e2e: the same metric with the host<->device copies of every step's inputs
  (from pinned host memory) and of its two outputs inside the timed region;
  consecutive steps are pipelined (copy-in, compute, copy-out on three streams
  over two device buffer sets).
* roofline: the step kernel's algorithmic HBM bytes per launch over its
  average launch time, against the measured HBM copy bandwidth; beside it an
  "fp64" block: the binary64 operations the kernel executes per point (from its
  ncu summary), their rate, and the GPU's FP64 FMA issue rate measured in the
  same run by an FMA-chain probe kernel (the pipe that binds the column solve).
* cpu_baseline: the FP64 CPU oracle on the host cores (one thread per J-slab,
  every core the process may run on) on a bounded sample, with the
  single-thread figure beside it.
* precision: FP32 storage at 512x512x80 (binary32 hdiff; vadv in binary32,
  binary64 and double-float column arithmetic) beside the FP64 path there,
  with each form's error against the FP64 oracle (checked after the timing).
* batched: the 48-member ensemble of uneven domains, autotuned plan replayed
  from a CUDA graph vs the loop of single-domain launches, with its algorithmic
  HBM bytes and their rate.
* call_overhead: the paper's split of Python-call vs compiled-call time, for
  one step on the small 64x64x40 workload (device time, C-ABI call, Python call),
  and hdiff alone at 64x64x40 FP64 in microseconds.
* fused_chain: the chained step (vadv of hdiff's output) as two launches vs
  gtb_hdiff_vadv, one kernel that keeps h on chip.
* adjoint_forward_ratio: backward / forward time of one chained step
  (periodic halo + hdiff + vadv) through the adjoint kernels.
* literal_chain: the 10-step chain at 256x256x80 FP64 with wcon ~ U(-0.5, 0.5)
  as drawn, whose field grows without bound: max |field| after every step.
* --impl reference: the oracle itself (all host cores) as the reference arm.
Per-kernel times come from a second pass with an event around each kernel.
Under torchrun every rank runs its own replica (independent problems, no
collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hdiff/vadv Mpoints/s & HBM GB/s vs 8 TB/s roofline; adjoint/forward time ratio"
I, J, K = 256, 256, 80
POINTS = I * J * K
HDIFF_HALO, VADV_HALO = 2, 1
VADV_NAMES = ("u_stage", "wcon", "u_pos", "utens", "utens_stage")
WORKLOAD = "hdiff+vadv FP64 256x256x80 (hdiff halo 2, vadv halo 1 in I/J), dtr_stage=3/20, beta_v=0"


def hdiff_bytes(I, J, K, es):
    """Compulsory HBM bytes of one hdiff launch: in on the domain + 2-ring, coeff and out on the domain."""
    return es * ((I + 4) * (J + 4) * K + 2 * I * J * K)


def vadv_bytes(I, J, K, es):
    """u_stage, u_pos, utens, utens_stage read and out written on the domain; wcon on I+1 columns."""
    return es * (5 * I * J * K + (I + 1) * J * K)


def batched_bytes(shapes, es):
    """Compulsory HBM bytes of the batched form: per member, hdiff reads in on the domain
    and its 2-ring and coeff and writes h; vadv reads h (as u_stage and u_pos), wcon on
    I+1 columns, utens, utens_stage and writes out."""
    return sum(es * ((I + 4) * (J + 4) * K + 7 * I * J * K + J * K) for I, J, K in shapes)


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2311_08322_b300", "csrc")
    for n in sorted(os.listdir(csrc)):
        if n.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(csrc, n), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(kernel):
    """DRAM bytes per launch of `kernel` from profiles/ncu_*.txt, if captured on this source."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    src = kernel_source_hash()
    for n in sorted(os.listdir(pdir)):
        if not n.endswith(".txt"):
            continue
        txt = open(os.path.join(pdir, n)).read()
        m = re.search(r"^kernel_source_sha: (\w+)", txt, re.M)
        t = re.search(r"^dram_bytes_per_launch\[%s\]: ([0-9.eE+]+)" % kernel, txt, re.M)
        if m and t and m.group(1) == src:
            return float(t.group(1))
    return None


def profile_field(kernel, pattern):
    """A figure from the ncu summary of `kernel` (profiles/ncu_*.txt) captured on this
    source, by regular expression (first group), or None."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    src = kernel_source_hash()
    for n in sorted(os.listdir(pdir)):
        if not n.endswith(".txt"):
            continue
        txt = open(os.path.join(pdir, n)).read()
        m = re.search(r"^kernel_source_sha: (\w+)", txt, re.M)
        t = re.search(r"^dram_bytes_per_launch\[%s\]" % kernel, txt, re.M)
        v = re.search(pattern, txt, re.M)
        if m and t and v and m.group(1) == src:
            return float(v.group(1))
    return None


def fp64_fma_rate(reps=5):
    """The GPU's binary64 FMA issue rate (G FMA/s): gtb_probe_fp64_fma, 8 resident CTAs of
    256 threads per SM, each thread 8 independent FMA chains, timed with CUDA events;
    best of `reps` launches of ~10 G FMAs."""
    import torch
    from paper_2311_08322_b300 import gtb
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    gtb.probe_fp64_fma(sms * 8, 64, sink, stream)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n = gtb.probe_fp64_fma(sms * 8, 4096, sink, stream)
        b.record(stream)
        torch.cuda.synchronize()
        best = max(best, n / (a.elapsed_time(b) / 1e3))
    gtb.device_status()
    return best / 1e9


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.lines = []
        self.p = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 3.0:
            time.sleep(0.02)

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        rows = [r.split(", ") for r in self.lines if r and r[0].isdigit()]
        sm = [float(r[0]) for r in rows if len(r) >= 8]
        mx = [float(r[1]) for r in rows if len(r) >= 8]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows if len(r) >= 8 for q in range(4) if r[4 + q].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm),
                "power_w_max": max(float(r[2]) for r in rows) if rows else None}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest value of x over all ranks (the slowest rank's time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpoints(world: int, points_per_rank: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: every rank's points over the slowest rank's time."""
    return world * points_per_rank * steps / (max_ms / 1e3) / 1e6


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


_POOLS = {}


def oracle_slabs(fn, J_, n):
    """Run fn(j0, nj) over n contiguous J-slabs of [0, J_) on n threads (the oracle's C
    calls release the GIL, so the slabs run on n cores), returning when all are done.
    The thread pool of each size is created once and kept (its start-up stays out of
    the timings)."""
    from concurrent.futures import ThreadPoolExecutor
    n = max(1, min(n, J_))
    bounds = [(J_ * q // n, J_ * (q + 1) // n) for q in range(n)]
    if n == 1:
        fn(0, J_)
        return
    ex = _POOLS.get(n)
    if ex is None:
        ex = _POOLS[n] = ThreadPoolExecutor(n)
    list(ex.map(lambda b: fn(b[0], b[1] - b[0]), bounds))


def oracle_hdiff_par(inp, coeff, out, dom, threads):
    """The oracle's hdiff, unchanged, on J-slabs of the domain in parallel (origin 2, 2, 0)."""
    import oracle
    I_, J_, K_ = dom

    def slab(j0, nj):
        o = (2, 2 + j0, 0)
        oracle.hdiff(inp, coeff, out, origin_in=o, origin_coeff=o, origin_out=o, domain=(I_, nj, K_))
    oracle_slabs(slab, J_, threads)
    return out


def oracle_vadv_par(fields, out, dom, threads):
    """The oracle's vadv, unchanged, on J-slabs of the domain in parallel (origin 1, 1, 0)."""
    import oracle
    I_, J_, K_ = dom

    def slab(j0, nj):
        oracle.vadv(*fields, out, origin=(1, 1 + j0, 0), domain=(I_, nj, K_))
    oracle_slabs(slab, J_, threads)
    return out


def oracle_step(f, jrows=None, threads=1, outs=None):
    """One oracle hdiff + vadv pass (optionally on the first `jrows` rows of J) on
    `threads` J-slabs in parallel; returns points."""
    Jr = J if jrows is None else jrows
    ho, vo = outs if outs is not None else (np.zeros_like(f["coeff"]), np.zeros_like(f["utens"]))
    oracle_hdiff_par(f["in"], f["coeff"], ho, (I, Jr, K), threads)
    oracle_vadv_par([f[n] for n in VADV_NAMES], vo, (I, Jr, K), threads)
    return I * Jr * K


def cpu_rate(f, threads, min_seconds):
    outs = (np.zeros_like(f["coeff"]), np.zeros_like(f["utens"]))
    oracle_step(f, threads=threads, outs=outs)  # warm-up (page faults, thread start)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle_step(f, threads=threads, outs=outs)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds and reps >= 2:
            break
    return POINTS * reps / el / 1e6, reps, el


def cpu_baseline(f, precision=None, prec_outs=None, min_seconds=10.0):
    """The oracle as it stands (C, binary64) on every host core this process may use, one
    thread per J-slab: full 256x256x80 hdiff+vadv steps for >= min_seconds (the line's
    value), the single-thread rate beside it, hdiff alone at 64x64x40 and one hdiff+vadv
    pass at 512x512x80.  The 512x512x80 runs (FP64 inputs, and the same draws rounded to
    FP32) also check the GPU outputs that the precision leg kept: each form's error is
    written into that block."""
    from paper_2311_08322_b300 import inputs
    cores = host_cores()
    v, reps, el = cpu_rate(f, cores, min_seconds)
    v1, reps1, el1 = cpu_rate(f, 1, min_seconds / 2)
    c1 = inputs.hdiff_small(0)
    c1_out = np.zeros_like(c1["coeff"])
    t0, n1 = time.perf_counter(), 0
    while time.perf_counter() - t0 < 1.0:
        oracle_hdiff_par(c1["in"], c1["coeff"], c1_out, (64, 64, 40), 1)
        n1 += 1
    c1_ms = (time.perf_counter() - t0) / n1 * 1e3
    out = {"value": round(v, 3), "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
           "sample": f"{reps} full hdiff+vadv steps at 256x256x80 FP64 ({el:.1f} s), the C oracle on {cores} "
                     f"threads, one J-slab each",
           "single_thread": {"value": round(v1, 3), "unit": "Mpoints/s", "cores": 1,
                             "sample": f"{reps1} full steps ({el1:.1f} s)"},
           "hdiff_64x64x40_ms": round(c1_ms, 3)}
    I3, J3, K3 = 512, 512, 80
    f3 = inputs.hdiff_vadv(I3, J3, K3, seed=0)
    for name, dt in (("fp64", np.float64), ("fp32", np.float32)):
        fin = {k: a.astype(dt).astype(np.float64) for k, a in f3.items()}
        t0 = time.perf_counter()
        ref_h = oracle_hdiff_par(fin["in"], fin["coeff"], np.zeros_like(fin["coeff"]), (I3, J3, K3), cores)
        ref_v = oracle_vadv_par([fin[n] for n in VADV_NAMES], np.zeros_like(fin["utens"]), (I3, J3, K3), cores)
        if name == "fp64":
            out["step_512x512x80_s"] = round(time.perf_counter() - t0, 3)
        if precision is not None and prec_outs is not None and name in prec_outs:
            errs = {}
            for key, got in prec_outs[name].items():
                ref = ref_h[:, 2:-2, 2:-2] if key == "hdiff" else ref_v[:, 1:-1, 1:-1]
                errs[key] = field_errors(got, ref)
            precision[name]["error_vs_fp64_oracle"] = errs
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2311_08322_b300 import inputs
    import oracle
    oracle.build()
    f = inputs.hdiff_vadv(I, J, K, seed=0)
    cores = host_cores()
    outs = (np.zeros_like(f["coeff"]), np.zeros_like(f["utens"]))
    # size each step so that warmup + steps finish in about two minutes
    oracle_step(f, jrows=min(J, 4 * cores), threads=cores, outs=outs)
    t0 = time.perf_counter()
    oracle_step(f, jrows=min(J, 4 * cores), threads=cores, outs=outs)
    tq = time.perf_counter() - t0
    per_step_budget = 120.0 / max(1, args.steps + args.warmup)
    jrows = int(max(1, min(J, min(J, 4 * cores) * per_step_budget / max(tq, 1e-6))))
    for _ in range(args.warmup):
        oracle_step(f, jrows, threads=cores, outs=outs)
    t0 = time.perf_counter()
    pts = 0
    for _ in range(args.steps):
        pts += oracle_step(f, jrows, threads=cores, outs=outs)
    el = time.perf_counter() - t0
    v = pts / el / 1e6
    line = {"metric": METRIC, "value": round(v, 3), "unit": "Mpoints/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_rows_j": jrows},
            "cpu_baseline": {"value": round(v, 3), "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: hdiff+vadv on 256x{jrows}x80 of the 256x256x80 fields, "
                                       f"{cores} threads (one J-slab each)"},
            "e2e": {"value": round(v, 3), "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gtb(args):
    import torch
    import torch.distributed as dist
    from paper_2311_08322_b300 import build, gtb, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    build.build()
    gtb.lib()

    f = inputs.hdiff_vadv(I, J, K, seed=rank)
    o2, o1 = (HDIFF_HALO, HDIFF_HALO, 0), (VADV_HALO, VADV_HALO, 0)
    sets = []
    for _ in range(args.sets):
        s = {"in": gtb.storage_from(f["in"], o2), "coeff": gtb.storage_from(f["coeff"], o2),
             "hout": gtb.storage_from(np.zeros_like(f["coeff"]), o2),
             "vout": gtb.storage_from(np.zeros_like(f["utens"]), o1)}
        for n in VADV_NAMES:
            s[n] = gtb.storage_from(f[n], o1)
        sets.append(s)
    stream = torch.cuda.current_stream()

    def step(s, ev=None):
        """Both stencils on their own fields: one co-scheduled launch (gtb_step)."""
        if ev is not None:
            ev[0].record(stream)
        gtb.step(s["in"], s["coeff"], s["hout"], *[s[n] for n in VADV_NAMES], s["vout"], stream=stream)
        if ev is not None:
            ev[1].record(stream)

    def separate(s, ev):
        """The same step as two launches, gtb_hdiff then gtb_vadv (per-kernel context)."""
        ev[0].record(stream)
        gtb.hdiff(s["in"], s["coeff"], s["hout"], stream=stream)
        ev[1].record(stream)
        gtb.vadv(*[s[n] for n in VADV_NAMES], s["vout"], stream=stream)
        ev[2].record(stream)

    # the FP64 rate probe (outside the timed region, on every rank's GPU) and the clock
    # sampler's start come before the warm-up steps, so that the timed steps follow the
    # warm-up with no idle gap in between
    fma_gops = fp64_fma_rate()
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = str(dev)
    clocks = ClockSampler(uuid)
    clocks.start()
    for w in range(args.warmup - 1):
        step(sets[w % len(sets)])
    gtb.device_status()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # the last of the W warm-up steps goes after the barrier: the start event then fires
    # as it completes, with the first timed step already queued behind it, so the timed
    # region holds the K steps' device time and not the host's first launch latency
    if args.warmup > 0:
        step(sets[(args.warmup - 1) % len(sets)])
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for q in range(args.steps):  # the input sets rotate on from the warm-up's
        step(sets[(args.warmup + q) % len(sets)])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    gtb.device_status()
    el_ms = t_start.elapsed_time(t_end)
    # the step kernel's average launch duration for its roofline: the timed region holds
    # exactly one launch of it per step, back to back on this stream.  The same steps with
    # an event around each launch are a cross-check only (host gaps land inside those
    # intervals whenever the host falls behind the GPU); then the step as two separate
    # kernels with an event around each
    st_ms = el_ms / args.steps
    nser = 500  # per-kernel figures over 500 launches whatever K is (about 0.2 s)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(nser)]
    torch.cuda.synchronize()
    # each evented loop starts behind one untimed call, so that its first interval holds
    # no host launch latency
    step(sets[-1])
    for q in range(nser):
        step(sets[q % len(sets)], evs[q])
    torch.cuda.synchronize()
    st_ev_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nser)]
    gtb.hdiff(sets[-1]["in"], sets[-1]["coeff"], sets[-1]["hout"], stream=stream)
    gtb.vadv(*[sets[-1][n] for n in VADV_NAMES], sets[-1]["vout"], stream=stream)
    for q in range(nser):
        separate(sets[q % len(sets)], evs[q])
    torch.cuda.synchronize()
    gtb.device_status()
    h_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    v_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    sep_ms = float(np.mean([e[0].elapsed_time(e[2]) for e in evs]))
    chain = fused_chain_compare(gtb, f, sets) if rank == 0 and not args.no_fused else None
    calls = call_overhead() if rank == 0 and not args.no_fused else None
    adj = adjoint_ratio(gtb, f, sets) if rank == 0 and not args.no_adjoint else None
    adj32 = adjoint_ratio(gtb, f, sets, dtype=np.float32) if rank == 0 and not args.no_adjoint else None
    el_ms = max_over_ranks(el_ms, dist if world > 1 else None, "cuda")
    value = whole_job_mpoints(world, POINTS, args.steps, el_ms)

    # e2e through the C ABI: every step copies its inputs from pinned host memory to the
    # device, runs the step and copies both outputs back.  Steps are pipelined over two
    # device buffer sets: copy-in, compute and copy-out run on three streams, so step q's
    # copy-in overlaps step q-1's compute and step q-2's copy-out.
    host = {n: torch.from_numpy(f[n]).pin_memory() for n in ("in", "coeff", *VADV_NAMES)}
    hbuf = [(torch.empty(sets[0]["hout"].data.shape, dtype=torch.float64).pin_memory(),
             torch.empty(sets[0]["vout"].data.shape, dtype=torch.float64).pin_memory()) for _ in range(2)]
    dbuf = list(sets[:2])
    if len(dbuf) < 2:
        extra = {n: gtb.storage_from(f[n], o2 if n in ("in", "coeff") else o1) for n in ("in", "coeff", *VADV_NAMES)}
        extra["hout"] = gtb.storage_from(np.zeros_like(f["coeff"]), o2)
        extra["vout"] = gtb.storage_from(np.zeros_like(f["utens"]), o1)
        dbuf.append(extra)
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = hbuf[0][0].numel() * 8 + hbuf[0][1].numel() * 8
    s_in = [torch.cuda.Stream() for _ in range(args.e2e_in_streams)]
    s_out = torch.cuda.Stream()
    free = [torch.cuda.Event(), torch.cuda.Event()]  # buffer set b no longer read by a copy-out
    names_in = list(host)

    def e2e_run(n):
        for q in range(n):
            b = q % 2
            d = dbuf[b]
            for si, st_ in enumerate(s_in):  # the inputs split over the copy-in streams
                st_.wait_event(free[b])
                with torch.cuda.stream(st_):
                    for nm in names_in[si::len(s_in)]:
                        d[nm].data.copy_(host[nm], non_blocking=True)
                e_in = torch.cuda.Event()
                e_in.record(st_)
                stream.wait_event(e_in)
            step(d)
            e_c = torch.cuda.Event()
            e_c.record(stream)
            s_out.wait_event(e_c)
            with torch.cuda.stream(s_out):
                hbuf[b][0].copy_(d["hout"].data, non_blocking=True)
                hbuf[b][1].copy_(d["vout"].data, non_blocking=True)
            free[b].record(s_out)
        stream.wait_stream(s_out)

    for b in range(2):
        free[b].record(stream)
    e2e_run(2)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st_ in s_in:
        st_.wait_event(e0)
    e2e_run(args.e2e_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, dist if world > 1 else None, "cuda")
    e2e_value = whole_job_mpoints(world, POINTS, args.e2e_steps, e2e_ms)

    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs, torch copy)" if "hbm_gbs" in peaks else "fallback 6.4 TB/s"
    kern = {}
    hb, vb = hdiff_bytes(I, J, K, 8), vadv_bytes(I, J, K, 8)
    for name, ms, nbytes in (("step", st_ms, hb + vb), ("hdiff", h_ms, hb), ("vadv", v_ms, vb)):
        gbs = nbytes / (ms / 1e3) / 1e9
        kern[name] = {"ms": round(ms, 4), "mpoints_s": round(POINTS / (ms / 1e3) / 1e6, 1),
                      "algorithmic_bytes": nbytes, "hbm_gbs": round(gbs, 1),
                      "frac_of_measured_hbm": round(gbs / hbm, 4), "frac_of_8tbs": round(gbs / 8000.0, 4)}
    kern["step"]["kernel"] = "hdiff_vadv_pair_kernel (hdiff and vadv co-scheduled in one launch)"
    kern["step"]["event_bracketed_ms"] = round(st_ev_ms, 4)
    kern["separate_step_ms"] = round(sep_ms, 4)
    kd = kern["step"]  # the step is one launch: the dominant (only) kernel of the timed region
    traffic = profile_traffic("hdiff_vadv_pair_kernel")
    roof = {"bound": "hbm", "kernel": "hdiff_vadv_pair_kernel", "achieved": kd["hbm_gbs"], "peak": hbm,
            "unit": "GB/s", "frac": kd["frac_of_measured_hbm"], "traffic": traffic, "peak_source": hbm_src,
            "algorithmic_bytes_per_launch": hb + vb,
            "note": "HBM fraction of the step kernel; the binary64 column solve binds it on the FP64 pipe (fp64 block)"}
    ops = profile_field("hdiff_vadv_pair_kernel", r"^fp64 ops per domain point .* total ([0-9.]+)")
    pipe = profile_field("hdiff_vadv_pair_kernel", r"^sm__pipe_fp64_cycles_active\S* = ([0-9.]+)")
    fp64 = {"kernel": "hdiff_vadv_pair_kernel", "executed_ops_per_point": ops,
            "ops_source": "ncu smsp__sass_thread_inst_executed_op_{dadd,dfma,dmul}_pred_on of the committed summary "
                          "(null when the kernel changed since it was captured)",
            "peak_gops": None if fma_gops is None else round(fma_gops, 1),
            "peak_source": "gtb_probe_fp64_fma in this run: independent binary64 FMA chains, 8 CTAs x 256 threads "
                           "per SM, CUDA events, best of 5 (DADD and DMUL issue on the same pipe at the same rate)",
            "pipe_active_pct_ncu": pipe}
    if ops is not None and fma_gops:
        fp64["achieved_gops"] = round(ops * POINTS / (st_ms / 1e3) / 1e9, 1)
        fp64["frac"] = round(fp64["achieved_gops"] / fma_gops, 4)

    line = {"metric": METRIC, "value": round(value, 1), "unit": "Mpoints/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "I": I, "J": J, "K": K, "parallelism": f"replicas{world}",
                       "l2": f"{args.sets} rotating input sets of "
                             f"{(hdiff_bytes(I, J, K, 8) + vadv_bytes(I, J, K, 8)) / 1e6:.0f} MB each (> 126 MB L2)"},
            "kernels": kern, "roofline": roof, "fp64": fp64, "clocks": clk, "gpu_launches": args.steps,
            "fused_chain": chain, "call_overhead": calls,
            "adjoint_forward_ratio": None if adj is None else adj["ratio"], "adjoint": adj, "adjoint_fp32": adj32,
            "e2e": {"value": round(e2e_value, 1), "unit": "Mpoints/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps}}
    prec_outs = None
    if rank == 0 and not args.no_precision:
        line["precision"], prec_outs = precision_compare(hbm)
    if rank == 0 and not args.no_batched:
        line["batched"] = batched_compare(hbm)
    if rank == 0 and not args.no_adjoint:
        line["literal_chain"] = literal_chain()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        line["cpu_baseline"] = cpu_baseline(f, line.get("precision"), prec_outs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def call_overhead(reps=2000, host_reps=64):
    """The paper's timing split (Python call vs the compiled call alone) for one step on
    the small 64x64x40 FP64 workload, where launch and call costs show: device time per
    step (CUDA events), host time per call of the C ABI with prepared descriptors, and
    host time per call of the Python binding (descriptor marshalling included)."""
    import ctypes
    import torch
    from paper_2311_08322_b300 import gtb, inputs
    Is, Js, Ks = 64, 64, 40
    f = inputs.hdiff_vadv(Is, Js, Ks, seed=0)
    o2, o1 = (HDIFF_HALO, HDIFF_HALO, 0), (VADV_HALO, VADV_HALO, 0)
    s = {"in": gtb.storage_from(f["in"], o2), "coeff": gtb.storage_from(f["coeff"], o2),
         "hout": gtb.storage_from(np.zeros_like(f["coeff"]), o2),
         "vout": gtb.storage_from(np.zeros_like(f["utens"]), o1)}
    for n in VADV_NAMES:
        s[n] = gtb.storage_from(f[n], o1)
    args = [s["in"], s["coeff"], s["hout"], *[s[n] for n in VADV_NAMES], s["vout"]]
    stream = torch.cuda.current_stream()
    dom = (Is, Js, Ks)
    ws = gtb.workspace(gtb.vadv_workspace_bytes(torch.float64, "native", dom))
    fields = [gtb._as_field(x) for x in args]
    refs = [ctypes.byref(x) for x in fields]
    c_dom = (ctypes.c_int64 * 3)(*dom)
    c_ws, c_st, lib = ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(stream.cuda_stream), gtb.lib()
    nbytes = ws.numel()

    def c_call():
        lib.gtb_step(*refs, 0.15, 0.0, 0, 0, c_dom, c_ws, nbytes, c_st)

    def py_call():
        gtb.step(*args, domain=dom, stream=stream)

    # the timed bursts discard the return code: check once that the call enqueues work
    rc = lib.gtb_step(*refs, 0.15, 0.0, 0, 0, c_dom, c_ws, nbytes, c_st)
    if rc != 0:
        raise RuntimeError(f"gtb_step failed in call_overhead: {rc} {lib.gtb_last_error().decode()}")
    gtb.device_status()
    out = {"workload": "one hdiff+vadv step (gtb_step) at 64x64x40 FP64"}
    # host time per call over bursts short enough that the launch queue never fills (a
    # full queue makes the host wait for the device inside the timed region: bursts of
    # 200 calls of this 45 us kernel did), median of several bursts
    for name, fn in (("c_abi_us_per_call", c_call), ("python_us_per_call", py_call)):
        for _ in range(50):
            fn()
        torch.cuda.synchronize()
        per = []
        for _ in range(9):
            t0 = time.perf_counter()
            for _ in range(host_reps):
                fn()
            per.append((time.perf_counter() - t0) / host_reps * 1e6)
            torch.cuda.synchronize()
        out[name] = round(statistics.median(per), 2)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        c_call()
    b.record(stream)
    torch.cuda.synchronize()
    out["device_us_per_step"] = round(a.elapsed_time(b) / reps * 1e3, 2)
    # hdiff alone at 64x64x40 FP64 (its launch-bound smallest configuration)
    for _ in range(20):
        gtb.hdiff(s["in"], s["coeff"], s["hout"], stream=stream)
    a.record(stream)
    for _ in range(reps):
        gtb.hdiff(s["in"], s["coeff"], s["hout"], stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    out["hdiff_64x64x40_fp64_us"] = round(a.elapsed_time(b) / reps * 1e3, 2)
    gtb.device_status()
    return out


def fused_chain_compare(gtb, f, sets, reps=50):
    """The chained step h = hdiff(in, coeff), out = vadv(h, wcon, h, utens, utens_stage) at
    256x256x80 FP64: gtb_hdiff + gtb_vadv (h through HBM) vs gtb_hdiff_vadv (one kernel)."""
    import torch
    dom = (I, J, K)
    hs = [gtb.storage_from(np.zeros_like(f["utens"]), (VADV_HALO, VADV_HALO, 0)) for _ in sets]

    def separate(q):
        s, h = sets[q % len(sets)], hs[q % len(sets)]
        gtb.hdiff(s["in"], s["coeff"], h, domain=dom)
        gtb.vadv(h, s["wcon"], h, s["utens"], s["utens_stage"], s["vout"], domain=dom)

    def fused(q):
        s = sets[q % len(sets)]
        gtb.hdiff_vadv(s["in"], s["coeff"], s["wcon"], s["utens"], s["utens_stage"], s["vout"], domain=dom)

    def timed(fn):
        for q in range(5):
            fn(q)
        torch.cuda.synchronize()
        fn(-1)  # untimed: the start event then fires behind it, with the first timed call queued
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for q in range(reps):
            fn(q)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    sep, fus = timed(separate), timed(fused)
    gtb.device_status()
    return {"workload": "chained step 256x256x80 FP64: h = hdiff(in, coeff); out = vadv(h, wcon, h, utens, "
                        "utens_stage)", "separate_ms": round(sep, 4), "fused_ms": round(fus, 4),
            "speedup": round(sep / fus, 3), "fused_mpoints_s": round(POINTS / (fus / 1e3) / 1e6, 1)}


def adjoint_ratio(gtb, f, sets, reps=50, dtype=np.float64):
    """Time of one chained step's backward over its forward at 256x256x80 (C ABI,
    preallocated storages), as the differentiable chain runs them: forward = periodic halo
    refresh + the chained hdiff -> vadv call keeping the column factors (one fused kernel for
    FP64; hdiff then vadv, h in the workspace, for FP32), backward = vadv_adj
    on those factors (merged u_stage/u_pos cotangent) + hdiff_adj (with coeff_bar) + halo
    fold.  Forward and backward alternate (each backward consumes its forward's factors);
    events around each side give both times.  FP64 storage, or FP32 storage with
    double-float columns (its own storages, rounded from the same draws)."""
    import torch
    o2, o1 = (HDIFF_HALO, HDIFF_HALO, 0), (VADV_HALO, VADV_HALO, 0)
    dom = (I, J, K)
    f64 = dtype == np.float64
    prec = "native" if f64 else "df"
    tdt = torch.float64 if f64 else torch.float32
    nfac = gtb.hdiff_vadv_workspace_bytes(tdt, prec, dom, save_factors=True)
    bufs = []
    for s in (sets if f64 else range(2)):
        if not f64:  # binary32 storages of the same draws
            s = {n: gtb.storage_from(f[n].astype(np.float32), o2 if n in ("in", "coeff") else o1)
                 for n in ("in", "coeff", "wcon", "utens", "utens_stage")}
        bufs.append({"fs": s["in"], "cs": s["coeff"], "y": gtb.storage_from(np.zeros((K, J, I), dtype), (0, 0, 0)),
                     "wcon": s["wcon"], "ut": s["utens"], "uts": s["utens_stage"],
                     "yb": gtb.storage_from(f["u_pos"][:, 1:-1, 1:-1].astype(dtype), (0, 0, 0)),
                     "hb": gtb.storage_from(np.zeros((K, J, I), dtype), (0, 0, 0)),
                     "ib": gtb.storage_from(np.zeros(f["in"].shape, dtype), o2),
                     "cb": gtb.storage_from(np.zeros(f["coeff"].shape, dtype), o2),
                     "F": torch.empty(nfac, dtype=torch.uint8, device="cuda")})
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def fwd(b):
        gtb.halo_periodic(b["fs"], 2, 2, domain=dom)
        gtb.hdiff_vadv(b["fs"], b["cs"], b["wcon"], b["ut"], b["uts"], b["y"], prec=prec, domain=dom,
                       workspace=b["F"], save_factors=True)

    def bwd(b, e):
        gtb.vadv_adj(b["wcon"], b["yb"], b["hb"], b["hb"], prec=prec, domain=dom, workspace=b["F"], factors=True)
        e[2].record(stream)
        gtb.hdiff_adj(b["fs"], b["cs"], b["hb"], b["ib"], b["cb"], accumulate=True, domain=dom)
        e[3].record(stream)
        gtb.halo_periodic_adj(b["ib"], 2, 2, domain=dom)

    es = [[ev() for _ in range(5)] for _ in range(reps + 5)]
    for q in range(reps + 5):  # the first 5 pairs warm up
        b, e = bufs[q % len(bufs)], es[q]
        e[0].record(stream)
        fwd(b)
        e[1].record(stream)
        bwd(b, e)
        e[4].record(stream)
    torch.cuda.synchronize()
    gtb.device_status()
    es = es[5:]
    mean = lambda a, b: float(np.mean([e[a].elapsed_time(e[b]) for e in es]))
    f_ms, b_ms = mean(0, 1), mean(1, 4)
    out = {"ratio": round(b_ms / f_ms, 3), "forward_ms": round(f_ms, 4), "backward_ms": round(b_ms, 4),
           "vadv_adj_ms": round(mean(1, 2), 4), "hdiff_adj_ms": round(mean(2, 3), 4),
           "halo_adj_ms": round(mean(3, 4), 4),
           "workspace_mb_per_step": round(nfac / 1e6, 1),
           "workload": f"one chained step at 256x256x80 {'FP64' if f64 else 'FP32 storage, double-float columns'} "
                       "(halo refresh + hdiff -> vadv keeping the column factors vs the adjoints)"}
    del bufs
    torch.cuda.empty_cache()
    return out


def literal_chain(steps=10):
    """The 10-step chain at 256x256x80 FP64 exactly as drawn (wcon ~ U(-0.5, 0.5), seed 0):
    field <- vadv(hdiff(field)) with the periodic 2-point halo, forward only.  Its
    ill-conditioned columns amplify the field every step; the line records max |field|
    after each step (the gradient checks draw wcon from U(-0.3, 0.3) instead)."""
    import torch
    from paper_2311_08322_b300.autograd import chain, chain_inputs
    field, coeff, fixed, _ = chain_inputs(I, J, K, seed=0, dtype=torch.float64, wcon_amp=0.5)
    fixed.save_factors = False
    growth = []
    with torch.no_grad():
        x = field
        for _ in range(steps):
            x = chain(x, coeff, fixed, 1)
            growth.append(float(x.abs().max()))
    from paper_2311_08322_b300 import gtb
    gtb.device_status()
    return {"workload": "10-step chain field <- vadv(hdiff(field)) at 256x256x80 FP64, wcon ~ U(-0.5, 0.5) (seed 0), "
                        "periodic halo", "max_abs_per_step": [float(f"{g:.4e}") for g in growth],
            "initial_max_abs": round(float(field.abs().max()), 4)}


def batched_compare(hbm, reps=20):
    """The batched form: a 48-member ensemble of uneven domains (I=J in
    {48..384}, K in {40, 60, 80, 137}, seed-fixed), FP32 storage with
    double-float vadv, each member hdiff then vadv (h fed to vadv as u_stage and
    u_pos).  Graph replay of the autotuned plan vs a loop of the 96
    single-domain launches, both timed with CUDA events after warm-up."""
    import torch
    from paper_2311_08322_b300 import autotune, gtb, inputs
    shapes = inputs.ensemble_shapes(48, 0)
    members = []
    for q, (I_, J_, K_) in enumerate(shapes):
        f = inputs.hdiff_vadv(I_, J_, K_, seed=1 + q)
        f = {k: v.astype(np.float32) for k, v in f.items()}
        members.append(gtb.member_storages(f, I_, J_, K_))
        del f
    cfg, log = autotune.tune(members, prec="df", reps=3)
    plan = gtb.BatchPlan(members, prec="df", config=cfg)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        fn()  # untimed: the start event then fires behind it, with the first timed call queued
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    g_ms = timed(lambda: plan.run(stream))
    l_ms = timed(lambda: [gtb.run_member_single(m, prec="df", stream=stream) for m in members])
    gtb.device_status()
    info = plan.info()
    pts = info["points"]
    plan.close()
    nbytes = batched_bytes(shapes, 4)
    gbs = nbytes / (g_ms / 1e3) / 1e9
    return {"workload": "48-member ensemble, I=J in {48,96,128,192,256,384}, K in {40,60,80,137}, FP32 storage, "
                        "double-float vadv", "points": pts, "graph_ms": round(g_ms, 4), "loop_ms": round(l_ms, 4),
            "speedup_vs_loop": round(l_ms / g_ms, 3), "mpoints_s": round(pts / (g_ms / 1e3) / 1e6, 1),
            "algorithmic_bytes": nbytes, "hbm_gbs": round(gbs, 1), "frac": round(gbs / hbm, 4),
            "config": cfg, "autotune_cached": log.get("cached"), "launches_graph": 2,
            "launches_loop": 2 * len(members)}


def field_errors(got, ref):
    """Max-norm relative error and the worst column's relative error of one output field."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    d = np.abs(got - ref)
    den = np.max(np.abs(ref))
    col = np.max(d, axis=0) / np.maximum(np.max(np.abs(ref), axis=0), 1e-300)
    return {"max_norm": float(f"{float(d.max() / (den if den > 0 else 1.0)):.3e}"),
            "worst_column": float(f"{float(col.max()):.3e}")}


def precision_compare(hbm, reps=20):
    """The precision form at 512x512x80 (same generators): FP32 storage with binary32
    hdiff and vadv in its three column-arithmetic forms (binary32, binary64 on the
    FP64 pipe, double-float on the FP32 pipe), beside the FP64 path at the same size
    on the same GPU.  Two input sets alternate (each larger than L2).  After the timing,
    every form's outputs are kept on the host; the cpu_baseline leg, which runs the FP64
    oracle on this workload (on the inputs the GPU saw: FP32-rounded for the FP32 forms),
    adds each form's error (max-norm and worst column per output field)."""
    import torch
    from paper_2311_08322_b300 import gtb, inputs
    I3, J3, K3 = 512, 512, 80
    f = inputs.hdiff_vadv(I3, J3, K3, seed=0)
    o2, o1 = (2, 2, 0), (1, 1, 0)

    def make(dt):
        sets = []
        for _ in range(2):
            st = {"in": gtb.storage_from(f["in"].astype(dt), o2), "coeff": gtb.storage_from(f["coeff"].astype(dt), o2),
                  "hout": gtb.storage_from(np.zeros(f["coeff"].shape, dt), o2),
                  "vout": gtb.storage_from(np.zeros(f["utens"].shape, dt), o1)}
            for n in VADV_NAMES:
                st[n] = gtb.storage_from(f[n].astype(dt), o1)
            sets.append(st)
        return sets

    stream = torch.cuda.current_stream()

    def timed(fn):
        for q in range(4):
            fn(q)
        torch.cuda.synchronize()
        fn(-1)  # untimed: the start event then fires behind it, with the first timed call queued
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for q in range(reps):
            fn(q)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    pts = I3 * J3 * K3
    res = {"workload": "hdiff + vadv at 512x512x80 (same generators as the FP64 path)"}
    outs = {}
    for name, dt in (("fp64", np.float64), ("fp32", np.float32)):
        sets = make(dt)
        es = 8 if dt == np.float64 else 4
        r = {"hdiff_ms": timed(lambda q: gtb.hdiff(sets[q % 2]["in"], sets[q % 2]["coeff"], sets[q % 2]["hout"]))}
        # df48: double-float with the column state in 48 bits (GTB_STATE48)
        precs = ("native",) if dt == np.float64 else ("native", "f64", "df", "df48")
        kw = lambda pr: {"prec": pr[:2] if pr == "df48" else pr, "state48": pr == "df48"}
        for pr in precs:
            r[f"vadv_{pr}_ms"] = timed(lambda q: gtb.vadv(*[sets[q % 2][n] for n in VADV_NAMES], sets[q % 2]["vout"],
                                                          **kw(pr)))
        r["hdiff_gbs"] = round(hdiff_bytes(I3, J3, K3, es) / (r["hdiff_ms"] / 1e3) / 1e9, 1)
        for pr in precs:
            r[f"vadv_{pr}_gbs"] = round(vadv_bytes(I3, J3, K3, es) / (r[f"vadv_{pr}_ms"] / 1e3) / 1e9, 1)
        r["hdiff_frac_of_measured_hbm"] = round(r["hdiff_gbs"] / hbm, 4)
        for pr in precs:
            r[f"vadv_{pr}_frac_of_measured_hbm"] = round(r[f"vadv_{pr}_gbs"] / hbm, 4)
        best_v = min(r[f"vadv_{pr}_ms"] for pr in precs if pr != "native" or dt == np.float64)
        r["step_mpoints_s"] = round(pts / ((r["hdiff_ms"] + best_v) / 1e3) / 1e6, 1)
        res[name] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
        # the outputs of one more call of every form, kept on the host: the cpu_baseline leg
        # checks them against the oracle (its 512x512x80 runs) after all GPU timing
        st = sets[0]
        gtb.hdiff(st["in"], st["coeff"], st["hout"])
        kept = {"hdiff": st["hout"].numpy()[:, 2:-2, 2:-2]}
        for pr in precs:
            gtb.vadv(*[st[n] for n in VADV_NAMES], st["vout"], **kw(pr))
            kept[f"vadv_{pr}"] = st["vout"].numpy()[:, 1:-1, 1:-1]
        gtb.device_status()
        outs[name] = kept
        del sets
        torch.cuda.empty_cache()
    gtb.device_status()
    res["note"] = ("fp32 step uses the fastest vadv form that meets the 1e-5 bound (f64, df or df48: df with its "
                   "column state in 48 bits); all-binary32 vadv does not meet it on ill-conditioned columns")
    return res, outs


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("gtb", "reference"), default="gtb")
    ap.add_argument("--sets", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--e2e-in-streams", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gtb(args)


if __name__ == "__main__":
    sys.exit(main())
