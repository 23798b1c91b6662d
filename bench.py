#!/usr/bin/env python
"""xGETT benchmark: one JSON line on rank 0.

Default workload (N=1): the coupled-cluster-like contraction
C[a,b,i,j] += sum_{c,d} A[a,b,c,d] B[c,d,i,j], a=b=c=d=128, i=j=32, FP64,
N(0,1) inputs, column-major -- 0.55 TFLOP per call.  A step is one dgett call
(validate, plan, select, kernel, epilogue) on inputs resident in HBM; A
(2.1 GB) is larger than L2, so no flush is needed between steps.

Extra measured forms (not part of `value`): the same contraction with output
permutation (i,a,j,b) and row-major A, the streaming outer product, the small
32x24x16x20 DGETT, the split-precision forms (modular DGETT on bf16 tensor
cores (every output compared with the native FP64 call), every precision form
on log-uniform data (against native FP64 on the same inputs), complex
split ZGETT), the inner product (REDUCE) and matrix-vector (SKINNY) kernels
against their HBM and FP64-FMA floors, and the batched launch of
4096 contractions (heuristic, tuned and learned configurations).

`e2e`: the same call with pinned host buffers; each step's uploads of A, B, C
and the download of C are inside the timed region (pipelined over two device
buffer sets).

--impl reference times the CPU oracle (the plain Alg. 1 loop nest) on the
host cores on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank runs its own copy of the workload (weak
scaling, no data-path collective); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "xGETT TFLOP/s & % roofline: plain FP64 vs split-precision at ≤1e-13 err; batch ops/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gett", choices=["gett", "reference"])
    ap.add_argument("--workload", default="cc", choices=["cc", "cc_perm_transA", "stream", "small"])
    ap.add_argument("--algo", default="native")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-tune-db", action="store_true", help="do not load the shipped tuning database")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, backend):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload(name):
    from paper_2410_06770_gb300 import synth
    if name == "cc":
        return synth.cfg_cc("plain"), "cc_plain: C[a,b,i,j]+=A[a,b,c,d]B[c,d,i,j], a..d=128, i,j=32, col-major"
    if name == "cc_perm_transA":
        return synth.cfg_cc("perm_transA"), "cc_perm_transA: output (i,a,j,b), row-major A, a..d=128, i,j=32"
    if name == "stream":
        return synth.cfg_stream(c_host=False), "stream_outer: A(256,256,64) x B(64,8), CONTS=0 -> C 17.2 GB"
    if name == "small":
        return synth.cfg_small_dgett(), "dgett_small: A(32,24,16,20) stride-2 mode a, B(20,28,24,12), out (e,a,f,c)"
    raise ValueError(name)


def flops_of(p) -> float:
    s = p.sig
    K = int(np.prod([s.exta[m] for m in s.conta], dtype=np.int64)) if s.conta else 1
    M = int(np.prod(s.extc(), dtype=np.int64)) if s.rank_c else 1
    return 2.0 * M * K


def bytes_of(p) -> float:
    """Algorithmic HBM bytes: read A and B once, read and write C once."""
    return 8.0 * (p.la.numel + p.lb.numel + 2 * p.lc.numel)


# ---------------------------------------------------------------------------
# the CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(p, seconds: float, want_values=False):
    """Time the oracle on a sample of output elements of `p`: the sub-problem
    that keeps A whole and restricts B (hence C) to its first j columns of the
    last B free mode (or, for a full outer product, the first columns).
    Returns (tflops, cores, description, seconds); with want_values also the
    sampled outputs' buffer positions in C (the sub-problem shares C's
    layout) and the oracle's values there, summed from zero."""
    import oracle
    cores = os.cpu_count() or 1
    s = p.sig
    rb = len(s.extb)
    # last free mode of B
    free_b = [m for m in range(rb) if m not in s.contb]
    lastb = free_b[-1]

    def sub(ncols):
        extb = list(s.extb)
        extb[lastb] = ncols
        # output extents follow
        fps = s.free_modes()
        extc = list(s.extc())
        for pidx, (t, m) in enumerate(fps):
            if t == 1 and m == lastb:
                extc[s.perm[pidx]] = ncols
        n = int(np.prod(extc, dtype=np.int64))
        reach = p.lc.off + sum((e - 1) * i for e, i in zip(extc, p.lc.inc) if e > 0 and i > 0)
        C = np.zeros(max(1, reach + 1))
        t0 = time.perf_counter()
        rc = oracle.gett_raw("f64", len(s.exta), s.exta, p.la.inc, p.A, p.la.off, rb, extb, p.lb.inc,
                             p.B, p.lb.off, s.conts, s.conta, s.contb, s.perm, p.lc.inc, C, p.lc.off,
                             nthreads=cores)
        dt = time.perf_counter() - t0
        assert rc == 0
        K = int(np.prod([s.exta[m] for m in s.conta], dtype=np.int64)) if s.conta else 1
        sub.last = (extc, C)
        return dt, 2.0 * n * K, n

    # calibrate on one column (bounded further by shrinking A's sample if needed)
    dt1, f1, n1 = sub(1)
    ncols = max(1, min(s.extb[lastb], int(seconds / max(dt1, 1e-6))))
    if ncols > 1:
        dt, f, n = sub(ncols)
    else:
        dt, f, n = dt1, f1, n1
    desc = (f"{n} of {int(np.prod(s.extc(), dtype=np.int64))} output elements "
            f"(first {ncols} of {s.extb[lastb]} values of B's last free mode), full sums, "
            f"{f / 1e9:.1f} GFLOP in {dt:.1f} s")
    if not want_values:
        return f / dt / 1e12, cores, desc, dt
    from paper_2410_06770_gb300 import synth
    extc, C = sub.last
    pos = synth._positions_f(extc, p.lc.inc, p.lc.off)
    return f / dt / 1e12, cores, desc, dt, pos, C[pos]


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f)
    except Exception:
        return {}


def traffic_entry(kernel_key: str):
    """Per-launch DRAM bytes from a committed ncu summary, if the kernel's
    source is unchanged since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            entries = json.load(f)
    except Exception:
        return None
    e = entries.get(kernel_key)
    if not e:
        return None
    h = hashlib.sha256()
    try:
        for src in e["sources"]:
            h.update(open(os.path.join(ROOT, src), "rb").read())
    except Exception:
        return None
    if h.hexdigest()[:16] != e.get("source_sha"):
        return None
    return e


def gpu_arm(args, dist: Dist):
    import torch

    from paper_2410_06770_gb300 import build, gett, synth

    torch.cuda.set_device(dist.local)
    build.build()
    L = gett.lib()
    dev = torch.cuda.current_device()

    # measured pipe peaks (our microbenchmarks) for the FP64 roofline
    from paper_2410_06770_gb300 import peaks as peaks_mod
    pk = peaks_mod.measure(copy_bytes=1 << 30)

    # the tuned step of the configuration choice: the shipped tuning
    # database (single-call entries of the bench workloads, measured by
    # `python -m paper_2410_06770_gb300.tune --single`)
    if not args.no_tune_db and os.path.exists(TUNE_DB):
        gett.tune_db_load(TUNE_DB)

    p, wdesc = workload(args.workload)
    flops = flops_of(p)
    stream = torch.cuda.current_stream()
    dA = torch.from_numpy(p.A).cuda()
    dB = torch.from_numpy(p.B).cuda()
    dC = torch.from_numpy(p.C).cuda()
    a = p.args()
    opts = gett.options(algo=args.algo)

    def call():
        return gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB,
                          a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC,
                          a_off=p.la.off, b_off=p.lb.off, c_off=p.lc.off, mode="async",
                          stream=stream.cuda_stream)

    # report of what runs (a synchronous _ex call on a scratch copy of C)
    dC2 = dC.clone()
    _, rep = gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB,
                        a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC2,
                        a_off=p.la.off, b_off=p.lb.off, c_off=p.lc.off, mode="ex", opts=opts,
                        stream=stream.cuda_stream)
    torch.cuda.synchronize()
    del dC2

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        ev[i][0].record(stream)
        call()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    per_call = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    ms_step = dist.max(total_ms / args.steps)
    value = flops * dist.world / (ms_step * 1e-3) / 1e12

    launches_per_call = {"dense": 4 + (1 if rep["split_k"] > 1 else 0), "outer": 1, "reduce": 2}.get(
        rep["family_name"], 1)

    # roofline of the dominant kernel
    kernel_ms = statistics.mean(per_call)
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    fam = rep["family_name"]
    if fam == "dense":
        peak = pk["dfma_tflops"]
        tiles = {0: "128,128,8,8,8", 1: "64,64,8,4,4", 2: "32,32,16,2,2"}
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_source": "measured DFMA microbenchmark (FP64 FMA pipe)",
                "kernel": f"dense_kernel<double,{tiles.get(rep['config'], '?')}>"}
    else:
        mp = measured_peaks()
        bw = mp.get("hbm_gbs", 6800.0)
        ach = bytes_of(p) / (kernel_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": bw, "unit": "GB/s", "frac": ach / bw,
                "peak_source": "MEASURED_PEAKS hbm_gbs (of measured)" if mp else "fallback 6.8 TB/s",
                "kernel": fam}
    te = traffic_entry(roof["kernel"])
    roof["traffic"] = te["bytes_per_launch"] if te else None

    result = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1), numpy default_rng seeds 2/3)",
        "config": {"workload": wdesc, "M": rep["M"], "N": rep["N"], "K": rep["K"],
                   "flops_per_step": flops, "algo": args.algo, "family": fam,
                   "tile_config": rep["config"], "split_k": rep["split_k"],
                   "selector": {0: "heuristic", 1: "tuning database", 2: "learned", 3: "forced"}.get(rep["selector"]),
                   "l2": "inputs larger than L2 (A is 2.1 GB), no flush"},
        "roofline": roof,
        "gpu_launches": launches_per_call * args.steps,
        "clocks": clocks,
        "peaks_measured": pk,
    }

    if not args.no_e2e:
        result["e2e"] = e2e_measure(p, flops, call_host=None, dA=dA, dB=dB, dC=dC, a=a, stream=stream,
                                    steps=args.steps, dev=dev)
    held = {}
    if not args.no_forms and dist.world == 1:
        del dA, dB, dC
        torch.cuda.empty_cache()
        result["forms"] = measure_forms(args.workload)
        result["forms"].update(measure_split_forms(held))
        result["forms"].update(measure_streaming_forms(pk.get("dfma_tflops")))
        result["forms"]["batched"] = measure_batched(ffma_tflops=pk.get("ffma_tflops"))
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu:
        cpu, split = cpu_baseline_leg(p, args.cpu_seconds, held, value)
        result["cpu_baseline"] = cpu
        if split:
            # last keys of the line: the driver keeps the line's tail
            bt = result.get("forms", {}).get("batched")
            if bt:
                result["batched"] = {k: _r(bt[k]["ms"]) for k in bt if k.startswith("batched_") or k == "per_call"}
                result["batched"]["contractions_per_s_learned"] = _r(bt.get("batched_learned", {}).get(
                    "contractions_per_s", 0.0))
                if "roofline" in bt:
                    result["batched"]["roofline_ms"] = _r(bt["roofline"]["ms"])
            result["split"] = split
    return result


def _r(x, d=4):
    """Round to d significant digits (keeps the JSON line short)."""
    return float(f"{x:.{d}g}") if x is not None else None


def cpu_baseline_leg(p, seconds, held, plain_tflops):
    """The oracle on the host cores: timed on a bounded sample of the CC
    workload (the cpu_baseline), and its sampled outputs -- plus the oracle
    on the small log-uniform workload and on a one-column sample of the fp32
    CC inputs -- serve as the reference of every precision form's normwise
    error.  Returns (cpu_baseline dict, compact split summary or None)."""
    import oracle
    v, cores, desc, dt, pos, ref = oracle_sample(p, seconds, want_values=True)
    cpu = {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": desc}
    if "cc_fp64" not in held:
        return cpu, None

    def rel(x, r):
        nr = float(np.linalg.norm(r))
        return float(np.linalg.norm(np.asarray(x, dtype=np.float64) - r) / (nr if nr else 1.0))

    cc = held["cc_fp64"]
    ms = held["cc_fp64_ms"]
    f = flops_of(p)
    split = {
        "cc_fp64": {"algo": "ozaki_bf16", "moduli": held["cc_fp64_moduli"], "ms": _r(ms),
                    "tflops_eff": _r(f / (ms * 1e-3) / 1e12),
                    "vs_plain": _r(f / (ms * 1e-3) / 1e12 / plain_tflops),
                    "err": _r(rel(cc["ozaki_bf16"][pos], ref), 3),
                    "plain_err": _r(rel(cc["native"][pos], ref), 3), "tol": 1e-13},
        "err_ref": "normwise vs the FP64 oracle over the cpu_baseline sample",
    }
    # SGETT forms on the CC workload in fp32: oracle of the fp32 values on one
    # column of B's last free mode
    if "cc_fp32" in held:
        p32 = held["cc_fp32"]["problem"]
        q = p32.copy()
        q.A, q.B, q.C = p32.A.astype(np.float64), p32.B.astype(np.float64), p32.C.astype(np.float64)
        _, _, desc32, _, pos32, ref32 = oracle_sample(q, 1e-9, want_values=True)
        split["cc_fp32"] = {a: {"ms": _r(e["ms"]), "tflops": _r(e["tflops"]),
                                "err": _r(rel(held["cc_fp32"][a][pos32], ref32), 3)}
                            for a, e in held["cc_fp32_timing"].items()}
        split["cc_fp32_tol"] = 1e-5
    # every form on the small log-uniform workload, all outputs
    if "small" in held:
        from paper_2410_06770_gb300 import synth
        errs = {}
        for key, (q, got) in held["small"].items():
            q64 = q.copy()
            q64.A, q64.B, q64.C = q.A.astype(np.float64), q.B.astype(np.float64), q.C.astype(np.float64)
            r = synth.gather(q64.lc, oracle.gett_problem(q64, "f64", nthreads=cores))
            errs[key] = _r(rel(synth.gather(q.lc, got), r), 3)
        split["small_logu_err"] = errs
    return cpu, split


def e2e_measure(p, flops, call_host, dA, dB, dC, a, stream, steps, dev=0):
    """Host buffers in pinned memory.  Every step copies its A, B and C from
    the host, runs the dgett call and copies C back, all inside the timed
    region.  Two device buffer sets and separate H2D / D2H streams let step
    i+1's upload overlap step i's contraction (a serving pipeline); step i+2
    reuses set i only after set i's result has reached the host."""
    import torch
    from paper_2410_06770_gb300 import gett
    hA = torch.from_numpy(p.A).pin_memory()
    hB = torch.from_numpy(p.B).pin_memory()
    hC = torch.from_numpy(p.C).pin_memory()
    sets = [(dA, dB, dC), (torch.empty_like(dA), torch.empty_like(dB), torch.empty_like(dC))]
    outs = [torch.empty_like(hC).pin_memory(), torch.empty_like(hC).pin_memory()]
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()

    calls = []  # (start, end) events of each timed call on the compute stream

    def run(nsteps, timed=False):
        free = [None, None]
        for i in range(nsteps):
            k = i % 2
            xA, xB, xC = sets[k]
            with torch.cuda.stream(h2d):
                if free[k] is not None:
                    h2d.wait_event(free[k])
                xA.copy_(hA, non_blocking=True)
                xB.copy_(hB, non_blocking=True)
                xC.copy_(hC, non_blocking=True)
                ready = torch.cuda.Event()
                ready.record(h2d)
            stream.wait_event(ready)
            if timed:
                calls.append((torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)))
                calls[-1][0].record(stream)
            gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], xA, a["RANKB"], a["EXTB"], a["INCB"], xB,
                       a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], xC,
                       a_off=p.la.off, b_off=p.lb.off, c_off=p.lc.off, mode="async", stream=stream.cuda_stream)
            if timed:
                calls[-1][1].record(stream)
            done = torch.cuda.Event()
            done.record(stream)
            with torch.cuda.stream(d2h):
                d2h.wait_event(done)
                outs[k].copy_(xC, non_blocking=True)
                free[k] = torch.cuda.Event()
                free[k].record(d2h)
        for ev in free:
            if ev is not None:
                stream.wait_event(ev)

    run(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(dev)
    sampler.start()
    e0.record(stream)
    h2d.wait_stream(stream)
    run(steps, timed=True)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / steps
    call_ms = statistics.mean(c0.elapsed_time(c1) for c0, c1 in calls)
    bi = hA.numel() * 8 + hB.numel() * 8 + hC.numel() * 8
    bo = outs[0].numel() * 8
    del sets[1]
    # call_ms: the contraction alone inside this pipeline (device time between
    # its stream's events), to tell copy overhead from a slower call
    return {"value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bo, "ms_per_step": ms, "steps": steps, "call_ms": call_ms,
            "clocks": clocks,
            "pipeline": "2 device buffer sets; H2D of step i+1 overlaps the call of step i"}


def time_calls(call, reps, warm=2):
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        call()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return min(times), statistics.median(times)


def measure_split_forms(held):
    """Split-precision DGETT on the CC workload, SGETT's forms on the CC
    workload in fp32, and every precision form on the small workload with
    log-uniform magnitudes.  Timing only, plus each form's difference from
    the native FP64 path on the GPU; the results are kept in `held` so the
    CPU-baseline leg can state every form's error against the oracle."""
    import torch
    from paper_2410_06770_gb300 import gett, synth
    out = {}
    mp = measured_peaks()
    bf16_peak = mp.get("bf16_tflops", 1900.0)
    stream = torch.cuda.current_stream()

    def run(prefix, q, algo, dA, dB, C0):
        """One call on a fresh copy of C0; returns (device C, report)."""
        dC = C0.clone()
        _, rep = gett.xgett(prefix, len(q.sig.exta), q.sig.exta, q.la.inc, dA, len(q.sig.extb), q.sig.extb,
                            q.lb.inc, dB, q.sig.conts, q.sig.conta, q.sig.contb, q.sig.perm, q.lc.inc, dC,
                            a_off=q.la.off, b_off=q.lb.off, c_off=q.lc.off, mode="ex",
                            opts=gett.options(algo=algo), stream=stream.cuda_stream)
        torch.cuda.synchronize()
        return dC, rep

    def rel(x, ref):
        d = (x - ref).to(torch.complex128 if x.is_complex() else torch.float64)
        r = ref.to(d.dtype)
        return float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(r))

    # CC at full size: modular split vs native FP64, every output compared
    p, desc = workload("cc")
    dA = torch.from_numpy(p.A).cuda()
    dB = torch.from_numpy(p.B).cuda()
    C0 = torch.from_numpy(p.C).cuda()
    ref, rep_plain = run("d", p, "native", dA, dB, C0)
    dC, rep = run("d", p, "ozaki_bf16", dA, dB, C0)
    diff = rel(dC, ref)
    held["cc_fp64"] = {"native": ref.cpu().numpy(), "ozaki_bf16": dC.cpu().numpy()}
    del dC, ref

    def call():
        return gett.xgett("d", len(p.sig.exta), p.sig.exta, p.la.inc, dA, len(p.sig.extb), p.sig.extb, p.lb.inc,
                          dB, p.sig.conts, p.sig.conta, p.sig.contb, p.sig.perm, p.lc.inc, C0, a_off=p.la.off,
                          b_off=p.lb.off, c_off=p.lc.off, mode="ex", opts=gett.options(algo="ozaki_bf16"),
                          stream=stream.cuda_stream)
    best, med = time_calls(call, 5)
    f = flops_of(p)
    L = rep["moduli"]
    held["cc_fp64_ms"] = best
    held["cc_fp64_moduli"] = L
    out["cc_split_fp64"] = {
        "workload": desc, "algo": "ozaki_bf16 (modular, bf16 tcgen05)", "moduli": L,
        "ms": best, "ms_median": med, "tflops_effective": f / (best * 1e-3) / 1e12,
        "slice_tflops": L * f / (best * 1e-3) / 1e12, "slice_frac_of_bf16_peak": L * f / (best * 1e-3) / 1e12 / bf16_peak,
        "normwise_diff_vs_native_fp64": diff, "compared": "all 16.8M outputs against the native FP64 call on the GPU"}
    del dA, dB, C0
    torch.cuda.empty_cache()
    # SGETT at scale: the CC contraction in fp32, native FFMA against the bf16
    # split forms on tcgen05 (C from zero for each call)
    p32 = p.copy()
    p32.A, p32.B, p32.C = p.A.astype(np.float32), p.B.astype(np.float32), p.C.astype(np.float32)
    dA, dB = torch.from_numpy(p32.A).cuda(), torch.from_numpy(p32.B).cuda()
    C0 = torch.from_numpy(p32.C).cuda()
    held["cc_fp32"] = {"problem": p32}
    sf = {}
    for algo in ("native", "bf16x3", "bf16x6"):
        got, rep32 = run("s", p32, algo, dA, dB, C0)
        held["cc_fp32"][algo] = got.cpu().numpy()
        del got

        dCt = C0.clone()  # the timed calls accumulate here, not into C0

        def c32():
            return gett.xgett("s", len(p32.sig.exta), p32.sig.exta, p32.la.inc, dA, len(p32.sig.extb),
                              p32.sig.extb, p32.lb.inc, dB, p32.sig.conts, p32.sig.conta, p32.sig.contb,
                              p32.sig.perm, p32.lc.inc, dCt, mode="ex", opts=gett.options(algo=algo),
                              stream=stream.cuda_stream)
        b32, m32 = time_calls(c32, 5)
        del dCt
        sf[algo] = {"ms": b32, "ms_median": m32, "tflops": f / (b32 * 1e-3) / 1e12, "family": rep32["family_name"]}
        held.setdefault("cc_fp32_timing", {})[algo] = sf[algo]
    out["cc_sgett_forms"] = {"workload": desc + ", fp32", "forms": sf}
    del dA, dB, C0
    torch.cuda.empty_cache()
    # small workload, log-uniform magnitudes: every form against native FP64 on
    # the same (for s: fp32-rounded) inputs
    ps = synth.cfg_small_dgett(dist="logu")
    held["small"] = {}
    forms = {}
    for prefix, algo in (("d", "native"), ("d", "ozaki_bf16"), ("s", "native"), ("s", "bf16x3"), ("s", "bf16x6")):
        q = ps.copy()
        if prefix == "s":
            q.A = ps.A.astype(np.float32)
            q.B = ps.B.astype(np.float32)
            q.C = ps.C.astype(np.float32)
        # FP64 reference on exactly the values this form sees
        dA64 = torch.from_numpy(q.A.astype(np.float64)).cuda()
        dB64 = torch.from_numpy(q.B.astype(np.float64)).cuda()
        ref, _ = run("d", q, "native", dA64, dB64, torch.from_numpy(q.C.astype(np.float64)).cuda())
        dA, dB = torch.from_numpy(q.A).cuda(), torch.from_numpy(q.B).cuda()
        C0 = torch.from_numpy(q.C).cuda()
        got, _ = run(prefix, q, algo, dA, dB, C0)
        pos = torch.from_numpy(synth.gather(q.lc, np.arange(q.C.size, dtype=np.int64))).cuda()
        err = rel(got[pos].double(), ref[pos])
        held["small"][f"{prefix}gett/{algo}"] = (q, got.cpu().numpy())

        def c2():
            return gett.xgett(prefix, len(q.sig.exta), q.sig.exta, q.la.inc, dA, len(q.sig.extb), q.sig.extb,
                              q.lb.inc, dB, q.sig.conts, q.sig.conta, q.sig.contb, q.sig.perm, q.lc.inc, C0,
                              a_off=q.la.off, b_off=q.lb.off, c_off=q.lc.off, mode="ex",
                              opts=gett.options(algo=algo), stream=stream.cuda_stream)
        best, _ = time_calls(c2, 20)
        forms[f"{prefix}gett/{algo}"] = {"normwise_err_vs_native_fp64": err, "ms": best,
                                         "tflops": flops_of(q) / (best * 1e-3) / 1e12}
    out["small_logu_forms"] = {"workload": "dgett_small shapes, 10^U(-8,8) magnitudes, random signs",
                               "forms": forms}
    # complex double: the CC contraction at a..d = 64, i,j = 16, native vs split
    pz = synth.cfg_cc("plain", dtype=np.complex128, scale=64, small_ij=16)
    dA, dB = torch.from_numpy(pz.A).cuda(), torch.from_numpy(pz.B).cuda()
    C0 = torch.from_numpy(pz.C).cuda()
    zref = None
    zf = {}
    for algo in ("native", "ozaki_bf16"):
        got, rep = run("z", pz, algo, dA, dB, C0)
        if zref is None:
            zref = got
        dCz = C0.clone()

        def cz():
            return gett.xgett("z", len(pz.sig.exta), pz.sig.exta, pz.la.inc, dA, len(pz.sig.extb), pz.sig.extb,
                              pz.lb.inc, dB, pz.sig.conts, pz.sig.conta, pz.sig.contb, pz.sig.perm, pz.lc.inc, dCz,
                              mode="ex", opts=gett.options(algo=algo), stream=stream.cuda_stream)
        best, _ = time_calls(cz, 3)
        fz = 4 * flops_of(pz)
        zf[f"zgett/{algo}"] = {"ms": best, "tflops": fz / (best * 1e-3) / 1e12, "moduli": rep["moduli"],
                               "normwise_diff_vs_native": rel(got, zref)}
        del dCz
    del dA, dB, C0, zref
    out["cc64_complex_forms"] = {"workload": "complex CC, a..d=64, i,j=16 (8 real flops per complex MAC)",
                                 "forms": zf}
    return out


MODEL_PATH = os.path.join(ROOT, "paper_2410_06770_gb300", "planner_mlp.npz")
TUNE_DB = os.path.join(ROOT, "paper_2410_06770_gb300", "tune_db.txt")


def measure_batched(n=4096, ffma_tflops=None):
    """The batched workload: one batched launch (CUDA graph replay) for all
    contractions vs one plain call per contraction, with heuristic, tuned and
    (if a trained model is committed) learned tile configurations.  Roofline:
    the sum over problems of max(2|C|K / FFMA peak, bytes / HBM), bytes = A
    and B at their storage size plus C read and written (fp32)."""
    import torch
    from paper_2410_06770_gb300 import batch as gb
    from paper_2410_06770_gb300 import gett, tune
    probs = tune.draw_problems(n, 7, 64)
    total_flops = sum(tune.flops(p) for p in probs)
    bufs = tune.DeviceBuffers(probs, values=True)
    stream = torch.cuda.current_stream()
    out = {"workload": f"{n} contractions, seed 7, ranks 2-5, extents 2-64 (<= 2^18 elements), "
                       "0-3 contracted, 25% padded, fp32/bf16 operands, fp32 C",
           "gflop": total_flops / 1e9}

    def per_call():
        for pr, d in zip(probs, bufs.descs):
            a = tune.args_of(pr)
            gett.xgett("sb" if pr["dtype"] == "bf16" else "s", len(a["EXTA"]), a["EXTA"], a["INCA"], d["A"],
                       len(a["EXTB"]), a["EXTB"], a["INCB"], d["B"], len(a["CONTA"]), a["CONTA"], a["CONTB"],
                       a["PERM"], a["INCC"], d["C"], mode="async", stream=stream.cuda_stream)
    per_call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    per_call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t0))
    out["per_call"] = {"ms": ms, "contractions_per_s": n / (ms * 1e-3), "tflops": total_flops / (ms * 1e-3) / 1e12}
    del bufs
    torch.cuda.empty_cache()
    out["batched_heuristic"] = tune.throughput(probs, "heuristic")
    T = tune.measure(probs, reps=2)
    tuned = list(np.nanargmin(T, axis=1))
    out["batched_tuned"] = tune.throughput(probs, "table", configs=tuned)
    if os.path.exists(MODEL_PATH):
        tune.install(tune.load_model(MODEL_PATH))
        out["batched_learned"] = tune.throughput(probs, "learned")
        # the same launch with every kernel on one stream (no concurrent branches)
        out["batched_learned_serial"] = tune.throughput(probs, "learned", serial=True)
        gb.clear_model()
    out["speedup_batched_vs_per_call"] = out["per_call"]["ms"] / out["batched_heuristic"]["ms"]
    if ffma_tflops:
        mp = measured_peaks()
        bw = mp.get("hbm_gbs", 6800.0) * 1e9
        bf16_peak = mp.get("bf16_tflops", 1900.0) * 1e12
        roof_s = roof_dt = 0.0
        for pr in probs:
            esz = 2 if pr["dtype"] == "bf16" else 4
            nbytes = esz * (pr["la"].numel + pr["lb"].numel) + 8 * pr["lc"].numel
            roof_s += max(tune.flops(pr) / (ffma_tflops * 1e12), nbytes / bw)
            peak = bf16_peak if pr["dtype"] == "bf16" else ffma_tflops * 1e12
            roof_dt += max(tune.flops(pr) / peak, nbytes / bw)
        best = min(v["ms"] for k, v in out.items() if k.startswith("batched_"))
        out["roofline"] = {"ms": roof_s * 1e3, "frac_of_best": roof_s * 1e3 / best,
                           "definition": "sum over problems of max(flops / FFMA peak, bytes / HBM), "
                                         "FFMA peak measured, HBM of MEASURED_PEAKS",
                           "ms_bf16_on_tensor_peak": roof_dt * 1e3, "frac_of_best_bf16_on_tensor_peak":
                           roof_dt * 1e3 / best}
    return out


def measure_streaming_forms(dfma_tflops=None):
    """Low-intensity kernels beyond the outer product: a full inner product of
    two 128^4 tensors (REDUCE, 4.3 GB read) and a matrix-vector contraction
    A(16384, 16384) x B(16384, 2) (SKINNY, 2.1 GB read).  Each is bounded by
    HBM or, in FP64 on this GPU, by the FMA rate (2 flops per element and
    short-class column): both fractions are given, and `bound` names the
    larger floor."""
    import torch
    from paper_2410_06770_gb300 import gett, synth
    mp = measured_peaks()
    bw = mp.get("hbm_gbs", 6800.0)
    out = {}
    stream = torch.cuda.current_stream()
    cases = {
        "inner_product": (synth.Signature((128,) * 4, (128,) * 4, (0, 1, 2, 3), (0, 1, 2, 3), ()), "reduce"),
        "gemv": (synth.Signature((16384, 16384), (16384, 2), (1,), (0,), (0, 1)), "skinny"),
    }
    for name, (sig, fam) in cases.items():
        la, lb, lc = synth.layout_contiguous(sig.exta), synth.layout_contiguous(sig.extb), synth.layout_contiguous(sig.extc())
        g = torch.Generator(device="cuda")
        g.manual_seed(9)
        dA = torch.rand(la.size, dtype=torch.float64, device="cuda", generator=g)
        dB = torch.rand(lb.size, dtype=torch.float64, device="cuda", generator=g)
        dC = torch.zeros(lc.size, dtype=torch.float64, device="cuda")
        a = dict(RANKA=len(sig.exta), EXTA=sig.exta, INCA=la.inc, RANKB=len(sig.extb), EXTB=sig.extb,
                 INCB=lb.inc, CONTS=sig.conts, CONTA=sig.conta, CONTB=sig.contb, PERM=sig.perm, INCC=lc.inc)

        def call():
            return gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB,
                              a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC, mode="ex",
                              stream=stream.cuda_stream)
        _, rep = call()
        best, _ = time_calls(call, 5)
        nbytes = 8.0 * (la.numel + lb.numel + 2 * lc.numel)
        flops = 2.0 * rep["M"] * rep["N"] * rep["K"]
        ent = {"family": rep["family_name"], "ms": best, "gbs": nbytes / (best * 1e-3) / 1e9,
               "hbm_frac": nbytes / (best * 1e-3) / 1e9 / bw,
               "tflops": flops / (best * 1e-3) / 1e12,
               "shape": f"A{sig.exta} x B{sig.extb}, CONTS={sig.conts}"}
        if dfma_tflops:
            ent["dfma_frac"] = ent["tflops"] / dfma_tflops
            hbm_floor = nbytes / (bw * 1e9)
            alu_floor = flops / (dfma_tflops * 1e12)
            ent["bound"] = "hbm" if hbm_floor >= alu_floor else "alu"
            ent["floor_ms"] = max(hbm_floor, alu_floor) * 1e3
            ent["floor_frac"] = ent["floor_ms"] / best
        out[name] = ent
        del dA, dB, dC
        torch.cuda.empty_cache()
    out.update(measure_aux_forms(bw, dfma_tflops))
    return out


def measure_aux_forms(bw, dfma_tflops):
    """Transpose (xGETP) of a 128^4 FP64 tensor with its modes reversed (read
    2.1 GB, write 2.1 GB; C is not read), and reductions (xGETR) of a
    16384 x 16384 FP64 matrix over either mode (read 2.1 GB, one FMA per
    element: FP64-bound on this GPU)."""
    import torch
    from paper_2410_06770_gb300 import gett, synth
    out = {}
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    ext = (128, 128, 128, 128)
    la = synth.layout_contiguous(ext)
    perm = (3, 2, 1, 0)
    lc = synth.layout_contiguous(tuple(ext[perm.index(q)] for q in range(4)))
    dA = torch.rand(la.size, dtype=torch.float64, device="cuda", generator=g)
    dC = torch.empty(lc.size, dtype=torch.float64, device="cuda")

    def tcall():
        gett.getp("d", 4, ext, la.inc, dA, perm, lc.inc, dC, alpha=1.0, beta=0.0)
    best, _ = time_calls(tcall, 5)
    nbytes = 16.0 * la.numel
    out["transpose"] = {"op": "dgetp", "shape": "A(128,128,128,128) -> C with PERM (3,2,1,0), beta = 0",
                        "ms": best, "gbs": nbytes / (best * 1e-3) / 1e9,
                        "hbm_frac": nbytes / (best * 1e-3) / 1e9 / bw}
    del dA, dC
    torch.cuda.empty_cache()
    n = 16384
    dA = torch.rand(n * n, dtype=torch.float64, device="cuda", generator=g)
    dC = torch.empty(n, dtype=torch.float64, device="cuda")
    for red, name in (((0,), "reduce_fast_mode"), ((1,), "reduce_slow_mode")):
        def rcall():
            gett.getr("d", 2, (n, n), (1, n), dA, 1, red, (0,), (1,), dC, alpha=1.0, beta=0.0)
        best, _ = time_calls(rcall, 5)
        nbytes = 8.0 * n * n
        ent = {"op": "dgetr", "shape": f"A({n},{n}) summed over mode {red[0]}", "ms": best,
               "gbs": nbytes / (best * 1e-3) / 1e9, "hbm_frac": nbytes / (best * 1e-3) / 1e9 / bw}
        if dfma_tflops:
            alu_floor = n * n / (dfma_tflops * 1e12 / 2)
            hbm_floor = nbytes / (bw * 1e9)
            ent["bound"] = "hbm" if hbm_floor >= alu_floor else "alu"
            ent["floor_ms"] = max(alu_floor, hbm_floor) * 1e3
            ent["floor_frac"] = ent["floor_ms"] / best
        out[name] = ent
    del dA, dC
    torch.cuda.empty_cache()
    return out


def measure_forms(main_workload):
    """Other forms of the headline metric, each timed on its own (CUDA events,
    3 warm-up calls, best of the timed calls)."""
    import torch
    from paper_2410_06770_gb300 import gett
    out = {}
    names = [w for w in ("cc_perm_transA", "stream", "small") if w != main_workload]
    for name in names:
        p, desc = workload(name)
        a = p.args()
        dA = torch.from_numpy(p.A).cuda()
        dB = torch.from_numpy(p.B).cuda()
        if p.meta.get("c_zero"):
            dC = torch.zeros(p.lc.size, dtype=torch.float64, device="cuda")
        else:
            dC = torch.from_numpy(p.C).cuda()
        stream = torch.cuda.current_stream()

        def call():
            return gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB,
                              a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC,
                              a_off=p.la.off, b_off=p.lb.off, c_off=p.lc.off, mode="async",
                              stream=stream.cuda_stream)
        _, rep = gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB,
                            a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC,
                            a_off=p.la.off, b_off=p.lb.off, c_off=p.lc.off, mode="ex",
                            stream=stream.cuda_stream)
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        times = []
        reps = 5 if name != "small" else 50
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = min(times)
        f = flops_of(p)
        entry = {"workload": desc, "ms": ms, "tflops": f / (ms * 1e-3) / 1e12,
                 "family": rep["family_name"], "config": rep["config"], "split_k": rep["split_k"]}
        if rep["family_name"] in ("outer", "reduce"):
            entry["gbs"] = bytes_of(p) / (ms * 1e-3) / 1e9
            mp = measured_peaks()
            entry["hbm_frac"] = entry["gbs"] / mp.get("hbm_gbs", 6800.0)
        out[name] = entry
        if name == "stream":
            # the scaled form with beta = 0 writes C without reading it
            def call0():
                return gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB,
                                  a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC,
                                  a_off=p.la.off, b_off=p.lb.off, c_off=p.lc.off, mode="scaled", alpha=1.0,
                                  beta=0.0, stream=stream.cuda_stream)
            best0, _ = time_calls(call0, 5)
            nb0 = 8.0 * (p.la.numel + p.lb.numel + p.lc.numel)
            mp = measured_peaks()
            out["stream_beta0"] = {"workload": desc + ", scaled form alpha = 1, beta = 0 (C not read)",
                                   "ms": best0, "gbs": nb0 / (best0 * 1e-3) / 1e9,
                                   "hbm_frac": nb0 / (best0 * 1e-3) / 1e9 / mp.get("hbm_gbs", 6800.0),
                                   "speedup_vs_accumulate": ms / best0}
        del dA, dB, dC
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# reference arm: the oracle on host cores
# ---------------------------------------------------------------------------
def reference_arm(args, dist: Dist):
    import oracle
    oracle.build()
    p, wdesc = workload(args.workload)
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(p, per_step)
    vals, times, desc, cores = [], [], "", 1
    for _ in range(args.steps):
        v, cores, desc, dt = oracle_sample(p, per_step)
        vals.append(v)
        times.append(dt)
    value = statistics.mean(vals)
    return {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1))", "impl": "reference",
        "config": {"workload": wdesc},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    if args.impl == "reference":
        dist = Dist("gloo")
        if dist.rank != 0:
            dist.close()
            return 0
        res = reference_arm(args, dist)
        print(json.dumps(res), flush=True)
        dist.close()
        return 0
    dist = Dist("nccl")
    res = gpu_arm(args, dist)
    if dist.rank == 0:
        print(json.dumps(res), flush=True)
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
