#!/usr/bin/env python3
"""Benchmark: sgemm TFLOP/s at m = n = k = 8192 on one GB300, split-BF16 tensor
path (the headline) against the plain FP32 SIMT path, same inputs.

Workload: the square sgemm sweep's 8192^3 point -- column-major, transa =
transb = 'N', lda = ldb = ldc = 8200 (rows + 8), alpha = 1.5, beta = -0.25,
A, B, C uniform[-1, 1) from seed 1 (SplitMix64 generator).  A step is one
gbgemm_sgemm call on the split path: hi/lo packing of both operands (with
their row maxima), the re-pack of badly scaled rows and the tcgen05 GEMM,
everything the call does.  TFLOP/s =
2 m n k / time (the paper's FLOP convention, Tables I-VI).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (FP64 triple loop) on the host cores
on bounded samples of the same workload: each step computes one 128 x 128
block of C (k = 8192) with every core.

Prints one JSON line (rank 0).  With N > 1 (torchrun, one rank per GPU) every
rank runs its own replica of the workload (the path does not shard) and
value = all ranks' FLOPs / the slowest rank's time.
"""

from __future__ import annotations

import argparse
import csv
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sgemm TFLOP/s at 8192^3: 3xBF16 tensor vs FP32 SIMT, same GPU, same error bound"
# DRAM bytes (read + write) of one split_gemm_kernel launch at 8192^3 NN, ld 8200,
# from one ncu capture of the current kernel (profiles/split_gemm_8192_nn_traffic.md);
# None until that capture has been taken of this kernel.
GEMM_TRAFFIC_8192 = 2810343936 + 257446656
UNIT = "TFLOP/s"
N = 8192
LD = N + 8
ALPHA, BETA = 1.5, -0.25
SEED = 1


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", 0.0)), float(d["hbm_gbs"]), "measured"
    except Exception:
        return 1900.0, 1700.0, 6800.0, "fallback"


def config(**extra):
    c = {"workload": "sgemm m=n=k=8192 NN, ld=8200, alpha=1.5, beta=-0.25, uniform[-1,1) seed 1",
         "m": N, "n": N, "k": N, "transa": "N", "transb": "N", "lda": LD, "ldb": LD, "ldc": LD,
         "l2": "inputs larger than L2 (3 x 268 MB vs 126 MB L2); no flush"}
    c.update(extra)
    return c


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for r in csv.reader(f):
                r = [x.strip() for x in r]
                if len(r) < 9:
                    continue
                if self.uuid and self.uuid not in r[0]:
                    continue
                rows.append(r)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
# CPU oracle sample (the reference arm and the cpu_baseline field)
# ---------------------------------------------------------------------------
def oracle_sample(steps: int, block: int = 128, warmup: int = 0, nthreads: int = 0):
    """Time the FP64 oracle on `steps` blocks of the 8192^3 product (all cores,
    or `nthreads` threads)."""
    import numpy as np

    from oracle import oracle as O
    from paper_1608_05265_gb300 import synth

    threads = nthreads if nthreads > 0 else O.max_threads()
    times = []
    flops = 0.0
    for s in range(warmup + steps):
        i0 = (s * 977) % (N - block)
        j0 = (s * 1531) % (N - block)
        # rows i0.. of A (m x k, N layout), columns j0.. of B (k x n) and the C block
        A = synth.uniform_block(SEED, 0, N, i0, i0 + block, 0, N)
        B = synth.uniform_block(SEED, 2, N, 0, N, j0, j0 + block)
        C = synth.uniform_block(SEED, 4, N, i0, i0 + block, j0, j0 + block)
        t0 = time.perf_counter()
        O.gemm_f64("N", "N", block, block, N, ALPHA, A, block, B, N, BETA, C, block, want_bound=False,
                   nthreads=threads)
        dt = time.perf_counter() - t0
        if s >= warmup:
            times.append(dt)
            flops += 2.0 * block * block * N
    total = sum(times)
    return {"value": flops / total / 1e12 if total > 0 else 0.0, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{steps} blocks of {block}x{block} of C (k={N}), FP64 triple loop, {threads} threads",
            "seconds": total}


def host_cpu_model() -> str:
    """The host CPU's model name and logical core count, from lscpu or /proc/cpuinfo."""
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        name = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return f"{name or 'unknown'} x {os.cpu_count()}"


def run_reference(args, rank, world):
    if rank != 0:
        return
    res = oracle_sample(args.steps, warmup=args.warmup)
    secs = res.pop("seconds")
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1000.0 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(), "cpu_baseline": dict(res),
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1608_05265_gb300 import build as gbuild
    from paper_1608_05265_gb300 import gbgemm, metrics, synth

    gbuild.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()

    # Inputs: generated on the host (seeded), pinned for the end-to-end leg.
    A_h = torch.from_numpy(synth.uniform_matrix(SEED, 0, N, N, LD)).pin_memory()
    B_h = torch.from_numpy(synth.uniform_matrix(SEED, 2, N, N, LD)).pin_memory()
    C_h = torch.from_numpy(synth.uniform_matrix(SEED, 4, N, N, LD)).pin_memory()
    Cout_h = torch.empty_like(C_h).pin_memory()
    A = A_h.to(dev)
    B = B_h.to(dev)
    C0 = C_h.to(dev)
    C = C0.clone()

    h = gbgemm.Handle(local_rank)
    h.set_stream(stream)
    h.reserve_workspace(gbgemm.split_workspace_bytes(N, N, N))
    flop = metrics.gemm_flops(N, N, N)

    def step(path):
        h.set_path(path)
        h.sgemm("N", "N", N, N, N, ALPHA, A, LD, B, LD, BETA, C, LD)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # ---- split path (the headline) ----
    for _ in range(args.warmup):
        step(gbgemm.PATH_SPLIT_BF16)
    barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    barrier()
    h.profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(gbgemm.PATH_SPLIT_BF16)
    e1.record(stream)
    barrier()
    gemm_ms, gemm_launches, launches = h.profile_end()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms)
    status = h.get_device_status()
    if status != 0:
        raise RuntimeError(f"device status {status} ({gbgemm.status_string(status)})")
    value = world * args.steps * flop / (ms_max * 1e-3) / 1e12

    # ---- SIMT path on the same inputs (comparison, not the headline) ----
    simt_steps = max(2, min(args.steps, 5))
    step(gbgemm.PATH_SIMT)
    barrier()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(simt_steps):
        step(gbgemm.PATH_SIMT)
    s1.record(stream)
    barrier()
    simt_ms = max_over_ranks(s0.elapsed_time(s1)) / simt_steps
    simt_tflops = flop / (simt_ms * 1e-3) / 1e12

    # ---- end to end: pinned host buffers in, C back to the host, every step ----
    # Each step copies its A, B and C from pinned host memory, multiplies and
    # reads C back.  Three device buffer sets let step i+1's host-to-device
    # copies and step i-1's read-back run on copy streams while step i
    # multiplies: the throughput of a pipelined caller, every byte still moved.
    e2e_steps = max(4, min(args.steps, 12))
    h.set_path(gbgemm.PATH_SPLIT_BF16)
    NSET = 3
    sets = [(A, B, C)] + [(torch.empty_like(A), torch.empty_like(B), torch.empty_like(C)) for _ in range(NSET - 1)]
    outs = [Cout_h] + [torch.empty_like(Cout_h).pin_memory() for _ in range(NSET - 1)]
    h2d = [torch.cuda.Stream(device=dev) for _ in range(3)]  # one per input: several copy engines
    d2h = torch.cuda.Stream(device=dev)
    ev_in = [[torch.cuda.Event() for _ in range(3)] for _ in range(NSET)]
    ev_done = [torch.cuda.Event() for _ in range(NSET)]
    ev_out = [torch.cuda.Event() for _ in range(NSET)]
    barrier()
    x0 = torch.cuda.Event(enable_timing=True)
    x1 = torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    for hs in h2d:
        hs.wait_event(x0)
    used = [False] * NSET
    for it in range(e2e_steps):
        b = it % NSET
        for q, (hs, dst, src, ev) in enumerate(zip(h2d, sets[b], (A_h, B_h, C_h), ev_in[b])):
            if used[b]:
                # A and B of the set may be overwritten once its previous sgemm is done;
                # C only once that result has been read back
                hs.wait_event(ev_out[b] if q == 2 else ev_done[b])
            with torch.cuda.stream(hs):
                dst.copy_(src, non_blocking=True)
                ev.record(hs)
            stream.wait_event(ev)
        Ab, Bb, Cb = sets[b]
        h.sgemm("N", "N", N, N, N, ALPHA, Ab, LD, Bb, LD, BETA, Cb, LD)
        ev_done[b].record(stream)
        d2h.wait_event(ev_done[b])
        with torch.cuda.stream(d2h):
            outs[b].copy_(Cb, non_blocking=True)
            ev_out[b].record(d2h)
        used[b] = True
    stream.wait_stream(d2h)
    x1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(x0.elapsed_time(x1)) / e2e_steps
    e2e_value = world * flop / (e2e_ms * 1e-3) / 1e12
    assert h.get_device_status() == 0
    assert all(np.isfinite(o[:1000].numpy()).all() for o in outs)
    del sets

    # ---- roofline of the dominant kernel (the tcgen05 GEMM) ----
    bf16_peak, bf16_sust, hbm, peak_src = load_peaks()
    gemm_avg_ms = gemm_ms / max(gemm_launches, 1)
    achieved = flop / (gemm_avg_ms * 1e-3) / 1e12
    peak = bf16_peak / 3.0
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": GEMM_TRAFFIC_8192, "kernel": "split_gemm_kernel<SingleSched, 6, 256, pair>",
                "note": (f"sgemm-equivalent 2mnk per launch / launch time; peak = {peak_src} bf16 dense "
                         f"{bf16_peak:.1f} TFLOP/s / 3 products (sustained {bf16_sust:.1f}/3 = "
                         f"{bf16_sust / 3:.1f}: frac {achieved / (bf16_sust / 3) if bf16_sust else float('nan'):.3f})"),
                "gemm_share_of_step": gemm_ms / ms if ms > 0 else None}

    # ---- accuracy of one call, FP64 on the GPU (outside the timed region) ----
    C.copy_(C0)
    h.set_path(gbgemm.PATH_SPLIT_BF16)
    h.sgemm("N", "N", N, N, N, ALPHA, A, LD, B, LD, BETA, C, LD)
    torch.cuda.synchronize()
    err = {"max_error_ratio": max(
        h.check_error("N", "N", N, N, N, ALPHA, A, LD, B, LD, BETA, C0, C, LD, rows=(i0, i0 + 512), cols=(j0, j0 + 512))
        for (i0, j0) in ((0, 0), (N - 512, N - 512), (3584, 1024))),
        "blocks": "3 blocks of 512x512 (corner, corner, interior), FP64 on the GPU",
        "bound": "|C - C64| <= 2 k 2^-24 (|alpha||A||B| + |beta||C|)"}
    extras = {}
    if args.extras and rank == 0:
        extras = run_extras(h, stream, flop)

    if rank == 0:
        cpu = oracle_sample(steps=max(1, args.cpu_blocks)) if args.cpu_blocks > 0 else None
        if cpu:
            cpu.pop("seconds", None)
            one = oracle_sample(steps=1, nthreads=1)
            one.pop("seconds", None)
            cpu["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample")}
            cpu["host_cpu"] = host_cpu_model()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3-split (fp32 in/out, fp32 accumulate)",
            "data": "synthetic", "config": config(parallelism=f"replicas x{world}"),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * N * LD * 4,
                    "d2h_bytes_per_step": N * LD * 4, "steps": e2e_steps,
                    "pipelining": "copies of step i+1 (in) and i-1 (out) overlap step i's sgemm; 3 buffer sets"},
            "gpu_launches": launches,
            "roofline": roofline,
            "simt": {"value": simt_tflops, "unit": UNIT, "ms_per_step": simt_ms, "steps": simt_steps},
            "split_over_simt": value / world / simt_tflops if simt_tflops > 0 else None,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "error_check": err,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()


def _time(fn, stream, reps):
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _time_stats(fn, stream, reps, flush=None):
    """Median and minimum of `reps` individually timed calls (CUDA events on the
    launching stream); `flush`, a buffer larger than L2, is rewritten before
    every call, outside the timed pair."""
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    pairs = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        pairs.append((e0, e1))
    torch.cuda.synchronize()
    t = sorted(x.elapsed_time(y) for x, y in pairs)
    return t[len(t) // 2], t[0]


def run_extras(h, stream, flop8192):
    """The square sweep, the Linpack-shaped updates, the 256^3 SIMT case and the
    grouped uneven batch.  Inputs generated on the device (seeded torch
    generators); L2 (129 MB) flushed before every timed call of a sweep point."""
    import torch
    from paper_1608_05265_gb300 import gbgemm, metrics, synth
    out = {}
    g = torch.Generator(device="cuda")
    flush = torch.empty(64 * 1024 * 1024, device="cuda")  # 256 MB
    _, _, hbm, peak_src = load_peaks()

    # -- 256^3 NN, ld 256, alpha 1, beta 0.5, uniform (seed 0): SIMT only --
    A0_, B0_, C0_ = (torch.from_numpy(x).cuda() for x in synth.gemm_problem("uniform", 0, "N", "N", 256, 256, 256)[0::2])
    Cw = C0_.clone()
    h.set_path(gbgemm.PATH_SIMT)
    med, mn = _time_stats(lambda: h.sgemm("N", "N", 256, 256, 256, 1.0, A0_, 256, B0_, 256, 0.5, Cw, 256), stream, 20,
                          flush)
    Cw.copy_(C0_)
    h.sgemm("N", "N", 256, 256, 256, 1.0, A0_, 256, B0_, 256, 0.5, Cw, 256)
    torch.cuda.synchronize()
    out["simt_256"] = {"us_median": med * 1e3, "us_min": mn * 1e3,
                       "tflops": metrics.gemm_flops(256, 256, 256) / (med * 1e-3) / 1e12,
                       "max_error_ratio": h.check_error("N", "N", 256, 256, 256, 1.0, A0_, 256, B0_, 256, 0.5, C0_, Cw,
                                                        256)}
    del A0_, B0_, C0_, Cw

    # -- square sweep: n in {1024, 2048, 4096, 8192}, four transposes, ld = n + 8,
    #    alpha 1.5, beta -0.25, uniform (device generator, seed 1), both paths --
    sweep = {}
    rates = {}
    for n in (1024, 2048, 4096, 8192):
        ld = n + 8
        g.manual_seed(1)
        A = torch.rand(n * ld, device="cuda", generator=g) * 2 - 1
        B = torch.rand(n * ld, device="cuda", generator=g) * 2 - 1
        C0 = torch.rand(n * ld, device="cuda", generator=g) * 2 - 1
        C = C0.clone()
        blocks = [((0, n), (0, n))] if n <= 2048 else [((0, 256), (0, 256)), ((n - 256, n), (n // 2, n // 2 + 256))]
        for ta, tb in (("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")):
            pt = {}
            for path, name in ((gbgemm.PATH_SPLIT_BF16, "split"), (gbgemm.PATH_SIMT, "simt")):
                h.set_path(path)
                reps = 10 if (name == "split" or n <= 4096) else 3
                med, mn = _time_stats(lambda: h.sgemm(ta, tb, n, n, n, 1.5, A, ld, B, ld, -0.25, C, ld), stream, reps,
                                      flush)
                C.copy_(C0)
                h.sgemm(ta, tb, n, n, n, 1.5, A, ld, B, ld, -0.25, C, ld)
                torch.cuda.synchronize()
                err = max(h.check_error(ta, tb, n, n, n, 1.5, A, ld, B, ld, -0.25, C0, C, ld, rows=r, cols=c)
                          for r, c in blocks)
                fl = metrics.gemm_flops(n, n, n)
                pt[name] = {"tflops": fl / (med * 1e-3) / 1e12, "tflops_best": fl / (mn * 1e-3) / 1e12,
                            "ms_median": med, "max_error_ratio": err}
            pt["split_over_simt"] = pt["split"]["tflops"] / pt["simt"]["tflops"]
            sweep[f"{n}_{ta}{tb}"] = pt
            if n == 4096 and ta == "N" and tb == "N":
                rates = {"split": pt["split"]["tflops"], "simt": pt["simt"]["tflops"]}
        del A, B, C, C0
    out["square_sweep"] = dict(sweep, note=("ld = n + 8, alpha 1.5, beta -0.25; median of 10 calls (3 for SIMT at "
                                            "8192), L2 flushed before each; error ratio on the full result for "
                                            "n <= 2048, on two 256x256 blocks above"))

    # -- Linpack-shaped trailing updates: C(m x m) -= A(m x nb) B(nb x m), m in
    #    {4096, 8192, 16384}, nb in {128, 256}, entries normal(0,1) 2^e per row --
    lp = {}
    for m in (4096, 8192, 16384):
        for nb in (128, 256):
            g.manual_seed(20 + nb)
            def rowscaled(rows, cols):
                x = torch.randn(cols, rows, device="cuda", generator=g)
                e = torch.randint(-20, 21, (rows,), device="cuda", generator=g).float()
                return (x * torch.exp2(e)[None, :]).reshape(-1).contiguous()
            A = rowscaled(m, nb)
            B = rowscaled(nb, m)
            C0 = rowscaled(m, m)
            C = C0.clone()
            h.set_path(gbgemm.PATH_AUTO)
            med, mn = _time_stats(lambda: h.sgemm("N", "N", m, m, nb, -1.0, A, m, B, nb, 1.0, C, m), stream, 10,
                                  flush if m < 8192 else None)
            C.copy_(C0)
            h.sgemm("N", "N", m, m, nb, -1.0, A, m, B, nb, 1.0, C, m)
            torch.cuda.synchronize()
            blk = [((0, m), (0, m))] if m <= 4096 else [((0, 1024), (0, 1024)), ((m - 1024, m), (m // 2, m // 2 + 1024))]
            err = max(h.check_error("N", "N", m, m, nb, -1.0, A, m, B, nb, 1.0, C0, C, m, rows=r, cols=c) for r, c in blk)
            fl = metrics.gemm_flops(m, m, nb)
            by = 8.0 * m * m + 4.0 * (2 * m) * nb
            gbs = by / (med * 1e-3) / 1e9
            lp[f"m{m}_nb{nb}"] = {"ms_median": med, "tflops": fl / (med * 1e-3) / 1e12, "hbm_gbs": gbs,
                                  "hbm_frac": gbs / hbm, "roofline_tflops": min(642.6, fl / by * hbm / 1e3),
                                  "max_error_ratio": err, "path": "split" if h.last_path() == 2 else "simt"}
            del A, B, C, C0
    out["linpack_updates"] = dict(lp, note=(f"bytes = 8 m n + 4 (m + n) nb; HBM peak {hbm:.0f} GB/s ({peak_src}); "
                                            "median of 10 calls; L2 flushed before each call for m = 4096"))
    # -- strided batch of the paper's micro-kernel problem (Table I: m 192, n 256,
    #    K 4096), 64 problems, NN, alpha 1, beta 0, uniform --
    mb, nbat, kb, batch = 192, 256, 4096, 64
    g.manual_seed(5)
    Ab = torch.rand(mb * kb * batch, device="cuda", generator=g) * 2 - 1
    Bb = torch.rand(kb * nbat * batch, device="cuda", generator=g) * 2 - 1
    Cb = torch.zeros(mb * nbat * batch, device="cuda")
    h.set_path(gbgemm.PATH_AUTO)
    run_b = lambda: h.sgemm_strided_batched("N", "N", mb, nbat, kb, 1.0, Ab, mb, mb * kb, Bb, kb, kb * nbat, 0.0,
                                            Cb, mb, mb * nbat, batch)
    med_b, min_b = _time_stats(run_b, stream, 10, flush)
    run_s = lambda: [h.sgemm("N", "N", mb, nbat, kb, 1.0, Ab[z * mb * kb:], mb, Bb[z * kb * nbat:], kb, 0.0,
                             Cb[z * mb * nbat:], mb) for z in range(batch)]
    med_s, _ = _time_stats(run_s, stream, 5, flush)
    run_b()
    torch.cuda.synchronize()
    errb = max(h.check_error("N", "N", mb, nbat, kb, 1.0, Ab[z * mb * kb:], mb, Bb[z * kb * nbat:], kb, 0.0,
                             Cb[z * mb * nbat:], Cb[z * mb * nbat:], mb) for z in (0, batch - 1))
    flb = batch * metrics.gemm_flops(mb, nbat, kb)
    out["batched_192x256x4096"] = {
        "batch": batch, "ms_median": med_b, "tflops": flb / (med_b * 1e-3) / 1e12,
        "tflops_best": flb / (min_b * 1e-3) / 1e12, "single_calls_ms": med_s,
        "single_calls_tflops": flb / (med_s * 1e-3) / 1e12, "max_error_ratio": errb,
        "path": "split" if h.last_path() == 2 else "simt",
        "note": ("the paper's micro-kernel problem (Table I, 192 x 256 x 4096), 64 at once through "
                 "gbgemm_sgemm_strided_batched; single_calls = the same 64 problems as gbgemm_sgemm calls; "
                 "error ratio on problems 0 and 63 (FP64 on the GPU)")}
    del Ab, Bb, Cb
    # -- split-K: a small output with a long k (512 x 512 x 65536, NN, alpha 1,
    #    beta 0): 4 tiles of 128 x 256 without slicing, sliced over the SMs --
    ms_, ns_, ks_ = 512, 512, 65536
    g.manual_seed(6)
    As_ = torch.rand(ms_ * ks_, device="cuda", generator=g) * 2 - 1
    Bs_ = torch.rand(ks_ * ns_, device="cuda", generator=g) * 2 - 1
    Cs_ = torch.zeros(ms_ * ns_, device="cuda")
    h.set_path(gbgemm.PATH_SPLIT_BF16)
    run_k = lambda: h.sgemm("N", "N", ms_, ns_, ks_, 1.0, As_, ms_, Bs_, ks_, 0.0, Cs_, ms_)
    med_k, min_k = _time_stats(run_k, stream, 10, flush)
    h.profile_begin()
    run_k()
    torch.cuda.synchronize()
    launches_k = h.profile_end()[2]
    errk = h.check_error("N", "N", ms_, ns_, ks_, 1.0, As_, ms_, Bs_, ks_, 0.0, Cs_, Cs_, ms_)
    flk = metrics.gemm_flops(ms_, ns_, ks_)
    out["splitk_512x512x65536"] = {
        "ms_median": med_k, "tflops": flk / (med_k * 1e-3) / 1e12, "tflops_best": flk / (min_k * 1e-3) / 1e12,
        "kernels_per_call": launches_k, "max_error_ratio": errk,
        "note": ("split path; the k range is cut into slices so that the 4-16 output tiles fill the SMs, "
                 "and a reduction sums the slices in order (kernels_per_call 3 = packing of both operands, "
                 "GEMM, reduction); error ratio over the whole 512 x 512 result (FP64 on the GPU)")}
    del As_, Bs_, Cs_
    # -- sgemv (Level 2, HBM-bound): A 32768 x 32768 (4.3 GB), both transposes --
    mv = 32768
    g.manual_seed(7)
    Av = torch.rand(mv * mv, device="cuda", generator=g) * 2 - 1
    xv = torch.rand(mv, device="cuda", generator=g) * 2 - 1
    yv = torch.rand(mv, device="cuda", generator=g) * 2 - 1
    gv = {}
    for tr in ("N", "T"):
        med_v, min_v = _time_stats(lambda: h.sgemv(tr, mv, mv, 1.0, Av, mv, xv, 1, 0.0, yv, 1), stream, 10)
        by = 4.0 * (mv * mv + 2 * mv)
        gv[tr] = {"ms_median": med_v, "gbs": by / (med_v * 1e-3) / 1e9, "hbm_frac": by / (med_v * 1e-3) / 1e9 / hbm,
                  "tflops": 2.0 * mv * mv / (med_v * 1e-3) / 1e12}
    out["sgemv_32768"] = dict(gv, note=(f"bytes = 4 (m n + m + n); HBM peak {hbm:.0f} GB/s ({peak_src}); A (4.3 GB) "
                                        "is larger than L2, so no flush; median of 10 calls"))
    del Av, xv, yv
    # -- HPL-shaped LU (Section IV-C, Table VII: N = 4608 on the Parallella,
    #    0.495 GFLOPS): sgetrf + sgetrs, uniform [-0.5, 0.5) matrix and right-hand
    #    side (seed 8), default block width; rate = (2/3 N^3 + 2 N^2) / time;
    #    HPL's scaled residual computed here in FP64 --
    hpl = {}
    for nh in (4608, 16384):
        g.manual_seed(8)
        A0h = torch.rand(nh * nh, device="cuda", generator=g) - 0.5
        b0h = torch.rand(nh, device="cuda", generator=g) - 0.5
        Ah, bh = A0h.clone(), b0h.clone()
        piv = torch.empty(nh, dtype=torch.int32, device="cuda")
        inf_ = torch.empty(1, dtype=torch.int32, device="cuda")
        times = []
        for it in range(4):
            Ah.copy_(A0h)
            bh.copy_(b0h)
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            h.sgetrf(nh, Ah, nh, piv, inf_)
            e1.record(stream)
            h.sgetrs(nh, 1, Ah, nh, piv, bh, nh)
            e2.record(stream)
            torch.cuda.synchronize()
            if it > 0:  # the first call allocates the workspace
                times.append((e0.elapsed_time(e2), e0.elapsed_time(e1)))
        t_all = sorted(times)[len(times) // 2]
        Ad = A0h.view(nh, nh).double().T  # column-major storage: A(i, j) = A0h[j * n + i]
        xd, bd = bh.double(), b0h.double()
        resid = ((Ad @ xd - bd).abs().max() /
                 (2.0 ** -24 * (Ad.abs().sum(1).max() * xd.abs().max() + bd.abs().max()) * nh)).item()
        flh = 2.0 / 3.0 * nh ** 3 + 2.0 * nh ** 2
        hpl[str(nh)] = {"ms": t_all[0], "getrf_ms": t_all[1], "getrs_ms": t_all[0] - t_all[1],
                        "tflops": flh / (t_all[0] * 1e-3) / 1e12, "info": int(inf_.item()),
                        "scaled_residual": resid, "passed": resid < 16.0}
        del A0h, b0h, Ah, bh, Ad, xd, bd
    out["hpl_lu"] = dict(hpl, note=("sgetrf + sgetrs (FP32, partial pivoting, library sgemm for the trailing "
                                    "updates), median of 3 calls after one warm-up; the paper's HPL run (N 4608, "
                                    "NB 768, FP64 API over an FP32 gemm) took 131.81 s, 0.495 GFLOPS, residual "
                                    "check passed at 16 with eps 2^-53; here eps = 2^-24"))
    del flush
    # -- grouped uneven batch: 4096 problems, m, n, k log-uniform in [16, 1024] (seed 3) --
    shapes = synth.grouped_shapes(3, 4096)
    bufs, probs = [], []
    fl_total = 0.0
    g.manual_seed(3)
    for (ta, tb, mm, nn, kk) in shapes:
        ar, ac = synth.op_shape(ta, mm, kk)
        br, bc = synth.op_shape(tb, kk, nn)
        Ag = torch.rand(ar * ac, device="cuda", generator=g) * 2 - 1
        Bg = torch.rand(br * bc, device="cuda", generator=g) * 2 - 1
        Cg = torch.empty(mm * nn, device="cuda")
        bufs.append((Ag, Bg, Cg))
        probs.append(gbgemm.problem(ta, tb, mm, nn, kk, 1.0, Ag, ar, Bg, br, 0.0, Cg, mm))
        fl_total += metrics.gemm_flops(mm, nn, kk)
    # The equivalent single-large-GEMM rate: the batch's FLOPs at the 4096^3 rate
    # of the path each problem is eligible for (split from k = 128, SIMT below),
    # as one harmonic mean; it does not depend on the configurations a plan picks.
    fl_split = sum(metrics.gemm_flops(mm, nn, kk) for (_, _, mm, nn, kk) in shapes if kk >= 128)
    fs = fl_split / fl_total
    equiv = 1.0 / (fs / rates["split"] + (1 - fs) / rates["simt"])
    # (Every problem of the batch has k >= 16 and runs on the split path; against
    # the 4096^3 split rate alone the bar is higher, reported as well.)
    # Sum of per-problem rooflines: each problem at the larger of its FLOPs at its
    # path's peak (BF16 dense / 3 from k = 128, FP32 SIMT below) and its
    # 4 (mk + kn + mn) bytes at the HBM rate.
    bf16_peak, _, hbm_gbs, _ = load_peaks()
    simt_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    roof_s = 0.0
    for (_, _, mm, nn, kk) in shapes:
        pk = bf16_peak / 3.0 if kk >= 128 else simt_peak
        roof_s += max(metrics.gemm_flops(mm, nn, kk) / (pk * 1e12), 4.0 * (mm * kk + kk * nn + mm * nn) / (hbm_gbs * 1e9))
    grouped = {}
    sources = [("default", gbgemm.CONFIG_DEFAULT)]
    weights = os.path.join(ROOT, "paper_1608_05265_gb300", "data", "predictor_gb300.bin")
    if os.path.exists(weights):
        from paper_1608_05265_gb300 import predictor
        h.predictor_set(predictor.load_weights(weights)[0])
        sources.append(("predicted", gbgemm.CONFIG_PREDICTED))
    sources.append(("tuned", gbgemm.CONFIG_TUNED))  # exhaustive tuner: seconds of plan time
    for name, src in sources:
        t0 = time.time()
        plan = gbgemm.GroupedPlan(h, probs, config_source=src)
        t_plan = time.time() - t0
        ms = _time(lambda: plan.run(stream), stream, 20)
        st = plan.stats()
        tf = fl_total / (ms * 1e-3) / 1e12
        grouped[name] = {"ms": ms, "tflops": tf, "plan_seconds": t_plan, "fraction_of_roofline_sum": roof_s * 1e3 / ms,
                         "plan_split_flop_share": st["flops_split"] / max(st["flops_split"] + st["flops_simt"], 1.0),
                         "fraction_of_equivalent": tf / equiv, "fraction_of_split_4096": tf / rates["split"],
                         "kernels_per_run": st["kernels_per_run"]}
        plan.close()
    out["grouped_4096"] = dict(grouped, problems=4096, flops=fl_total, split_eligible_flop_share=fs,
                               equivalent_single_gemm_tflops=equiv, roofline_sum_ms=roof_s * 1e3,
                               split_4096_tflops=rates["split"],
                               note=("equivalent rate = harmonic mean of the 4096^3 split and SIMT rates, weighted by "
                                     "the FLOPs of problems with k >= 128 (split-eligible) and k < 128"))
    assert h.get_device_status() == 0
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-blocks", type=int, default=3, help="oracle blocks timed for cpu_baseline (0: skip)")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the Linpack-shaped, grouped and 4096^3 measurements")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
