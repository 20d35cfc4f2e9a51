#!/usr/bin/env python
"""Benchmark of the matrix-free H x on GB300.

One step = one pass of the hot path: y = H x for the Tavis-Cummings model of
24 spin-1/2 sites and one boson mode truncated at 64 levels (boson last,
D = 2^24 * 64 = 1,073,741,824 states), FP64 storage, one right-hand side,
inputs resident in HBM. x and y (17.2 GB) exceed the 129 MB L2 many times
over, so no flush is needed between steps.

Prints ONE JSON line (rank 0). Extra keys report the other forms of the path
against this plain FP64 kernel: FP32 storage on the same model, the
ferrimagnetic chain of 6.05e7 states, 200-step Lanczos on the 1.07e9-state
model in FP32 and FP64 storage against its exact ground-state energy, the
batched persistent launch, the adjoint, the paper's Table I models, a
fixed-magnetization sector beside the full basis, time evolution and a
complex H.

--impl reference times the CPU oracle (the reference arm of this build) on
a bounded sample of the same workload, on the host cores.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·x Gstates/s & HBM GB/s vs peak; batched/FP32/adjoint vs plain FP64"
WORKLOAD = "tavis_cummings_n24_l64"
WORKLOAD_DESC = ("Tavis-Cummings: 24 spin-1/2 sites + one boson mode truncated at 64 levels, boson last "
                 "(D=2^24*64=1073741824); H = omega a^dag a + omega0 sum Sz_i + sum g_i (a^dag S-_i + a S+_i), "
                 "omega=omega0=1, g_i~U[0.05,0.15] (seed 7)")
# ground-state energy of the headline model: the vacuum |n=0, all spins down>
# is annihilated by every coupling term, and with sqrt(sum g_i^2) ~ 0.5 < 1 no
# excitation sector lies below it, so E0 = -omega0 * 24 / 2
HEADLINE_E0 = -12.0


def headline_model():
    import workloads as W
    return W.tavis_cummings(24, 64, seed=7)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-variants", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--profile", action="store_true",
                    help="only warm-up + timed applies of --workload/--dtype (for ncu); prints one timing line")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(PROFILE_WORKLOADS))
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "tile", "general", "staged"],
                    help="--profile only: force one apply kernel (auto: library or tuned choice)")
    ap.add_argument("--apply-ex", default=None,
                    help="--profile only: JSON keyword arguments of Hamiltonian.apply_ex for every timed "
                         "apply, e.g. '{\"kernel\": \"general\", \"prefetch\": true, \"s\": 8}'")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="use the library's default launch shape instead of autotuning it first")
    return ap.parse_args()


def _ring_sector(n):
    """Periodic spin-1/2 Heisenberg chain of n sites restricted to M = 0 (the
    fixed digit-sum sector with total n / 2)."""
    import workloads as W
    terms = []
    for i in range(n):
        j = (i + 1) % n
        terms += [(i, "Sp", j, "Sm", 0.5), (i, "Sm", j, "Sp", 0.5), (i, "Sz", j, "Sz", 1.0)]
    return W.Model(f"sector_chain_n{n}_m0", [("spin", 2)] * n, terms, {"sector_total": n // 2})


def _workload(name):
    import workloads as W
    if name.startswith("sector_chain_n"):
        return _ring_sector(int(name[len("sector_chain_n"):].split("_")[0]))
    return {
        "ferrimagnet_chain_n20": lambda: W.ferrimagnet_chain(20),
        "tavis_cummings_n20_l64": lambda: W.tavis_cummings(20, 64, seed=7),
        "tavis_cummings_n24_l64": lambda: W.tavis_cummings(24, 64, seed=7),
        "square_lattice_4x5": lambda: W.square_lattice_xxz(4, 5, seed=4),
        "heisenberg_ring_n12": lambda: W.heisenberg_ring(12),
    }[name]()


PROFILE_WORKLOADS = {"ferrimagnet_chain_n20", "tavis_cummings_n20_l64", "tavis_cummings_n24_l64",
                     "square_lattice_4x5", "heisenberg_ring_n12", "sector_chain_n26_m0", "sector_chain_n30_m0"}


def run_profile(args):
    """Kernel-only run for profilers: the applies of one workload, nothing else."""
    import torch

    import workloads as W
    from paper_2606_02169_gb300 import Hamiltonian
    m = _workload(args.workload)
    total = m.meta.get("sector_total")
    h = Hamiltonian(m.sites, m.terms, sector_total=total)
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    fixed = json.loads(args.apply_ex) if args.apply_ex else None
    cfg = h.tune(1, dt) if args.tune and args.kernel == "auto" and total is None and fixed is None else None
    x = W.torch_vector(h.D, 3, dtype=dt)
    y = torch.empty_like(x)
    if fixed is not None:
        def step():
            h.apply_ex(x, out=y, **fixed)
    elif args.kernel == "auto":
        def step():
            h.apply(x, out=y)
    else:
        def step():
            h.apply_ex(x, out=y, kernel=args.kernel)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the timed applies sit in an NVTX range "timed", so that a profiler can
    # select them (ncu --nvtx --nvtx-include "timed/") past the tuner's launches
    nvtx = getattr(torch.cuda, "nvtx", None)
    try:
        nvtx.range_push("timed")
    except Exception:
        nvtx = None
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    if nvtx is not None:
        nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    print(json.dumps({"profile": args.workload, "dtype": args.dtype, "kernel": fixed or args.kernel, "D": h.D,
                      "ms_per_apply": ms, "gstates_s": h.D / ms / 1e6, "tuned": cfg}))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    # the device code of the general apply kernel (its body, arithmetic
    # policies, launch shapes and the units that instantiate its scalar
    # variants); a change to how the plan builder derives its tables needs
    # the records taken again as well
    for f in ("apply_kernel.cuh", "apply_launch.cuh", "device_common.cuh", "apply_df64.cu", "apply_f32.cu",
              "apply_pf_df64.cu", "apply_pf_f32.cu", "apply_vi_df64.cu", "apply_vi_f32.cu", "apply_pf_vi_df64.cu",
              "apply_pf_vi_f32.cu"):
        with open(os.path.join(ROOT, "paper_2606_02169_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_profile(key, launch=None):
    """The committed ncu record of one apply (DRAM bytes, thread instructions
    per launch), or None if the kernel sources changed since it was taken or
    it was taken on another launch variant than `launch` (a tuned_config)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        rec = t.get(key)
        if rec and launch is not None and rec.get("launch"):
            if any(int(launch.get(k, 0)) != int(v) for k, v in rec["launch"].items()):
                return None
        if rec and rec.get("source_hash") == kernel_source_hash():
            return rec
    except Exception:
        pass
    return None


def recorded_traffic(key, launch=None):
    rec = recorded_profile(key, launch)
    return rec["dram_bytes_per_launch"] if rec else None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # nvidia-smi's start-up can stall kernel submission: time only
            # after it has produced samples
            t0 = time.time()
            while time.time() - t0 < 15:
                with open(self.path) as f:
                    if sum(1 for _ in f) >= 3:
                        break
                time.sleep(0.05)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [v.strip() for v in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx.append(float(c[2]))
                    pw.append(float(c[3]))
                except ValueError:
                    continue
                for n, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons)}


def dist():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as td
        torch.cuda.set_device(local)
        td.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as td
        td.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    from paper_2606_02169_gb300 import shard
    return shard.max_over_ranks(v, device="cuda")


def timed(fn, steps, warmup, ws, stream):
    """Total ms of `steps` calls of fn, CUDA events on the launching stream,
    barrier + synchronize on both sides, max over ranks."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    return max_over_ranks(e0.elapsed_time(e1), ws)


def e2e_pipelined(h, x, s_c, steps, ws, warmup=3):
    """Total ms of `steps` end-to-end applies through the public API with x
    and y in pinned host memory: each hm_apply reads its x from host memory
    (the FP64 split pass) and writes y to host memory (the apply kernel) over
    the CPU-GPU link. Consecutive steps alternate between two streams and two
    host y buffers, so one step's read of x overlaps the previous step's
    apply; barrier + synchronize on both sides, max over ranks."""
    import torch
    xh = torch.empty(x.numel(), dtype=x.dtype, pin_memory=True)
    xh.copy_(x.cpu())
    yh = [torch.empty(x.numel(), dtype=x.dtype, pin_memory=True) for _ in range(2)]
    ss = [s_c, torch.cuda.Stream()]

    def run(k):
        for i in range(k):
            h.apply(xh, out=yh[i & 1], stream=ss[i & 1])

    run(warmup)
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ss[0])
    ss[1].wait_event(e0)
    run(steps)
    ss[0].wait_stream(ss[1])
    e1.record(ss[0])
    torch.cuda.synchronize()
    barrier(ws)
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    # the last host result equals a plain device apply of the same x
    if not torch.equal(yh[(steps - 1) & 1].to(x.device), h.apply(x)):
        raise RuntimeError("end-to-end result in host memory differs from hm_apply on device vectors")
    return ms


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): bounded row samples
# ---------------------------------------------------------------------------

def oracle_input(D):
    """The oracle's x for a timing sample: seeded uniform values (its cost
    does not depend on them; a cheaper draw than normals for 2^30 states)."""
    import numpy as np
    return np.random.default_rng(3).random(D) - 0.5


def oracle_rate(model, seconds, threads=0, x=None):
    """CPU oracle on a contiguous sample of target rows sized to take about
    `seconds`; returns (Gstates/s, rows, seconds taken, threads)."""
    import oracle
    D = oracle.dimension(model.sites)
    if x is None:
        x = oracle_input(D)
    oracle.build()
    nthreads = threads or len(os.sched_getaffinity(0))
    r0 = 20000 if nthreads > 1 else 4000
    t0 = time.perf_counter()
    oracle.apply(model.sites, model.terms, x, row_begin=0, row_end=r0, nthreads=nthreads)
    dt = max(time.perf_counter() - t0, 1e-4)
    rows = int(min(D, max(r0, r0 * seconds / dt)))
    start = (D - rows) // 2
    t0 = time.perf_counter()
    oracle.apply(model.sites, model.terms, x, row_begin=start, row_end=start + rows, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return rows / dt / 1e9, rows, dt, nthreads


def run_reference(args):
    """The oracle as it stands, on the host cores, each step a bounded row
    sample of the headline workload; times what it actually ran."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    m = headline_model()
    D = oracle.dimension(m.sites)
    x = oracle_input(D)
    oracle.build()
    nthreads = len(os.sched_getaffinity(0))
    budget = 120.0 / max(1, args.steps + args.warmup)    # whole run within a few minutes
    t0 = time.perf_counter()
    oracle.apply(m.sites, m.terms, x, row_begin=0, row_end=20000, nthreads=nthreads)
    dt = max(time.perf_counter() - t0, 1e-4)
    rows = int(min(D, max(20000, 20000 * min(budget, 5.0) / dt)))
    start = (D - rows) // 2
    for _ in range(args.warmup):
        oracle.apply(m.sites, m.terms, x, row_begin=start, row_end=start + rows, nthreads=nthreads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.apply(m.sites, m.terms, x, row_begin=start, row_end=start + rows, nthreads=nthreads)
    dt = time.perf_counter() - t0
    val = rows * args.steps / dt / 1e9
    sample = (f"rows [{start}, {start + rows}) of {D} per step ({rows / D:.4%} of one H x), "
              f"C oracle with OpenMP on {nthreads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Gstates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "D": D, "nvec": 1,
                                        "rows_per_step": rows},
        "cpu_baseline": {"value": val, "unit": "Gstates/s", "cores": nthreads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "Gstates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

KERNEL_NAMES = {0: "general", 1: "general", 2: "tile", 3: "staged"}


def split_pairs(x):
    """(hi, lo) float pairs of an FP64 tensor, interleaved: the input of the
    kernel-only measurement (built with torch outside any timed region)."""
    import torch
    hi = x.float()
    lo = (x - hi.double()).float()
    return torch.stack((hi, lo), dim=-1).reshape(-1)


def kernel_only_ms(h, x, y, cfg, steps, stream):
    """Average ms of the FP64 apply kernel alone: pre-split input (no split
    pass, no range check), the launch choice cfg (a tuned_config dict or
    None), CUDA events on its stream."""
    cfg = cfg or {}
    kernel = KERNEL_NAMES[cfg.get("kernel", 0)]
    kw = dict(kernel=kernel, ctas=cfg.get("ctas", 0))
    if kernel != "staged":
        kw.update(s=cfg.get("s", 0), mb=bool(cfg.get("mb", 0)))
    if kernel == "general":
        kw.update(small=bool(cfg.get("small", 0)), prefetch=bool(cfg.get("prefetch", 0)),
                  scalar=bool(cfg.get("scalar", 0)), split=bool(cfg.get("split", 0)),
                  split_sites=cfg.get("split_sites", 0), vinv=bool(cfg.get("vinv", 0)))
    xs = split_pairs(x)
    ms = timed(lambda: h.apply_ex(xs, out=y, presplit=True, **kw), steps, 3, 1, stream) / steps
    del xs
    return ms


def run_ours(args):
    import torch

    import workloads as W
    from paper_2606_02169_gb300 import Hamiltonian

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    hbm, peak_kind = peaks()

    m = headline_model()
    h = Hamiltonian(m.sites, m.terms)
    D = h.D
    # launch-shape autotuning is set-up, outside the timed region
    tuned = h.tune(1, torch.float64) if args.tune else None
    kernel = KERNEL_NAMES[(tuned or {}).get("kernel", 0)]
    x = W.torch_vector(D, 8 + rank, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)

    clocks = Clocks(local)
    for _ in range(args.warmup):
        h.apply(x, out=y)
    torch.cuda.synchronize()
    clocks.start()
    # the timed applies sit in an NVTX range "timed" (a profiler's launch
    # list can select exactly them: ncu --nvtx --nvtx-include "timed/")
    nvtx = getattr(torch.cuda, "nvtx", None)
    try:
        nvtx.range_push("timed")
    except Exception:  # noqa: BLE001
        nvtx = None
    ms = timed(lambda: h.apply(x, out=y), args.steps, 0, ws, stream)
    if nvtx is not None:
        nvtx.range_pop()
    clk = clocks.stop()
    ms_step = ms / args.steps
    value = ws * D / (ms_step * 1e-3) / 1e9
    bytes_alg = 16.0 * D
    # the dominant kernel alone: the double-float apply on pre-split input
    ms_kernel = kernel_only_ms(h, x, y, tuned, max(5, min(args.steps, 50)), stream)
    achieved = bytes_alg / (ms_kernel * 1e-3) / 1e9
    traffic = recorded_traffic("apply_f64_" + WORKLOAD, tuned)

    # end to end through the public API, run the way a caller streaming vectors
    # through the GPU would: every step copies its x from pinned host memory
    # and its y back to pinned host memory; copy-in, apply and copy-out use
    # three streams and two device buffers each, ordered by events, so one
    # step's copies overlap the neighbouring steps' work
    k_e2e = max(3, min(args.steps, 20))
    ms_e2e = e2e_pipelined(h, x, stream, k_e2e, ws)
    e2e_val = ws * D / (ms_e2e / k_e2e * 1e-3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": "Gstates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "D": D, "nvec": 1,
                   "l2": "inputs larger than L2 (x+y = 17.2 GB per step), no flush",
                   "parallelism": "replicas" if ws > 1 else "single GPU", "tuned_launch": tuned},
        "e2e": {"value": e2e_val, "unit": "Gstates/s", "h2d_bytes_per_step": 8 * D,
                "d2h_bytes_per_step": 8 * D, "steps": k_e2e,
                "how": "hm_apply on x and y in pinned host memory every step (the library reads x and "
                       "writes y over the CPU-GPU link inside the call); consecutive steps on two streams "
                       "overlap"},
        # per FP64 step: k_split_f64 (split + range check), the double-float
        # apply, and the native FP64 fallback launch that returns at once
        # unless the split flagged x
        "gpu_launches": 3 * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": f"{kernel} double-float apply kernel alone (pre-split input), "
                               f"{ms_kernel:.3f} ms per launch",
                     "algorithmic_bytes_per_launch": bytes_alg, "algorithmic_bytes_per_state": 16,
                     "step_frac": bytes_alg / (ms_step * 1e-3) / 1e9 / hbm,
                     "step": "one FP64 apply = split pass + apply kernel + gated fallback launch"},
        "clocks": clk,
    }
    # issue / FP32-pipe view of the same kernel: thread instructions per state
    # (ncu) times the measured rate, against 4 schedulers x 32 lanes per SM at
    # the sampled clock
    rec = recorded_profile("apply_f64_" + WORKLOAD, tuned)
    if rec and rec.get("thread_inst_per_launch"):
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        rate = D / (ms_kernel * 1e-3)
        peak_i = sms * 4 * 32 * mhz * 1e6
        ipk = rec["thread_inst_per_launch"] / D
        line["roofline"]["issue"] = {"thread_inst_per_state": ipk, "achieved_tinst_per_s": ipk * rate,
                                     "peak_tinst_per_s": peak_i, "frac": ipk * rate / peak_i}
        if rec.get("fp32_ops_per_launch"):
            fpk = rec["fp32_ops_per_launch"] / D
            line["roofline"]["alu"] = {"fp32_lane_ops_per_state": fpk, "achieved_ops_per_s": fpk * rate,
                                       "peak_ops_per_s": peak_i, "frac": fpk * rate / peak_i,
                                       "note": "double-float arithmetic runs on the FP32 pipe"}

    if rank == 0 and ws == 1 and not args.skip_variants:
        # the extra rows never cost the headline line: a failing one is recorded
        try:
            line["variants"] = variants(args, h, m, x, y, ms_step, stream, hbm)
        except Exception as e:  # noqa: BLE001
            line["variants"] = {"error": f"{type(e).__name__}: {e}"[:300]}
            try:
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
            except Exception:  # noqa: BLE001
                pass

    if rank == 0:
        del x, y
        torch.cuda.empty_cache()
        xo = oracle_input(D)
        rate, rows, dt, nth = oracle_rate(m, args.cpu_seconds, x=xo)
        rate1, rows1, dt1, _ = oracle_rate(m, args.cpu_seconds / 2, threads=1, x=xo)
        del xo
        line["cpu_baseline"] = {"value": rate, "unit": "Gstates/s", "cores": nth, "kind": "oracle",
                                "sample": f"{rows} contiguous target rows of {D} ({dt:.1f} s, "
                                          f"C oracle with OpenMP on {nth} threads)",
                                "one_thread": {"value": rate1, "rows": rows1, "seconds": dt1}}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as td
        td.destroy_process_group()


def variants(args, h, m, x, y, ms_f64, stream, hbm):
    import numpy as np
    import torch

    import workloads as W
    from paper_2606_02169_gb300 import Batch, Hamiltonian
    out = {}
    steps = max(20, min(args.steps, 200))
    D = h.D

    # FP32 storage on the same workload (no split pass: the step is the kernel)
    tuned32 = h.tune(1, torch.float32) if args.tune else None
    xf = x.float()
    yf = torch.empty_like(xf)
    k = max(10, min(args.steps, 50))
    ms = timed(lambda: h.apply(xf, out=yf), k, 3, 1, stream) / k
    out["fp32_storage_tc_1e9"] = {"gstates_s": D / ms / 1e6, "ms": ms, "speedup_vs_f64": ms_f64 / ms,
                                  "hbm_frac_algorithmic": 8 * D / ms / 1e6 / hbm, "tuned_launch": tuned32}
    del xf, yf
    torch.cuda.empty_cache()
    # native FP64 arithmetic on the same workload (the kernel the double-float
    # policy replaces; GB300's FP64 pipe is ~1/70 of its FP32 pipe)
    k = 5
    ms = timed(lambda: h.apply_ex(x, out=y, native_f64=True, kernel="staged"), k, 2, 1, stream) / k
    out["native_fp64_arith_tc_1e9"] = {"gstates_s": D / ms / 1e6, "ms": ms, "slowdown_vs_df64": ms / ms_f64}

    # 200-step Lanczos on the 1.07e9-state model, FP64 and FP32 storage, same
    # v0; the ground-state energy is known exactly (HEADLINE_E0)
    v0 = W.torch_vector(D, 11, dtype=torch.float64)
    res = {}
    for name, v in (("f64", v0), ("f32", None)):
        vv = v if v is not None else v0.float()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = h.lanczos(vv, 200)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name] = (r, dt)
        del vv
        torch.cuda.empty_cache()
    del v0
    torch.cuda.empty_cache()
    out["lanczos_200_tc_1e9"] = {
        "e0_exact": HEADLINE_E0,
        "e0_f64": res["f64"][0]["e0"], "e0_f32": res["f32"][0]["e0"],
        "abs_dE0_f64_vs_exact": abs(res["f64"][0]["e0"] - HEADLINE_E0),
        "abs_dE0_f32_vs_exact": abs(res["f32"][0]["e0"] - HEADLINE_E0),
        "abs_dE0_f32_vs_f64": abs(res["f32"][0]["e0"] - res["f64"][0]["e0"]),
        "ms_per_step_f64": res["f64"][1] * 1e3 / max(1, res["f64"][0]["steps"]),
        "ms_per_step_f32": res["f32"][1] * 1e3 / max(1, res["f32"][0]["steps"]),
        "steps": [res["f64"][0]["steps"], res["f32"][0]["steps"]], "reorth": "none",
        "timing": "wall clock of one hm_lanczos call (vector allocation included)"}

    # the mixed-spin ferrimagnetic chain N = 20 (D = 6.05e7), FP64 and FP32
    mf = W.ferrimagnet_chain(20)
    hf = Hamiltonian(mf.sites, mf.terms)
    Df = hf.D
    for name, dt, esz in (("ferrimagnet_chain_n20_f64", torch.float64, 8),
                          ("ferrimagnet_chain_n20_f32", torch.float32, 4)):
        tc = hf.tune(1, dt) if args.tune else None
        xt = W.torch_vector(Df, 3, dtype=dt)
        yt = torch.empty_like(xt)
        k = 50
        ms = timed(lambda: hf.apply(xt, out=yt), k, 5, 1, stream) / k
        entry = {"gstates_s": Df / ms / 1e6, "ms": ms, "hbm_frac_algorithmic": 2 * esz * Df / ms / 1e6 / hbm,
                 "tuned_launch": tc}
        if dt == torch.float64:
            mk = kernel_only_ms(hf, xt, yt, tc, k, stream)
            entry.update({"ms_kernel": mk, "hbm_frac_kernel": 16 * Df / mk / 1e6 / hbm})
        out[name] = entry
        del xt, yt
        torch.cuda.empty_cache()
    del hf

    # batched disorder ensemble: 256 XXZ spin-1 chains N in 8..14, 16 RHS, FP32
    models = W.disorder_ensemble(256, 8, 14, 1000)
    hams = [Hamiltonian(mm.sites, mm.terms) for mm in models]
    nvec = 16
    if args.tune:   # members that fill the GPU alone take their tuned launch (one tune per chain length)
        for hh in hams:
            hh.tune(nvec, torch.float32)
    xs = [W.torch_vector(hh.D * nvec, 1000 + i, dtype=torch.float32, normalize=False) for i, hh in enumerate(hams)]
    ys = [torch.empty_like(t) for t in xs]
    total = sum(hh.D for hh in hams) * nvec
    b = Batch(hams)
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        b.apply(xs, ys, stream=s2)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s2):
        b.apply(xs, ys, stream=s2)
    k = 5
    ms_b = timed(lambda: g.replay(), k, 1, 1, stream) / k

    def plain():
        for hh, xx, yy in zip(hams, xs, ys):
            hh.apply(xx, out=yy)

    ms_p = timed(plain, k, 1, 1, stream) / k
    out["batched_256_chains_16rhs_f32"] = {
        "states_x_rhs": total, "gstates_s_batched_graph": total / ms_b / 1e6,
        "gstates_s_per_instance_launches": total / ms_p / 1e6, "speedup": ms_p / ms_b,
        "hbm_frac_batched": 8 * total / ms_b / 1e6 / hbm}
    del xs, ys, b, hams, g
    torch.cuda.empty_cache()

    # the paper's Table I models (Sec. V testbeds C1, C2), FP64, one apply =
    # one matvec; the paper's matrix-free CPU rates (unstated CPU) as context
    for name, mk, paper in (("paper_c1_f64", W.paper_c1_chain, 6.137), ("paper_c2_f64", W.paper_c2_chain, 0.04387)):
        mc = mk()
        hc = Hamiltonian(mc.sites, mc.terms)
        if args.tune:
            hc.tune(1, torch.float64)
        xc = W.torch_vector(hc.D, 12, dtype=torch.float64)
        yc = torch.empty_like(xc)
        k = 20
        ms = timed(lambda: hc.apply(xc, out=yc), k, 3, 1, stream) / k
        out[name] = {"D": hc.D, "matvec_per_s": 1e3 / ms, "gstates_s": hc.D / ms / 1e6,
                     "paper_matrix_free_cpu_matvec_per_s": paper,
                     "note": "paper figure: Table I, CPU unstated; context only"}
        del hc, xc, yc
        torch.cuda.empty_cache()

    # fixed-magnetization sector (packed basis, combinatorial lookup): the
    # periodic Heisenberg chain N=30, M=0 (C(30,15) = 1.55e8 of 2^30 states),
    # FP64, beside the full-basis apply of the same chain and the sector
    # oracle's case-2 restatement on a bounded sample of rows
    ns = 30
    ss = [("spin", 2)] * ns
    st = []
    for i in range(ns):
        j = (i + 1) % ns
        st += [(i, "Sp", j, "Sm", 0.5), (i, "Sm", j, "Sp", 0.5), (i, "Sz", j, "Sz", 1.0)]
    hs = Hamiltonian(ss, st, sector_total=ns // 2)
    xs_ = W.torch_vector(hs.D, 21, dtype=torch.float64)
    ys_ = torch.empty_like(xs_)
    k = 5
    ms_s = timed(lambda: hs.apply(xs_, out=ys_), k, 2, 1, stream) / k          # block form
    ms_r = timed(lambda: hs.apply_ex(xs_, out=ys_, kernel="rows"), k, 2, 1, stream) / k   # per-row kernel
    import oracle
    rows = np.arange(2000) * (hs.D // 2000)
    xh = xs_.cpu().numpy()
    t0 = time.perf_counter()
    oracle.sector_rows(ss, st, ns // 2, xh, rows)
    t_or = time.perf_counter() - t0
    del hs, xs_, ys_
    torch.cuda.empty_cache()
    hf = Hamiltonian(ss, st)
    if args.tune:
        hf.tune(1, torch.float64)
    xf_ = W.torch_vector(hf.D, 22, dtype=torch.float64)
    yf_ = torch.empty_like(xf_)
    ms_f = timed(lambda: hf.apply(xf_, out=yf_), k, 2, 1, stream) / k
    out["sector_chain_n30_m0_f64"] = {
        "Dsec": math.comb(ns, ns // 2), "ms": ms_s, "gstates_s": math.comb(ns, ns // 2) / ms_s / 1e6,
        "ms_per_row_kernel": ms_r,
        "hbm_frac_algorithmic": 16 * math.comb(ns, ns // 2) / ms_s / 1e6 / hbm,
        "full_basis_ms": ms_f, "full_basis_gstates_s": hf.D / ms_f / 1e6,
        "vector_bytes_sector_vs_full": math.comb(ns, ns // 2) / hf.D,
        "cpu_oracle_rows_per_s": rows.size / t_or, "cpu_oracle_sample": f"{rows.size} rows, Python case-2 restatement"}
    del hf, xf_, yf_
    torch.cuda.empty_cache()

    # adjoint on the 4x5 lattice (D = 2^20, FP64): H^T gy + 113 coupling gradients
    ml = W.square_lattice_xxz(4, 5, seed=4)
    hl = Hamiltonian(ml.sites, ml.terms)
    xl = W.torch_vector(hl.D, 5, dtype=torch.float64)
    gl = W.torch_vector(hl.D, 6, dtype=torch.float64)
    yl = torch.empty_like(xl)
    gx = torch.empty_like(xl)
    gc = torch.empty(hl.nterms, dtype=torch.float64, device="cuda")
    k = 50
    ms_fwd = timed(lambda: hl.apply(xl, out=yl), k, 5, 1, stream) / k
    ms_adj = timed(lambda: hl.adjoint(gl, xl, gx=gx, gcoef=gc), k, 5, 1, stream) / k
    ms_grad = timed(lambda: hl.adjoint(gl, xl, want_gx=False, gcoef=gc), k, 5, 1, stream) / k
    out["adjoint_4x5_f64"] = {"ms_forward": ms_fwd, "ms_adjoint_gx_and_gcoef": ms_adj,
                              "ms_gcoef_only": ms_grad, "adjoint_over_forward": ms_adj / ms_fwd,
                              "nterms": hl.nterms}
    del hl, xl, gl, yl, gx, gc
    torch.cuda.empty_cache()

    # time evolution exp(-i t H) x of a complex128 vector on the ferrimagnetic
    # chain N = 20: one short-iterative Lanczos step of m = 30 Krylov vectors
    # (basis stored, and rebuilt by a second pass), beside the complex apply
    mf = W.ferrimagnet_chain(20)
    he = Hamiltonian(mf.sites, mf.terms)
    De = he.D
    xc = torch.complex(W.torch_vector(De, 3, dtype=torch.float64), W.torch_vector(De, 23, dtype=torch.float64))
    xc = xc / torch.linalg.vector_norm(xc)
    yc = torch.empty_like(xc)
    if args.tune:
        he.tune(1, torch.complex128)
    k = 10
    ms_capply = timed(lambda: he.apply(xc, out=yc), k, 3, 1, stream) / k
    mk, te = 30, 0.5

    def evolve_ms(recompute):
        he.evolve(xc, te, m=mk, out=yc, recompute=recompute)     # warm-up (allocations)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, est = he.evolve(xc, te, m=mk, out=yc, recompute=recompute)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3, est

    ms_ev, est = evolve_ms(False)
    drift = abs(float(torch.linalg.vector_norm(yc)) - 1.0)
    ms_ev2, _ = evolve_ms(True)
    out["evolve_ferrimagnet_chain_n20_c128"] = {
        "D": De, "t": te, "krylov_m": mk, "ms_per_step_stored_basis": ms_ev, "ms_per_step_rebuilt_basis": ms_ev2,
        "ms_complex_apply": ms_capply, "complex_gstates_s": De / ms_capply / 1e6,
        "apply_share_stored": mk * ms_capply / ms_ev, "error_estimate": est, "norm_drift": drift}
    del xc, yc, he
    torch.cuda.empty_cache()

    # complex H: periodic spin-1/2 chain N = 26 with a Dzyaloshinskii-Moriya
    # term and a transverse Sy field (imaginary elements), complex128,
    # beside the same chain without the imaginary terms (real H, complex x)
    nd = 26
    sd = [("spin", 2)] * nd
    real_t, cx_t = [], []
    for i in range(nd):
        j = (i + 1) % nd
        a, b = min(i, j), max(i, j)
        real_t += [(a, "Sx", b, "Sx", 1.0), (a, "Sy", b, "Sy", 1.0), (a, "Sz", b, "Sz", 0.8)]
        cx_t += [(a, "Sx", b, "Sy", 0.3), (a, "Sy", b, "Sx", -0.3), (i, "Sy", -1, "I", 0.2)]
    res = {}
    for name, terms in (("complex_h", real_t + cx_t), ("real_h", real_t)):
        hd = Hamiltonian(sd, terms)
        if args.tune:
            hd.tune(1, torch.complex128)
        xd = torch.complex(W.torch_vector(hd.D, 24, dtype=torch.float64), W.torch_vector(hd.D, 25, dtype=torch.float64))
        yd = torch.empty_like(xd)
        k = 10
        res[name] = timed(lambda: hd.apply(xd, out=yd), k, 3, 1, stream) / k
        if name == "complex_h":
            # the one-pass complex kernel and the two real passes (one
            # column per lane) with their combine, each as an explicit choice
            res["one_pass"] = timed(lambda: hd.apply_ex(xd, out=yd), k, 3, 1, stream) / k
            res["two_pass"] = timed(lambda: hd.apply_ex(xd, out=yd, scalar=True), k, 3, 1, stream) / k
        del hd, xd, yd
        torch.cuda.empty_cache()
    out["complex_h_dm_chain_n26_c128"] = {
        "D": 2 ** nd, "ms_complex_h": res["complex_h"], "gstates_s_complex_h": 2 ** nd / res["complex_h"] / 1e6,
        "hbm_frac_algorithmic": 32 * 2 ** nd / res["complex_h"] / 1e6 / hbm,
        "ms_one_pass_kernel": res["one_pass"], "ms_two_passes_and_combine": res["two_pass"],
        "ms_real_h_complex_x": res["real_h"], "complex_h_over_real_h": res["complex_h"] / res["real_h"]}
    return out


def main():
    args = parse()
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
