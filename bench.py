#!/usr/bin/env python
"""Throughput benchmark: EOM-CCSD Jacobian transformations per second.

Workload: the thymine/aug-cc-pVDZ-shaped synthetic Hamiltonian (o=33, v=228,
naux=900; seeded generator in paper_2301_13264_gb300.synth).  A step is one
right (A X) and one left (X^T A) block transformation of `nvec` trial vectors
at the converged ground-state amplitudes, i.e. 2*nvec Jacobian transforms.

Prints one JSON line (rank 0).  For --gpus N > 1 (torchrun) each rank runs an
independent replica on its own GPU (the path has no exchange step); the value
is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Jacobian transforms/s and time-to-converged coupling at o=33,v=228 vs FP64 GPU form"
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12
# DRAM bytes (read + write) of one ladder contraction (its + and - GEMM launches) from an
# ncu capture of the current kernel (profiles/k_tc_gemm_ladder_thymine_adz.md), keyed by
# (workload, nvec, products); a missing entry reports null (retaken whenever the kernel changes)
LADDER_TRAFFIC = {("thymine_adz", 8, 6): (54.516 + 0.948 + 50.029 + 0.944) * 1e9}
UNIT = "transforms/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="thymine_adz")
    ap.add_argument("--nvec", type=int, default=8)
    ap.add_argument("--precision", choices=["mixed", "fp64", "fp64tc"], default="mixed")
    ap.add_argument("--splits", type=int, default=3)
    ap.add_argument("--amplitudes", choices=["solve", "synthetic"], default="solve",
                    help="converge the ground state in set-up, or use seeded synthetic amplitudes")
    ap.add_argument("--ttc", default=None,
                    help="instead of transform throughput, time create -> ground -> EOM (2 roots) -> couplings "
                         "for the comma-separated forms among mixed, fp64, fp64tc ('both' = mixed,fp64)")
    ap.add_argument("--tol-eom", type=float, default=1e-8, help="--ttc: EOM residual-norm threshold")
    ap.add_argument("--max-sub", type=int, default=48, help="--ttc: Davidson subspace size before a restart")
    ap.add_argument("--tc-min-flops", type=float, default=None,
                    help="--ttc: smallest contraction (flops) run on the tensor cores (library default 1e8)")
    ap.add_argument("--ttc-profile", action="store_true",
                    help="--ttc: add the GEMM device time per arithmetic form (events around every GEMM)")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of the single-system bench, time batched transforms of this many small systems")
    ap.add_argument("--no-autotune", action="store_true", help="batch mode: tile widths from the output width")
    ap.add_argument("--mlp", action="store_true", help="instead, time the learned-guess kernels at the workload size")
    ap.add_argument("--batch-eom", type=int, default=0,
                    help="with --batch: time the batched right EOM solve for this many roots instead")
    ap.add_argument("--guess-eval", action="store_true",
                    help="instead, train the learned starts on smaller systems and compare iterations at the workload")
    ap.add_argument("--guess-train", type=int, default=40, help="--guess-eval: number of training systems")
    ap.add_argument("--guess-scale", type=float, default=4.0, help="--guess-eval: size reduction of the training systems")
    ap.add_argument("--contractions", default=None,
                    help="write a per-contraction table (markdown) of the timed steps to this file")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ttc", action="store_true", help="skip the time-to-coupling comparison of the default line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def allreduce_max(value, world, device):
    """The largest of the ranks' values (the slowest rank's time); the value itself at N = 1."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# algorithmic flop count of one Jacobian transformation, from the program the
# library runs: the sum over contractions of 2 * (product of label extents),
# except the particle-particle ladder (the contraction against the vvvv
# integrals), which the method evaluates in its pair-symmetric (+/-, i <= j,
# a <= b, c <= d) form: o^2 v^4 / 4 multiply-adds per vector, a quarter of its
# label product
# ---------------------------------------------------------------------------
ENGINES = {0: "FP64 DFMA", 1: "split-bf16 TC", 2: "FP64-grade TC"}


def contraction_table(records, steps: int, title: str) -> str:
    """Markdown table of the GEMM launches of `steps` benchmark steps, one row per contraction
    (its launches summed over the steps and divided by them), slowest first."""
    rows = {}
    n_tc = 0  # position among the tensor-core GEMM launches (an ncu launch-skip count)
    for r in records:
        key = (r["label"], r["engine"], r["batch"], r["m"], r["n"], r["k"])
        e = rows.setdefault(key, {"launches": 0, "ms": 0.0, "flops": 0.0, "issued": 0.0, "ladder": r["ladder"],
                                  "first": n_tc if r["engine"] != 0 else None})
        n_tc += r["engine"] != 0
        e["launches"] += 1
        e["ms"] += r["ms"]
        e["flops"] += r["flops"]
        e["issued"] += r["issued_flops"]
    total = sum(e["ms"] for e in rows.values()) / steps
    lines = [f"Per-contraction GEMM time of one benchmark step: {title}", "",
             f"{len(records) // max(steps, 1)} GEMM launches, {total:.1f} ms per step (CUDA events around each "
             "contraction on the library's stream; operand slicing included for the tensor-core forms).", "",
             "| contraction | engine | batch × M × N × K | launches | ms | share | alg. TFLOP/s | issued TFLOP/s "
             "| first TC launch |",
             "|---|---|---|---:|---:|---:|---:|---:|---:|"]
    for (label, eng, b, m, n, k), e in sorted(rows.items(), key=lambda kv: -kv[1]["ms"]):
        ms = e["ms"] / steps
        sec = max(e["ms"], 1e-9) * 1e-3
        shape = (f"{b} × " if b > 1 else "") + f"{m} × {n} × {k}"
        lines.append(f"| `{label}` | {ENGINES.get(eng, eng)}{' (ladder)' if e['ladder'] else ''} | {shape} | "
                     f"{e['launches'] / steps:g} | {ms:.2f} | {ms / max(total, 1e-9):.1%} | "
                     f"{e['flops'] / sec / 1e12:.1f} | {e['issued'] / sec / 1e12:.1f} | "
                     f"{'—' if e['first'] is None else e['first']} |")
    return "\n".join(lines) + "\n"


def transform_flops(o, v, naux, which="jvp"):
    """(all contractions, the ladder's share) in flops for one vector."""
    from paper_2301_13264_gb300 import binding as B
    ext = {"o": o, "v": v, "n": o + v, "x": naux, "z": 1}
    text = B.ccsd_describe_program(which)
    cls = {}
    total = ladder_total = 0.0
    for line in text.splitlines():
        f = line.split()
        if f[0] == "T":
            cls[int(f[1])] = "" if f[4] == "-" else f[4]
        elif f[0] == "C":
            labs = {}
            ladder = False
            for tid, blk, lab in ((int(f[1]), f[2], f[3]), (int(f[4]), f[5], f[6]), (int(f[7]), f[8], f[9])):
                if lab == "-":
                    continue
                c = cls[tid]
                ladder = ladder or c == "vvvv"
                for k, ch in enumerate(lab):
                    b = blk[k]
                    e = ext[b] if c[k] == "n" else ext[c[k]]
                    labs[ch] = e
            fl = 2.0 * float(np.prod(list(labs.values()))) * (0.25 if ladder else 1.0)
            total += fl
            ladder_total += fl if ladder else 0.0
    return total, ladder_total


def ladder_flops_per_vector(o, v):
    """Particle-particle ladder per vector, as the method counts it with the
    pair-symmetric (+/-) packing: o^2 v^4 / 4 multiply-adds."""
    return 2.0 * o * o * v ** 4 / 4.0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------
def oracle_transforms(workload_name, sides=(0, 1)):
    """Seconds of one oracle Jacobian transform per side (0: A R, 1: L^T A) at the
    full workload size, at seeded random amplitudes and vectors."""
    import torch
    from oracle.solvers import System, Vec
    from paper_2301_13264_gb300.synth import random_amplitudes, workload
    H = workload(workload_name)
    S = System(H.eps, H.h, H.B, H.o, vvvv_batch=24)
    X1, X2 = random_amplitudes(H.o, H.v, 31, scale=0.01, nvec=2)
    t = Vec(torch.as_tensor(X1[0]), torch.as_tensor(X2[0]))
    r = Vec(torch.as_tensor(X1[1]), torch.as_tensor(X2[1]))
    times = []
    for side in sides:
        t0 = time.perf_counter()
        (S.right if side == 0 else S.left)(t, r)
        times.append(time.perf_counter() - t0)
    return times, H, torch.get_num_threads()


def cpu_model():
    """The host CPU's model name (/proc/cpuinfo, else lscpu, else the machine type)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def cpu_baseline_entry(workload_name):
    """One right and one left oracle transform at the benchmark's own size, timed directly."""
    times, H, threads = oracle_transforms(workload_name)
    return {"value": len(times) / sum(times), "unit": UNIT, "cores": threads, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": (f"one oracle (numpy/torch FP64) right transform ({times[0]:.1f} s) and one left transform "
                       f"({times[1]:.1f} s) of one vector at o={H.o},v={H.v},naux={H.naux}, the benchmark's own "
                       f"size; value = 2 / their total")}


def run_reference(args, rank, world):
    """The oracle on the host cores, the benchmark's workload.  A full-size oracle
    transform takes minutes, so the timed steps are one right and one left
    transform whatever --steps says (the line states the number run); the warm-up
    is one transform at a tenth of the size.  Nothing of the CUDA library is loaded."""
    if rank != 0:
        return
    from paper_2301_13264_gb300.synth import WORKLOADS
    wl = WORKLOADS[args.workload]
    o, v, naux = wl["o"], wl["v"], wl["naux"]
    if args.warmup > 0:
        import torch
        from oracle.solvers import System, Vec
        from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes
        Hw = make_hamiltonian(o, max(v // 10, 2), max(naux // 10, 2), seed=1)
        Sw = System(Hw.eps, Hw.h, Hw.B, Hw.o)
        W1, W2 = random_amplitudes(Hw.o, Hw.v, 3, scale=0.01, nvec=2)
        Sw.right(Vec(torch.as_tensor(W1[0]), torch.as_tensor(W2[0])), Vec(torch.as_tensor(W1[1]),
                                                                          torch.as_tensor(W2[1])))
    sides = (0, 1)[:max(1, min(args.steps, 2))]
    times, H, threads = oracle_transforms(args.workload, sides)
    total = sum(times)
    value = len(times) / total
    sample = ("each timed step is one oracle transform of one vector at o={},v={},naux={}: ".format(o, v, naux)
              + ", ".join(f"{'right' if s == 0 else 'left'} {t:.1f} s" for s, t in zip(sides, times))
              + f"; {len(times)} of the {args.steps} requested steps run (a full-size oracle transform takes minutes)")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": len(times),
           "steps_requested": args.steps, "warmup": min(args.warmup, 1),
           "ms_per_step": total / len(times) * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"{args.workload} o={o} v={v} naux={naux}",
                      "side": "right + left" if len(times) == 2 else "right"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                            "cpu_model": cpu_model()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2301_13264_gb300 import binding as B
    from paper_2301_13264_gb300.synth import random_amplitudes, workload

    torch.cuda.set_device(local_rank)
    H = workload(args.workload)
    o, v, naux = H.o, H.v, H.naux
    dim = B.vector_dim(o, v)
    stream = torch.cuda.Stream()
    prec = precision_of(args.precision)
    opt = B.ccsd_default_options(precision=prec, splits=args.splits, stream=stream, tol_res=1e-7, tol_lin=1e-6,
                                 max_iter=100)
    h = B.ccsd_create(H.eps, H.h, H.B, o, v, naux, opt)
    t_setup = time.perf_counter()
    if args.amplitudes == "solve":
        e_ccsd, iters = B.ccsd_solve_ground(h)
    else:
        T1, T2 = random_amplitudes(o, v, 999, scale=0.01)
        tt = torch.as_tensor(np.concatenate([T1.reshape(-1), T2.reshape(-1)]), device="cuda")
        e_ccsd, iters = B.ccsd_set_amplitudes(h, tt, torch.zeros_like(tt)), 0
    t_setup = time.perf_counter() - t_setup
    X1, X2 = random_amplitudes(o, v, 1000 + rank, scale=0.01, nvec=args.nvec)
    X = torch.as_tensor(np.concatenate([X1.reshape(args.nvec, -1), X2.reshape(args.nvec, -1)], axis=1),
                        device="cuda").contiguous()
    Y = torch.zeros_like(X)

    def step():
        B.ccsd_jacobian_transform(h, 0, args.nvec, X, Y)
        B.ccsd_jacobian_transform(h, 1, args.nvec, X, Y)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    clocks = Clocks(vis.split(",")[local_rank] if vis and len(vis.split(",")) > local_rank else local_rank)
    B.ccsd_profile_start(h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps (ncu --nvtx-include timed/)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    prof = B.ccsd_profile_stop(h)
    clk = clocks.stop()
    if args.contractions and rank == 0:
        with open(args.contractions, "w") as f:
            f.write(contraction_table(B.ccsd_profile_records(h), args.steps,
                                      f"{args.workload} o={o} v={v} naux={naux}, {args.nvec}-vector blocks, "
                                      f"{args.precision} (S = {args.splits})"))
    ms = ev0.elapsed_time(ev1)
    ms = allreduce_max(ms, world, "cuda")
    value = job_throughput(2 * args.nvec * args.steps, world, ms / 1e3)
    n_tr = 2 * args.nvec * args.steps * world

    # separate right/left rates (short extra runs, not part of the timed region)
    def timed(side, reps=2, nv=None):
        nv = args.nvec if nv is None else nv
        Xs, Ys = X[:nv], Y[:nv]
        if nv != args.nvec:
            B.ccsd_jacobian_transform(h, side, nv, Xs, Ys)  # first use of this block size
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            B.ccsd_jacobian_transform(h, side, nv, Xs, Ys)
        b.record(stream)
        torch.cuda.synchronize()
        return reps * nv / (a.elapsed_time(b) / 1e3)

    right_rate, left_rate = timed(0), timed(1)
    right_rate1, left_rate1 = timed(0, nv=1), timed(1, nv=1)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        Xh = X.cpu().pin_memory()
        Yh = torch.zeros_like(Xh).pin_memory()
        # one untimed call per side: the library's staging buffers for host pointers are
        # allocated on first use
        B.ccsd_jacobian_transform(h, 0, args.nvec, Xh, Yh)
        B.ccsd_jacobian_transform(h, 1, args.nvec, Xh, Yh)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            B.ccsd_jacobian_transform(h, 0, args.nvec, Xh, Yh)
            B.ccsd_jacobian_transform(h, 1, args.nvec, Xh, Yh)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        el = allreduce_max(el, world, "cuda")
        nbytes = 2 * args.nvec * dim * 8
        e2e = {"value": n_tr / el, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    peaks, src = load_peaks()
    peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    # pp-ladder: two tensor-core GEMMs (the + and - parts) per ladder contraction,
    # one contraction per block transform side
    ladder_alg = ladder_flops_per_vector(o, v) * args.nvec
    n_ladder = max(prof["ladder_launches"] // 2, 1)
    lad_ms = prof["ladder_ms"] / n_ladder
    achieved = ladder_alg / (lad_ms * 1e-3) / 1e12 if lad_ms > 0 else 0.0
    issued = prof["ladder_issued_flops"] / n_ladder / (lad_ms * 1e-3) / 1e12 if lad_ms > 0 else 0.0
    executed = prof["ladder_flops"] / n_ladder / (lad_ms * 1e-3) / 1e12 if lad_ms > 0 else 0.0
    # frac: algorithmic flops over the measured bf16 tensor peak (sustained: the ladder
    # runs inside a long step); the split arithmetic issues nprod bf16 products per
    # FP64-equivalent multiply-add (S = 2: 3, S = 3: 6, fixed-point slices: 28), so the
    # peak of the arithmetic the kernel computes in is the bf16 peak / nprod, reported
    # beside it; the FP64 DFMA path is measured against the FP64 peak
    tensor = prec != B.PREC_FP64
    nprod = {B.PREC_MIXED: 3 if args.splits == 2 else 6, B.PREC_FP64_TC: 28}.get(prec, 1)
    peak_main = peak if tensor else FP64_PEAK_TFLOPS
    peak_split = peak / nprod if tensor else FP64_PEAK_TFLOPS
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak_main, "unit": "TFLOP/s",
                "frac": achieved / peak_main, "traffic": LADDER_TRAFFIC.get((args.workload, args.nvec, nprod)),
                "kernel": ("k_tc_gemm<256>" if prec == B.PREC_MIXED else
                           "k_tc_dgemm" if tensor else "k_dgemm") + " (pp-ladder, +/- GEMM pair)",
                "peak_source": (f"bf16_tflops_sustained of {src} MEASURED_PEAKS.json (algorithmic flops over the "
                                "raw bf16 tensor peak)") if tensor
                else "FP64 DFMA peak: 152 SMs x 2.07 GHz x 4 flop/clk",
                "peak_split": peak_split, "frac_of_split_peak": achieved / peak_split,
                "split_products": nprod,
                "split_peak_source": (f"bf16 peak / {nprod} bf16 products per FP64-equivalent multiply-add (" +
                                      ("split-bf16" if prec == B.PREC_MIXED else "fixed-point slice") +
                                      " arithmetic)") if tensor else "FP64 DFMA peak",
                "peak_fp64": FP64_PEAK_TFLOPS, "frac_of_fp64_peak": achieved / FP64_PEAK_TFLOPS,
                "algorithmic_flops_per_launch": ladder_alg,
                "algorithmic_definition": "o^2 v^4 / 4 multiply-adds per vector (pair-packed ladder) x nvec",
                "executed_tflops": executed, "issued_tflops": issued, "issued_frac": issued / peak,
                "launch_ms": lad_ms, "ladder_launches": prof["ladder_launches"],
                "all_tc": {"launches": prof["tc_launches"], "ms": prof["tc_ms"], "alg_tflops":
                           prof["tc_flops"] / max(prof["tc_ms"], 1e-9) / 1e9,
                           "issued_tflops": prof["tc_issued_flops"] / max(prof["tc_ms"], 1e-9) / 1e9},
                "fp64_gemm": {"launches": prof["fp64_launches"], "ms": prof["fp64_ms"],
                              "tflops": prof["fp64_flops"] / max(prof["fp64_ms"], 1e-9) / 1e9}}
    f_alg, _ = transform_flops(o, v, naux)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None,
           "dtype": DTYPE[prec] % nprod,
           "data": "synthetic",
           "config": {"workload": f"{args.workload} o={o} v={v} naux={naux}", "nvec": args.nvec,
                      "step": f"right + left block transform of {args.nvec} vectors",
                      "precision": args.precision, "splits": args.splits,
                      "l2": f"inputs larger than L2 (vvvv integrals {v ** 4 * 8 / 1e9:.1f} GB)"},
           "right_transforms_per_s": right_rate, "left_transforms_per_s": left_rate,
           "block1_transforms_per_s": {"right": right_rate1, "left": left_rate1},
           "alg_tflops_per_transform": f_alg / 1e12,
           "alg_tflops": value * f_alg / 1e12 / world,
           "setup": {"ground_iters": iters, "e_ccsd": e_ccsd, "ground_seconds": t_setup},
           "roofline": roofline, "e2e": e2e, "gpu_launches": prof["launches"], "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_entry(args.workload)
    if rank == 0 and world == 1 and not args.no_ttc:
        # time to converged coupling at equal accuracy, measured in this run: the refined mixed
        # form against the FP64-grade tensor-core form (FP64-accurate; the DFMA form takes minutes)
        # at the thymine/cc-pVDZ size, where both finish in about a minute and a half
        t = measure_ttc("thymine_dz", ["mixed", "fp64tc"], args.splits, 1e-9, 96)
        m = t["forms"]["mixed"]
        out["ttc"] = {"workload": t["workload"], "pairs": t["pairs"], "thresholds": t["thresholds"],
                      "mixed_s": m["seconds"], "reference_form": "fp64tc (FP64-grade tensor-core products)",
                      "reference_s": t["forms"]["fp64tc"]["seconds"], **m["vs_fp64tc"]}
    B.ccsd_destroy(h)
    if rank == 0:
        print(json.dumps(out), flush=True)


def precision_of(name):
    """The library's precision constant for a form name (mixed, fp64, fp64tc)."""
    from paper_2301_13264_gb300 import binding as B
    return {"mixed": B.PREC_MIXED, "fp64": B.PREC_FP64, "fp64tc": B.PREC_FP64_TC}[name]


DTYPE = {0: "f64", 1: "f64 (bf16x%d split tensor-core products, fp32 accumulate)",
         2: "f64 (FP64-grade tensor-core products: 7 fixed-point bf16 slices, %d products, exact chunk sums)"}


def run_ttc(args):
    """Time-to-converged coupling: wall time from ccsd_create through the
    derivative couplings F_12, F_01, F_20 along (h1, B1), per precision form, at
    the same convergence thresholds (1e-10 residual, --tol-eom (1e-8) EOM, 1e-9
    linear).  Every form is compared, root by root, with the FP64 DFMA form when
    it ran, else with the FP64-grade tensor-core form."""
    forms = ["mixed", "fp64"] if args.ttc == "both" else args.ttc.split(",")
    print(json.dumps(measure_ttc(args.workload, forms, args.splits, args.tol_eom, args.max_sub, args.ttc_profile,
                                 args.tc_min_flops)), flush=True)


def gemm_time_by_engine(records) -> dict:
    """GEMM launches, device milliseconds and algorithmic TFLOP per arithmetic form."""
    out = {}
    for r in records:
        e = out.setdefault(ENGINES.get(r["engine"], str(r["engine"])), {"launches": 0, "ms": 0.0, "alg_tflop": 0.0})
        e["launches"] += 1
        e["ms"] += r["ms"]
        e["alg_tflop"] += r["flops"] / 1e12
    return out


def measure_ttc(workload_name, forms, splits, tol_eom, max_sub, profile=False, tc_min_flops=None):
    """The time-to-converged-coupling comparison of run_ttc as a dict.  With profile, every
    GEMM after ccsd_create is bracketed by CUDA events (which slows the run a little) and the
    device time per arithmetic form is added."""
    import torch
    from paper_2301_13264_gb300 import binding as B
    from paper_2301_13264_gb300.synth import workload

    H = workload(workload_name)
    for f in forms:
        if f not in ("mixed", "fp64", "fp64tc"):
            raise SystemExit(f"unknown form {f!r}")
    out = {"metric": "time-to-converged coupling", "unit": "s", "higher_is_better": False,
           "workload": f"{workload_name} o={H.o} v={H.v} naux={H.naux}", "pairs": [[1, 2], [0, 1], [2, 0]],
           "forms": {}}
    for form in forms:
        prec = precision_of(form)
        kw = {} if tc_min_flops is None else {"tc_min_flops": tc_min_flops}
        opt = B.ccsd_default_options(precision=prec, splits=splits, tol_res=1e-10, tol_eom=tol_eom,
                                     tol_lin=1e-9, max_iter=300, refine=1, davidson_max_sub=max_sub, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = B.ccsd_create(H.eps, H.h, H.B, H.o, H.v, H.naux, opt)
        if profile:
            B.ccsd_profile_start(h)
        e, it_g = B.ccsd_solve_ground(h)
        t_g = time.perf_counter() - t0
        print(f"[ttc {form}] ground {t_g:.1f}s {it_g} iterations E={e:.12f}", file=sys.stderr, flush=True)
        w, it_r = B.eom_solve_right(h, 2)
        print(f"[ttc {form}] right EOM {time.perf_counter() - t0:.1f}s {it_r} iterations {w}", file=sys.stderr,
              flush=True)
        wl, it_l = B.eom_solve_left(h, 2)
        t_e = time.perf_counter() - t0
        F = [B.ccsd_derivative_coupling(h, k, l, 1, H.h1, H.B1)[0] for k, l in out["pairs"]]
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out["forms"][form] = {"seconds": t, "ground_s": t_g, "eom_s": t_e - t_g, "couplings_s": t - t_e,
                              "e_ccsd": e, "omega": w, "F": F, "iters": [it_g, it_r, it_l],
                              "stats": B.ccsd_stats(h)}
        if profile:
            B.ccsd_profile_stop(h)
            out["forms"][form]["gemm_time"] = gemm_time_by_engine(B.ccsd_profile_records(h))
        B.ccsd_destroy(h)
    out["thresholds"] = {"tol_res": 1e-10, "tol_eom": tol_eom, "tol_lin": 1e-9, "davidson_max_sub": max_sub}
    ref_name = "fp64" if "fp64" in out["forms"] else ("fp64tc" if "fp64tc" in out["forms"] else None)
    if ref_name:
        f = out["forms"][ref_name]
        out["reference_form"] = ref_name
        for name, m in out["forms"].items():
            if name == ref_name:
                continue
            m["vs_" + ref_name] = {
                "speedup": f["seconds"] / m["seconds"], "energy_diff": abs(m["e_ccsd"] - f["e_ccsd"]),
                "omega_diff_per_root": [abs(a - b) for a, b in zip(m["omega"], f["omega"])],
                "coupling_rel_diff_per_pair": [abs(a - b) / abs(b) for a, b in zip(m["F"], f["F"])],
                "omega_diff": max(abs(a - b) for a, b in zip(m["omega"], f["omega"])),
                "coupling_rel_diff": max(abs(a - b) / abs(b) for a, b in zip(m["F"], f["F"]))}
    return out


def batch_shapes(nsys, seed=4):
    """Uneven systems: o ~ U{4..20}, v ~ U{30..120}, naux = 3.5 (o + v)."""
    rng = np.random.default_rng(seed)
    o = rng.integers(4, 21, nsys)
    v = rng.integers(30, 121, nsys)
    return [(int(a), int(b), int(3.5 * (a + b))) for a, b in zip(o, v)]


def run_batch(args):
    """Batched block transforms of many small systems: one graph launch per side
    for all systems against the same transforms launched system by system."""
    import torch
    from paper_2301_13264_gb300 import binding as B
    from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes

    shapes = batch_shapes(args.batch)
    nvec = args.nvec
    prec = precision_of(args.precision)
    hs, X, Y = [], [], []
    t0 = time.perf_counter()
    for k, (o, v, naux) in enumerate(shapes):
        H = make_hamiltonian(o, v, naux, seed=500 + k)
        opt = B.ccsd_default_options(precision=prec, splits=args.splits, autotune=int(not args.no_autotune))
        h = B.ccsd_create(H.eps, H.h, H.B, o, v, naux, opt)
        T1, T2 = random_amplitudes(o, v, 900 + k, scale=0.02)
        t = torch.as_tensor(np.concatenate([T1.reshape(-1), T2.reshape(-1)]), device="cuda")
        B.ccsd_set_amplitudes(h, t, torch.zeros_like(t))
        X1, X2 = random_amplitudes(o, v, 1900 + k, scale=0.02, nvec=nvec)
        X.append(torch.as_tensor(np.concatenate([X1.reshape(nvec, -1), X2.reshape(nvec, -1)], axis=1),
                                 device="cuda").contiguous())
        Y.append(torch.zeros_like(X[-1]))
        hs.append(h)
    setup = time.perf_counter() - t0

    def seq_step():
        for h, x, y in zip(hs, X, Y):
            B.ccsd_jacobian_transform(h, 0, nvec, x, y)
            B.ccsd_jacobian_transform(h, 1, nvec, x, y)

    def timed(fn, steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / steps

    for _ in range(args.warmup):
        seq_step()
    seq_s = timed(seq_step, args.steps)
    b = B.ccsd_batch_create(hs, nvec)
    Yb = [torch.zeros_like(x) for x in X]

    def batch_step():
        B.ccsd_batch_transform(b, 0, X, Yb)
        B.ccsd_batch_transform(b, 1, X, Yb)

    t_cap = time.perf_counter()
    batch_step()  # direct run + capture, one per side
    t_cap = time.perf_counter() - t_cap
    for _ in range(max(args.warmup - 1, 1)):
        batch_step()
    clocks = Clocks(0)
    bat_s = timed(batch_step, args.steps)
    clk = clocks.stop()
    st = B.ccsd_batch_stats(b)
    diff = max(float((yb - y).abs().max() / y.abs().max()) for yb, y in zip(Yb, Y))
    B.ccsd_batch_destroy(b)
    for h in hs:
        B.ccsd_destroy(h)
    n_tr = 2 * nvec * len(hs)
    out = {"metric": "batched Jacobian transforms/s", "unit": "transforms/s", "higher_is_better": True,
           "value": n_tr / bat_s, "sequential_value": n_tr / seq_s, "speedup": seq_s / bat_s,
           "ms_per_step": bat_s * 1e3, "sequential_ms_per_step": seq_s * 1e3, "steps": args.steps,
           "warmup": args.warmup, "dtype": "f64 (bf16 split tensor-core products)" if prec else "f64",
           "config": {"workload": f"{len(hs)} systems, o~U{{4..20}}, v~U{{30..120}}, naux=3.5(o+v)", "nvec": nvec,
                      "step": "right + left block transform of nvec vectors for every system",
                      "autotune": not args.no_autotune, "precision": args.precision},
           "graph": {"captures": st["captures"], "launches": st["launches"], "kernel_nodes_per_launch": st["nodes"],
                     "capture_and_first_run_s": t_cap},
           "max_rel_diff_vs_sequential": diff, "setup_s": setup, "clocks": clk}
    print(json.dumps(out), flush=True)


def run_batch_eom(args):
    """Right EOM roots of many small systems: the lockstep batched Davidson (one graph
    launch per iteration for all systems) against per-system solves, same handles and
    thresholds."""
    import torch
    from paper_2301_13264_gb300 import binding as B
    from paper_2301_13264_gb300.synth import make_hamiltonian

    shapes = batch_shapes(args.batch)
    nroots = args.batch_eom
    prec = precision_of(args.precision)
    hs = []
    t0 = time.perf_counter()
    for k, (o, v, naux) in enumerate(shapes):
        H = make_hamiltonian(o, v, naux, seed=500 + k)
        opt = B.ccsd_default_options(precision=prec, splits=args.splits, autotune=int(not args.no_autotune),
                                     tol_res=1e-8, tol_eom=1e-6, tol_lin=1e-8, refine=1, max_iter=200)
        h = B.ccsd_create(H.eps, H.h, H.B, o, v, naux, opt)
        B.ccsd_solve_ground(h)
        hs.append(h)
    setup = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w_seq = [B.eom_solve_right(h, nroots)[0] for h in hs]
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    b = B.ccsd_batch_create(hs, args.nvec)
    t0 = time.perf_counter()
    w_bat, iters = B.ccsd_batch_eom_solve(b, 0, nroots, len(hs))
    torch.cuda.synchronize()
    bat_s = time.perf_counter() - t0
    st = B.ccsd_batch_stats(b)
    B.ccsd_batch_destroy(b)
    for h in hs:
        B.ccsd_destroy(h)
    diff = float(np.abs(np.array(w_seq) - w_bat).max())
    print(json.dumps({"metric": "batched EOM solve", "unit": "s", "higher_is_better": False,
                      "config": {"workload": f"{len(hs)} systems, o~U{{4..20}}, v~U{{30..120}}, naux=3.5(o+v)",
                                 "nroots": nroots, "nvec": args.nvec, "precision": args.precision,
                                 "tol_eom": 1e-6, "refine": 1},
                      "sequential_s": seq_s, "batched_s": bat_s, "speedup": seq_s / bat_s,
                      "max_root_diff": diff, "max_iterations": max(iters), "graph": st, "setup_s": setup}),
          flush=True)


def run_mlp(args):
    """Learned-guess kernels at a workload's size: features of every doubles element,
    inference over all of them (tensor-core kernel), and training steps."""
    import torch
    from paper_2301_13264_gb300 import binding as B
    from paper_2301_13264_gb300.synth import workload

    H = workload(args.workload)
    o, v = H.o, H.v
    n2 = o * o * v * v
    h = B.ccsd_create(H.eps, H.h, H.B, o, v, H.naux, B.ccsd_default_options(precision=B.PREC_MIXED))
    X = torch.zeros((n2, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros(n2, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(0)
    model = np.zeros(B.MLP_PARAMS, dtype=np.float32)
    model[:B.MLP_TRAINABLE] = rng.normal(0.0, 0.1, B.MLP_TRAINABLE)
    model[B.MLP_TRAINABLE + 3:B.MLP_TRAINABLE + 6] = 1.0
    model[B.MLP_TRAINABLE + 6] = 1.0
    m_dev = torch.as_tensor(model, device="cuda")

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    f_ms = timed(lambda: B.ccsd_guess_features(h, X), args.steps)
    p_ms = timed(lambda: B.ccsd_mlp_predict(m_dev, X, out), args.steps)
    T = torch.zeros(min(n2, 4_000_000), dtype=torch.float32, device="cuda")
    Xs = X[:T.shape[0]].contiguous()
    t0 = time.perf_counter()
    B.ccsd_mlp_train(Xs, T, 200, 8192, 1e-3, 1)
    torch.cuda.synchronize()
    tr_s = time.perf_counter() - t0
    B.ccsd_destroy(h)
    flop_row = 2 * (3 * 128 + 128 * 128 + 128)
    peaks, src = load_peaks()
    print(json.dumps({"metric": "learned-guess kernels", "workload": f"{args.workload} o={o} v={v}", "rows": n2,
                      "features_ms": f_ms, "inference_ms": p_ms, "inference_rows_per_s": n2 / (p_ms * 1e-3),
                      "inference_tflops": n2 * flop_row / (p_ms * 1e-3) / 1e12,
                      "inference_frac_of_bf16_peak": n2 * flop_row / (p_ms * 1e-3) / 1e12 / peaks["bf16_tflops"],
                      "train_200_steps_s": tr_s, "train_rows_per_s": 200 * 8192 / tr_s,
                      "peak_source": f"bf16_tflops of {src} MEASURED_PEAKS.json"}), flush=True)


def run_guess_eval(args):
    """The learned starts at the workload's size: train the doubles network (t_CCSD - t_MP2)
    and the multiplier network (lambda - (-eta/D)) on solved systems of the same generator
    at a reduced size (o, v and naux divided by args.guess_scale, seeds 1000...), then solve
    the workload's ground state and Lambda equations to residual 1e-7 from the plain and the
    learned starts, and report iteration counts and the distance of each start from the
    converged doubles."""
    import torch
    from paper_2301_13264_gb300 import binding as B
    from paper_2301_13264_gb300 import learned_guess as lg
    from paper_2301_13264_gb300.synth import WORKLOADS, make_hamiltonian, workload

    wl = WORKLOADS[args.workload]
    f = args.guess_scale
    to, tv, tx = max(2, round(wl["o"] / f)), max(4, round(wl["v"] / f)), max(8, round(wl["naux"] / f))
    systems = [make_hamiltonian(to, tv, tx, seed=1000 + s) for s in range(args.guess_train)]
    t0 = time.perf_counter()
    topt = B.ccsd_default_options(tol_res=1e-8, tol_lin=1e-8)
    models, losses = {}, {}
    for name, which in (("amplitudes", B.GUESS_AMPLITUDES), ("multipliers", B.GUESS_MULTIPLIERS)):
        X, T = lg.generate(systems, topt, rows_per_system=min(20000, to * to * tv * tv), seed=3, which=which)
        models[name], losses[name] = lg.train(X, T, steps=3000, batch=8192, lr=2e-3, seed=5)
    train_s = time.perf_counter() - t0
    H = workload(args.workload)
    o, v = H.o, H.v
    opt = B.ccsd_default_options(precision=B.PREC_MIXED, splits=args.splits, tol_res=1e-7, tol_lin=1e-7,
                                 max_iter=300)
    out = {}
    for name in ("plain", "learned"):
        h = B.ccsd_create(H.eps, H.h, H.B, o, v, H.naux, opt)
        try:
            if name == "learned":
                B.ccsd_set_guess_model(h, models["amplitudes"])
                B.ccsd_set_multiplier_guess_model(h, models["multipliers"])
            mt = models["amplitudes"] if name == "learned" else None
            mm = models["multipliers"] if name == "learned" else None
            st = lg.guess_doubles(h, o, v, mt).ravel()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            e, _ = B.ccsd_solve_ground(h)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t1
            it = B.ccsd_solve_iterations(h)
            sm = lg.guess_doubles(h, o, v, mm, which=B.GUESS_MULTIPLIERS).ravel()
            dim = B.vector_dim(o, v)
            t, lam = np.zeros(dim), np.zeros(dim)
            B.ccsd_get_amplitudes(h, t, lam)
            out[name] = {"ground_iterations": it["ground"], "lambda_iterations": it["lambda"],
                         "ground_and_lambda_s": secs, "e_ccsd": e,
                         "start_error_doubles": float(np.linalg.norm(st - t[o * v:])),
                         "start_error_multipliers": float(np.linalg.norm(sm - lam[o * v:]))}
        finally:
            B.ccsd_destroy(h)
    print(json.dumps({"metric": "iterations to residual 1e-7 from the learned and the plain starts",
                      "workload": f"{args.workload} o={o} v={v} naux={H.naux}",
                      "training": {"systems": len(systems), "o": to, "v": tv, "naux": tx, "seconds": train_s,
                                   "final_loss": losses},
                      "precision": f"mixed S={args.splits}, refined", "results": out}), flush=True)


def main():
    args = parse()
    if args.guess_eval:
        run_guess_eval(args)
        return
    if args.mlp:
        run_mlp(args)
        return
    if args.ttc:
        run_ttc(args)
        return
    if args.batch and args.batch_eom:
        run_batch_eom(args)
        return
    if args.batch:
        run_batch(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
