#!/usr/bin/env python
"""Throughput of the t-product hot path on one GB300 (or N GPUs as independent replicas).

Step = one batched prox_tnn call (Algorithm 3) over the batched workload: 512 independent
real tensors with n1, n2 uniform in {16..160}, n3 uniform in {4..64}, tubal rank r uniform
in {2..12} (t-product of N(0,1) factors) plus N(0, 0.05^2) noise, tau = 2x the noise level
of one Fourier slice.  Metric: prox_tnn Fourier slices per second (a slice is one of the
ceil((n3+1)/2) directly computed frontal slices of a tensor).

The headline value is the learned form (rank proposer + randomized SVT, Jacobi fallback),
with the plain FP32 Jacobi path measured beside it ("plain") on the same batch; the
proposer is trained beforehand, untimed, on batches drawn with other seeds.

The JSON line also carries:
  roofline      the dominant slice kernel of the step, timed live with CUDA events recorded
                by the library at stage boundaries, against the FP32 ALU peak;
  e2e           the same metric through tp_prox_tnn_batched_host: page-locked host inputs
                copied in and outputs copied back inside the timed region, consecutive steps
                on two alternating streams so copies overlap kernels;
  tprod         t-product TFLOP/s on A 2048x1024x64 times B 1024x1024x64 (--gemm-shape) in
                FP32, BF16x3 and 3xTF32 slice-GEMM arithmetic;
  tran          the conjugate transpose of that A, GB/s against the HBM copy peak;
  trpca         the synthetic TRPCA-style loop: 50 ADMM iterations on a 240x320x100 tensor
                (tubal rank 10, unit RMS, 10% of entries corrupted by U[-5, 5]), each one
                prox_tnn call at tau = 1/mu (library) plus two elementwise updates; plain
                Jacobi vs learned (proposer trained on the iterates of another draw);
  factor        tensor inverse (Def. 2.4) on 128x128x302 and economy t-QR (Thm. 2.4) on
                128x64x302 (152 independent slices each, one per SM), slices/s and the slice
                kernel's FP32 flop rate;
  plain.autotuned  the plain path again after tp_autotune_jacobi chose the Jacobi CTA shape
                by timing its candidates on this batch (the shape stays set for the learned
                step, whose fallback slices use it; the other legs run at the default);
  stream        the first 500 calls (--stream-calls) of the mixed call stream (prox_tnn and
                tprod calls on tensors up to 512x512x256): every call on its own in FP32 with
                Jacobi, against windows of calls as replayed learned batched plans plus BF16x3
                tprod;
  cpu_baseline  the FP64 oracle on a bounded sample of the same workload.

`--impl reference` times the FP64 oracle itself (host cores) on the same workload.
Multi-GPU (torchrun): every rank runs its own batch (seed = rank); no collective on the
data path; value = all ranks' slices / max-over-ranks time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "prox_tnn slices/s & tprod TFLOP/s vs plain FP32 GPU path at ≤1e-4 rel err"
UNIT = "slices/s"
WORKLOAD = ("batched prox_tnn, FP32: 512 tensors, n1,n2~U{16..160}, n3~U{4..64}, tubal rank "
            "r~U{2..12} t-product of N(0,1) factors + N(0,0.05^2) noise, tau = 2x noise level")
SM_COUNT_DEFAULT = 152  # GB300; the device's own count replaces it when a GPU is present


def load_peaks(path=os.path.join(ROOT, "MEASURED_PEAKS.json")):
    """Roofline denominators: the measured copy bandwidth, dense bf16 rate (burst) and maximum
    SM clock from MEASURED_PEAKS.json when it is present, else the values recorded from it on
    this GB300 pool."""
    peaks = {"hbm_gbs": 6685.5, "bf16_tflops": 1944.2, "sm_max_mhz": 2070.0,
             "source": "recorded values (MEASURED_PEAKS.json absent)"}
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "bf16_tflops", "sm_max_mhz"):
            v = d.get(k)
            if isinstance(v, (int, float)) and v > 0:
                peaks[k] = float(v)
        peaks["source"] = "MEASURED_PEAKS.json"
    except (OSError, ValueError, AttributeError):
        pass
    return peaks


PEAKS = load_peaks()


def sm_count() -> int:
    """Multiprocessors of the current CUDA device (the GB300 count without a GPU)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device())
                       .multi_processor_count)
    except Exception:  # pragma: no cover - no torch or no driver
        pass
    return SM_COUNT_DEFAULT


def fp32_peak_tflops(sms: int | None = None) -> float:
    """FFMA lanes (128 per SM) x 2 flops x maximum SM clock."""
    return (sms or sm_count()) * 128 * 2 * PEAKS["sm_max_mhz"] * 1e6 / 1e12


FP32_PEAK_TFLOPS = fp32_peak_tflops(SM_COUNT_DEFAULT)  # replaced in run_tp by the device's


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="tp", choices=["tp", "reference"])
    p.add_argument("--count", type=int, default=512)
    p.add_argument("--no-tprod", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-factor", action="store_true")
    p.add_argument("--no-trpca", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-stream", action="store_true")
    # the first 500 calls of the seeded stream: an unbiased sample of the 2000-call stream
    # (same generator and distributions) whose plain pass (~12 s) keeps the run within minutes
    p.add_argument("--stream-calls", type=int, default=500)
    p.add_argument("--host-parts", type=int, default=1, choices=[1, 2],
                   help="tp_options.host_parts of the e2e leg's calls")
    p.add_argument("--gemm-shape", default="2048,1024,1024,64",
                   help="n1,n2,l,n3 of the tprod leg (A n1 x n2 x n3 times B n2 x l x n3)")
    p.add_argument("--stream-window", type=int, default=16)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--train-batches", type=int, default=4,
                   help="512-tensor batches (other seeds) that label the proposer's training set")
    return p.parse_args()


def max_over_ranks(ms: float, device) -> float:
    """The slowest rank's time: every rank's timed region ends at a barrier, the job's
    time is the maximum."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(n: float, device) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(n)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_all_ranks: float, steps: int, ms_max: float) -> float:
    """Weak scaling: every rank processes its own batch; value = all ranks' units per step
    times the steps, over the slowest rank's time."""
    return units_all_ranks * steps / (ms_max / 1e3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of the SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- workload
# DRAM traffic of the sketch stage (dram__bytes_read.sum + dram__bytes_write.sum over the four
# class launches of one call) per byte of half spectrum, from an ncu capture of the 160-tensor
# batch of the same workload: 274.9 MB for 178.9 MB of spectrum.  The traffic of a batch is
# taken in proportion to its half-spectrum bytes.
SKETCH_DRAM_PER_SPEC_BYTE = 274.9 / 178.9


def svd_launch_groups(shapes, shape=None):
    """Kernel launches of the Jacobi stage of one batched prox call (mirrors the library's
    slice planner under a Jacobi CTA shape: lanes per column pair, float4 pairs per lane,
    shared or global memory, and the CTA size when launches are split by it)."""
    shape = shape or {"target_lane_pairs": 5, "max_warps": 32, "split_launches": 0}
    groups = set()
    for n1, n2 in shapes:
        m, n = max(n1, n2), min(n1, n2)
        best, lp = 1e30, 32
        for cand in (8, 16, 32):
            e2 = (m + 2 * cand - 1) // (2 * cand)
            if e2 > 8:
                continue
            score = (2 * cand * e2 - m) / m + 0.03 * abs(e2 - shape["target_lane_pairs"])
            if score < best:
                best, lp = score, cand
        e2 = (m + 2 * lp - 1) // (2 * lp)
        maxe2 = 2 if e2 <= 2 else (4 if e2 <= 4 else 8)
        ld = 2 * lp * e2
        aux = (6 * n * 4 + 256 + (m + 1) * 4 + 20 * m + 15) & ~15
        in_smem = n * ld * 8 + aux <= 227 * 1024 - 1024
        threads = 0
        if shape["split_launches"]:
            pairs, spw = (n + 1) // 2, 32 // lp
            wmax = min(shape["max_warps"], 16 if maxe2 >= 8 else 32)
            passes = -(-pairs // (wmax * spw))
            threads = 32 * max(2, -(-pairs // (passes * spw)))
        groups.add((in_smem, lp, maxe2, threads))
    return len(groups)


# Kernel launches of one learned batched prox call besides the Jacobi groups and the tube DFTs:
# features, proposer MLP, binning, one persistent sketch launch per size class (four shared-
# memory classes and the global-scratch class), a collect and a sketch launch per retry round.
SKETCH_CLASSES, SKETCH_RETRY_ROUNDS = 5, 4
LEARNED_FIXED_LAUNCHES = 3 + SKETCH_CLASSES + 2 * SKETCH_RETRY_ROUNDS

# Register classes of the per-length DFT kernels for n3 <= 64 (bit n3 - 1: class >= 1, class 2),
# the masks of the library's DFT source; a batch of mixed lengths launches each direction once
# per class present.
DFT_CLASS_AT_LEAST_1, DFT_CLASS_2 = 0xfffffff500000000, 0x0


def dft_launches(n3s):
    """Launches of one direction of the tube DFT over tensors of these lengths."""
    n3s = [int(n) for n in n3s if n > 0]
    if not n3s:
        return 0
    uniform = len(set(n3s)) == 1
    if uniform and n3s[0] & (n3s[0] - 1) == 0 and n3s[0] <= 64 and n3s[0] >= 2:
        return 1  # register radix-2 kernel
    if max(n3s) > 64:
        return 1  # direct kernel
    cls = {((DFT_CLASS_AT_LEAST_1 >> (n - 1)) & 1) + ((DFT_CLASS_2 >> (n - 1)) & 1) for n in n3s}
    return len(cls)


def make_batch(tp, synth, count, seed, device):
    import numpy as np
    import torch
    specs = synth.batched_specs(512, seed)[:count]
    Ys, taus = [], []
    for i, s in enumerate(specs):
        f = synth.batched_tensor(s, i, seed)
        Y = tp.tprod(tp.to_device(f["P"], device), tp.to_device(f["Q"], device))
        Y.add_(tp.to_device(f["E"], device))
        Ys.append(Y)
        taus.append(s.tau)
    torch.cuda.synchronize()
    slices = sum(s.n3 // 2 + 1 for s in specs)
    nbytes = sum(4 * s.n1 * s.n2 * s.n3 for s in specs)
    model_shapes = [(s.n1, s.n2, s.n3) for s in specs]
    return specs, Ys, taus, slices, nbytes, model_shapes


def jacobi_model_flops(shapes, sweeps):
    """Model count of the one-sided Jacobi: per sweep n(n-1)/2 column pairs, 40 m real flops
    per pair (16 m for the three dot products, 24 m for the complex rotation of two columns)."""
    total, idx = 0.0, 0
    for n1, n2, n3 in shapes:
        m, n = max(n1, n2), min(n1, n2)
        for _ in range(n3 // 2 + 1):
            total += float(sweeps[idx]) * n * (n - 1) / 2 * 40.0 * m
            idx += 1
    return total


# ----------------------------------------------------------------------------- oracle legs
def oracle_sample(specs, seed, seconds, max_items=None, inputs=None, check=None):
    """Time the FP64 oracle's prox_tnn on tensors 0, 1, ... of the batch until `seconds`
    of CPU work (at least one tensor). Returns (slices/s, slices, tensors, seconds).
    inputs(i), if given, returns tensor i as the FP32 array the GPU received (else the oracle
    forms it from the generator's factors); check(i, W), if given, receives each oracle
    result (outside the timed region)."""
    import numpy as np

    from oracle import tproduct as O
    from paper_1806_07247_gb300 import synth
    done_slices, done, t_total = 0, 0, 0.0
    for i, s in enumerate(specs):
        if inputs is not None:
            X = inputs(i)
        else:
            f = synth.batched_tensor(s, i, seed)
            X = (O.tprod_fourier(f["P"], f["Q"]) + f["E"]).astype(np.float32)
        t0 = time.perf_counter()
        W = O.prox_tnn(X, s.tau)
        t_total += time.perf_counter() - t0
        if check is not None:
            check(i, W)
        done_slices += s.n3 // 2 + 1
        done += 1
        if t_total >= seconds or (max_items and done >= max_items):
            break
    return done_slices / t_total, done_slices, done, t_total


def oracle_single_core(seed, seconds):
    """The same oracle sample with every BLAS/LAPACK/OpenMP pool at one thread (a child
    process, since the pools are sized when numpy loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "from paper_1806_07247_gb300 import synth; "
            "r = bench.oracle_sample(synth.batched_specs(512, %d), %d, %f); "
            "print(json.dumps(r))" % (ROOT, seed, seed, seconds))
    try:
        res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                             text=True, timeout=max(60.0, 10 * seconds))
        rate, sl, nt, secs = json.loads(res.stdout.strip().splitlines()[-1])
        return {"value": rate, "unit": UNIT, "cores": 1,
                "sample": f"tensors 0-{nt - 1} ({sl} free slices, {secs:.1f} s)"}
    except Exception as e:  # the bench line must still print
        return {"value": None, "error": str(e)[:200]}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1806_07247_gb300 import synth
    specs = synth.batched_specs(512, 0)[:args.count]
    sample = specs[:6]
    times, slices = [], sum(s.n3 // 2 + 1 for s in sample)
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle_sample(sample, 0, seconds=1e9, max_items=len(sample))
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = slices * args.steps / total
    cores = os.cpu_count()
    desc = (f"each step: FP64 oracle prox_tnn on tensors 0-5 of the 512-tensor batch "
            f"({slices} free slices), all n3 slices SVD'd by LAPACK")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tensors": len(specs), "seed": 0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def sketch_model_flops(shapes, widths, counts=None, one_product=False):
    """Flop counts of the sketch SVT stage over the slices it sketched (width l > 0).

    one_product=False, the work the kernel does for one slice of width l: five passes of an
    n1 x n2 by n2 x l complex product (range finder, one power iteration, B, residual check),
    four n1 x n2 complex mat-vecs (norm estimate) and the W update; 8 flops per complex MAC:
    8 n1 n2 (6 l + 4).
    one_product=True, the usual count of randomized SVD work, 8 m n (k + p) flops per
    sketched slice with k + p = l (one n1 x n2 by n2 x l complex product)."""
    total, idx = 0.0, 0
    for n1, n2, n3 in shapes:
        for _ in range(n3 // 2 + 1):
            l = int(widths[idx])
            if l > 0:
                total += 8.0 * n1 * n2 * (l if one_product else (5 * l + 4 + l))
            idx += 1
    return total


def time_prox(tp, args, Ys, Xs, taus, descs, method, world, barrier, device, clocks=None):
    """Warm-up, then `steps` timed batched calls with stage events; returns timing and the
    per-slice diagnostics of the last call."""
    import torch
    import torch.distributed as dist
    nsl = sum(Y.shape[2] // 2 + 1 for Y in Ys)
    sweeps = torch.zeros(nsl, dtype=torch.int32, device=device)
    flags = torch.zeros(nsl, dtype=torch.int32, device=device)
    widths = torch.zeros(nsl, dtype=torch.int32, device=device)
    for _ in range(args.warmup):
        tp.prox_tnn_batched(Ys, taus, outs=Xs, opts=tp.options(sync=False, method=method), descs=descs)
    torch.cuda.synchronize()
    tp.prox_tnn_batched(Ys, taus, outs=Xs, opts=tp.options(sync=True, method=method, sweeps_out=sweeps,
                                                          slice_flags_out=flags,
                                                          sketch_width_out=widths), descs=descs)

    def events():
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(tp.STAGE_EVENTS)]
        for e in evs:
            e.record()
        return evs

    stage = [events() for _ in range(args.steps)]
    opts = [tp.options(sync=False, method=method, stage_events=stage[i]) for i in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    if clocks:
        clocks.start()
    torch.cuda.nvtx.range_push(f"{method}_timed")  # lets a profiler select the timed steps
    t0.record()
    for i in range(args.steps):
        tp.prox_tnn_batched(Ys, taus, outs=Xs, opts=opts[i], descs=descs)
    t1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(t0.elapsed_time(t1), device)
    names = ["rfft", "proposer", "sketch_svt", "jacobi_svt", "irfft"]
    st = {n: sum(s_[j].elapsed_time(s_[j + 1]) for s_ in stage) / args.steps
          for j, n in enumerate(names)}
    return {"ms": ms, "stages": st, "sweeps": sweeps.cpu().numpy(), "clocks": clk,
            "flags": flags.cpu().numpy(), "widths": widths.cpu().numpy()}


def run_tp(args):
    global FP32_PEAK_TFLOPS
    import torch
    import torch.distributed as dist

    from paper_1806_07247_gb300 import synth, tp

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    FP32_PEAK_TFLOPS = fp32_peak_tflops()
    if world > 1:
        dist.init_process_group("nccl", device_id=device)

    def barrier():
        if world > 1:
            dist.barrier()

    tp.lib()
    specs, Ys, taus, slices, nbytes, shapes = make_batch(tp, synth, args.count, rank, device)
    Xs = [tp.empty(*Y.shape, device=device) for Y in Ys]
    descs = tp.make_descs(Ys, Xs, taus)
    spec_bytes = sum(8 * a * b * (c // 2 + 1) for a, b, c in shapes)

    # --- plain FP32 path (one-sided Jacobi on every slice)
    plain = time_prox(tp, args, Ys, Xs, taus, descs, "jacobi", world, barrier, device)
    X_plain = [X.clone() for X in Xs]
    jflops = jacobi_model_flops(shapes, plain["sweeps"])
    jt = plain["stages"]["jacobi_svt"]
    slices_all = sum_over_ranks(slices, device)
    plain_value = job_throughput(slices_all, args.steps, plain["ms"])
    plain_line = {"value": plain_value, "ms_per_step": plain["ms"] / args.steps,
                  "stages_ms": plain["stages"],
                  "roofline": {"kernel": "svd_kernel<SVD_PROX> (one-sided Jacobi + SVT)",
                               "bound": "alu", "achieved": jflops / (jt / 1e3) / 1e12,
                               "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": jflops / (jt / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                               "model": "sum over slices of sweeps*n(n-1)/2*40*m flops",
                               "sweeps_mean": float(plain["sweeps"].mean())}}

    # --- autotuned plain path: the Jacobi CTA shape chosen by timing the candidates on this
    # batch's own Fourier slices; the chosen shape stays set for the learned step's fallback
    shape = None
    if not args.no_autotune:
        t_at = time.perf_counter()
        shape, tune_def_ms, tune_best_ms = tp.autotune_jacobi(Ys, taus, reps=2)
        t_at = time.perf_counter() - t_at
        tuned = time_prox(tp, args, Ys, Xs, taus, descs, "jacobi", world, barrier, device)
        tuned_value = job_throughput(slices_all, args.steps, tuned["ms"])
        tdev = 0.0
        for Xt, Xp in zip(Xs, X_plain):
            d = float(torch.linalg.vector_norm(Xt - Xp) /
                      torch.linalg.vector_norm(Xp).clamp_min(1e-30))
            tdev = max(tdev, d)
        tj = jacobi_model_flops(shapes, tuned["sweeps"]) / (tuned["stages"]["jacobi_svt"] / 1e3) / 1e12
        plain_line["autotuned"] = {
            "shape": shape, "tune_seconds": t_at,
            "tune_ms_per_pass": {"default": tune_def_ms, "chosen": tune_best_ms},
            "value": tuned_value, "ms_per_step": tuned["ms"] / args.steps,
            "stages_ms": tuned["stages"], "max_rel_dev_vs_default": tdev,
            "jacobi_tflops": tj, "jacobi_frac": tj / FP32_PEAK_TFLOPS}
    best_plain = max(plain_value, plain_line["autotuned"]["value"]) if shape else plain_value

    # --- learned path: proposer trained (untimed) on separately seeded batches
    t_train = time.perf_counter()
    train_Y, train_tau = [], []
    for sd in range(args.train_batches):
        _, Yt, tt, _, _, _ = make_batch(tp, synth, 512, 1000 + 97 * rank + sd, device)
        train_Y += Yt
        train_tau += tt
    train_slices = sum(Y.shape[2] // 2 + 1 for Y in train_Y)
    mse = tp.proposer_train(train_Y, train_tau, steps=300, seed=11)
    del train_Y
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    learned = time_prox(tp, args, Ys, Xs, taus, descs, "learned", world, barrier, device,
                        clocks=Clocks(local))
    dev = 0.0
    for Xl, Xp in zip(Xs, X_plain):
        d = float(torch.linalg.vector_norm(Xl - Xp) / torch.linalg.vector_norm(Xp).clamp_min(1e-30))
        dev = max(dev, d)
    plan = plan_leg(args, tp, Ys, Xs, taus, descs, slices) if world == 1 else None
    ms_max = learned["ms"]
    value = job_throughput(slices_all, args.steps, ms_max)
    st = learned["stages"]
    sk_flops = sketch_model_flops(shapes, learned["widths"])
    sk_tflops = sk_flops / (st["sketch_svt"] / 1e3) / 1e12
    sk_tflops_one = sketch_model_flops(shapes, learned["widths"], one_product=True) / \
        (st["sketch_svt"] / 1e3) / 1e12
    fb = learned["flags"]
    # the learned method's fallback launches are never split by CTA size
    lshape = dict(shape, split_launches=0) if shape else shape
    groups = svd_launch_groups([(a, b) for a, b, _ in shapes], lshape)
    dominant = "sketch_svt" if st["sketch_svt"] >= st["jacobi_svt"] else "jacobi_svt"
    if dominant == "sketch_svt":
        roof = {"kernel": "sketch_svt_kernel (randomized range finder + small Jacobi SVD + SVT)",
                "bound": "alu", "achieved": sk_tflops_one, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": sk_tflops_one / FP32_PEAK_TFLOPS,
                "count": "randomized SVD work: 8*n1*n2*l flops per sketched slice (l = k + p, "
                         "the sketch width)",
                "work_model": {"achieved": sk_tflops, "frac": sk_tflops / FP32_PEAK_TFLOPS,
                               "count": "work done per sketched slice 8*n1*n2*(6*l+4) flops: five "
                                        "width-l products, four mat-vecs, the W update"},
                "traffic": SKETCH_DRAM_PER_SPEC_BYTE * spec_bytes,
                "traffic_note": "DRAM bytes of the sketch stage per step, scaled by half-spectrum "
                                "bytes from an ncu capture of the 160-tensor batch (algorithmic: "
                                "read and write each slice once, %.0f MB)" % (2 * spec_bytes / 1e6)}
    else:
        fl = jacobi_model_flops(shapes, learned["sweeps"] * (fb == 1))
        a = fl / (st["jacobi_svt"] / 1e3) / 1e12
        roof = {"kernel": "svd_kernel<SVD_PROX> on the fallback slices", "bound": "alu",
                "achieved": a, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": a / FP32_PEAK_TFLOPS, "traffic": None,
                "model": "sum over fallback slices of sweeps*n(n-1)/2*40*m flops"}
    dft_gbs = (nbytes + spec_bytes) / (st["rfft"] / 1e3) / 1e9
    idft_gbs = (nbytes + spec_bytes) / (st["irfft"] / 1e3) / 1e9

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "method": "learned rank proposer + randomized SVT, "
                       "Jacobi fallback", "tensors": len(specs), "free_slices": slices,
                       "seed": rank, "input_bytes": nbytes,
                       "l2": "inputs larger than L2 (%.2f GB in + out per step)" % (2 * nbytes / 1e9)},
            "gpu_launches": (LEARNED_FIXED_LAUNCHES + 2 * dft_launches([n3 for _, _, n3 in shapes])
                             + groups) * args.steps,
            "roofline": roof,
            "stages_ms": st,
            "learned": {"fallback_fraction": float((fb == 1).mean()),
                        "max_rel_dev_vs_plain": dev, "train_slices": train_slices,
                        "train_mse": mse, "train_seconds": t_train,
                        "sketch_width_mean": float(learned["widths"][fb == 0].mean()) if (fb == 0).any() else 0.0,
                        "vs_plain": value / best_plain},
            "plain": plain_line,
            "plan": plan,
            "dft_gbs": {"rfft": dft_gbs, "irfft": idft_gbs}}

    line["clocks"] = learned["clocks"]
    line["peaks"] = {"source": PEAKS["source"], "hbm_gbs": HBM_PEAK_GBS,
                     "bf16_tflops": BF16_PEAK_TFLOPS, "tf32_tflops": TF32_PEAK_TFLOPS,
                     "fp32_alu_tflops": FP32_PEAK_TFLOPS}
    if shape:
        tp.jacobi_shape_set(None)  # the other legs run at the default shape
    if not args.no_e2e:
        line["e2e"] = e2e_leg(args, tp, Ys, Xs, taus, descs, slices, world, barrier, device)
    if not args.no_tprod and rank == 0:
        line["tprod"] = tprod_leg(args, tp, synth, device)
        line["tran"] = line["tprod"].pop("tran")
    if not args.no_factor and rank == 0:
        line["factor"] = factor_leg(args, tp, synth, device)
    if not args.no_trpca and rank == 0:
        line["trpca"] = trpca_leg(args, tp, synth, device)
    if not args.no_stream and rank == 0:
        try:
            line["stream"] = stream_leg(args, tp, synth, device)
        except tp.TpError as e:  # reported in the line; the measured legs above stand
            line["stream"] = {"error": str(e)}
    if rank == 0:
        # the oracle on the GPU's own inputs: timed for the baseline, and its results give the
        # plain and learned outputs' error at the bench configuration
        import numpy as np
        par = {"tensors": 0, "plain_max_rel": 0.0, "learned_max_rel": 0.0,
               "bound": {"plain": 1e-5, "learned": 1e-4},
               "note": "relative Frobenius error per tensor against the FP64 oracle on the "
                       "same FP32 inputs, over the tensors of the cpu_baseline sample"}

        def gpu_input(i):
            return tp.to_numpy(Ys[i])

        def check(i, W):
            nW = float(np.linalg.norm(W)) or 1.0
            for key, X in (("plain_max_rel", X_plain[i]), ("learned_max_rel", Xs[i])):
                par[key] = max(par[key], float(np.linalg.norm(tp.to_numpy(X) - W)) / nW)
            par["tensors"] += 1

        try:
            rate, sl, nt, secs = oracle_sample(specs, rank, args.cpu_seconds, inputs=gpu_input,
                                               check=check)
        except Exception as e:  # the baseline still prints without the check
            par = {"error": repr(e)}
            rate, sl, nt, secs = oracle_sample(specs, rank, args.cpu_seconds)
        line["parity_vs_oracle"] = par
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"FP64 oracle prox_tnn on tensors 0-{nt - 1} of the batch "
                                          f"({sl} free slices, {secs:.1f} s); numpy/LAPACK threads",
                                "single_core": oracle_single_core(rank, args.cpu_seconds / 3)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def plan_leg(args, tp, Ys, Xs, taus, descs, slices):
    """The learned step recorded once as a CUDA graph (tp_prox_plan) and replayed: device time
    per step, and host time per call against the direct batched call."""
    import torch
    direct_opts = tp.options(sync=False, method="learned")
    plan = tp.ProxPlan(Ys, taus, outs=Xs, opts=tp.options(sync=False, method="learned"))
    for _ in range(max(1, args.warmup)):
        plan.run()
    torch.cuda.synchronize()

    def timed(call):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        h0 = time.perf_counter()
        for _ in range(args.steps):
            call()
        host = (time.perf_counter() - h0) / args.steps
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps, host * 1e6

    ms, host_us = timed(plan.run)
    _, direct_us = timed(lambda: tp.prox_tnn_batched(Ys, taus, outs=Xs, opts=direct_opts,
                                                     descs=descs))
    plan.close()
    return {"ms_per_step": ms, "value": slices / (ms / 1e3), "unit": UNIT,
            "host_us_per_call": host_us, "direct_host_us_per_call": direct_us}


def e2e_leg(args, tp, Ys, Xs, taus, descs, slices, world, barrier, device):
    """The same batch through the host-buffer entry point: every step copies the inputs from
    page-locked host memory, runs the learned batched prox and copies the results back (the
    library overlapping its copies with its kernels part by part).  Consecutive steps are
    issued on two streams, as a serving loop would, so one step's copies also overlap the
    neighbouring steps' kernels.  Each step reads its own input buffer and writes its own
    output buffer (two sets, page-locked)."""
    import torch
    shapes = [tuple(Y.shape) for Y in Ys]
    sets = []
    for _ in range(2):
        _, hin = tp.pinned_tensors(shapes)
        _, hout = tp.pinned_tensors(shapes)
        for h, Y in zip(hin, Ys):
            h.copy_(Y.cpu())
        sets.append((hin, hout, tp.make_descs(hin, hout, taus)))
    streams = [torch.cuda.Stream(device), torch.cuda.Stream(device)]
    # --host-parts (default 1): with consecutive calls on two streams, each call's copies
    # already overlap the neighbouring calls' kernels, and a second part only adds its own
    # launch tails (7.6 against 8.9-9.3 ms per step measured side by side)
    opts = tp.options(sync=False, method="learned", host_parts=args.host_parts)

    def step(i):
        hin, hout, d = sets[i % 2]
        tp.prox_tnn_batched_host(hin, taus, outs=hout, opts=opts, descs=d,
                                 stream=streams[i % 2])

    # at least 8 warm-up steps: the first calls on two streams grow the stream-ordered pool and
    # the library's page-locked staging
    for i in range(max(8, args.warmup)):
        step(i)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream(device)
    barrier()
    t0.record(cur)
    for st in streams:
        st.wait_event(t0)
    for i in range(args.steps):
        step(i)
    for st in streams:
        ev = torch.cuda.Event()
        ev.record(st)
        cur.wait_event(ev)
    t1.record(cur)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(t0.elapsed_time(t1), device)
    nb = sum(4 * Y.numel() for Y in Ys)
    return {"value": job_throughput(sum_over_ranks(slices, device), args.steps, ms), "unit": UNIT,
            "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
            "api": f"tp_prox_tnn_batched_host (host_parts={args.host_parts}) on two alternating streams "
                   "(page-locked host tensors; each step's copies overlap the neighbouring "
                   "steps' kernels)"}


HBM_PEAK_GBS = PEAKS["hbm_gbs"]          # measured copy bandwidth
BF16_PEAK_TFLOPS = PEAKS["bf16_tflops"]  # measured dense bf16, burst
TF32_PEAK_TFLOPS = 1051.2   # measured: torch.matmul 8192^3 FP32 with TF32 allowed, this GB300 pool


def tprod_oracle_sample(A32, B32, seconds):
    """The FP64 oracle on the t-product workload, bounded (host cores, numpy/LAPACK threads):
      literal   Eq. 9 entry by entry (a block row of bcirc(A) times a column of unfold(B),
                `tprod_entries`) on seeded random (i, l, k) until `seconds`, extrapolated to
                all n1*l*n3 entries; the sampled values are kept as the reference for the GPU
                results' error;
      dft       Eq. 10 on all n3 slices (`tprod_fourier`) for rows 0..63 of A and columns
                0..63 of B, extrapolated to the whole product by n1*l / (64*64) (the slice
                products dominate its cost).
    Returns a dict with the timings, the sampled indices and reference values."""
    import numpy as np

    from oracle import tproduct as O
    A = np.asarray(A32, dtype=np.float64)
    B = np.asarray(B32, dtype=np.float64)
    n1, n2, n3 = A.shape
    l = B.shape[1]
    h = n3 // 2 + 1
    nreal = 2 if n3 % 2 == 0 else 1
    flops = (2.0 * nreal + 8.0 * (h - nreal)) * n1 * n2 * l
    rng = np.random.default_rng(20180619)
    idx, ref, t = [], [], 0.0
    while t < seconds or not idx:
        blk = np.stack([rng.integers(0, n1, 64), rng.integers(0, l, 64),
                        rng.integers(0, n3, 64)], axis=1)
        t0 = time.perf_counter()
        ref.append(O.tprod_entries(A, B, blk))
        t += time.perf_counter() - t0
        idx.append(blk)
    idx = np.concatenate(idx)
    ref = np.concatenate(ref)
    lit_s = t / len(idx) * n1 * l * n3
    m, ls = min(64, n1), min(64, l)
    t0 = time.perf_counter()
    O.tprod_fourier(A[:m], B[:, :ls])
    blk_s = time.perf_counter() - t0
    dft_s = blk_s * (n1 / m) * (l / ls)
    return {"cores": os.cpu_count(), "kind": "oracle", "useful_flops": flops,
            "literal": {"entries": int(len(idx)), "seconds": t, "extrapolated_s": lit_s,
                        "tflops_equiv": flops / lit_s / 1e12},
            "dft_domain": {"block": [m, n2, ls, n3], "seconds": blk_s, "extrapolated_s": dft_s,
                           "tflops_equiv": flops / dft_s / 1e12},
            "idx": idx, "ref": ref}


def sampled_rel_err(C, oracle):
    """||C[idx] - ref|| / ||ref|| over the oracle's sampled entries (C: an n1 x l x n3 tensor)."""
    import numpy as np
    import torch
    idx = torch.as_tensor(oracle["idx"], dtype=torch.long, device=C.device)
    got = C[idx[:, 0], idx[:, 1], idx[:, 2]].double().cpu().numpy()
    ref = oracle["ref"]
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def tprod_leg(args, tp, synth, device):
    """t-product of A n1 x n2 x n3 and B n2 x l x n3 (--gemm-shape, default 2048x1024x64 and
    1024x1024x64; one rank) in the three slice-GEMM arithmetics. Useful flops =
    (2 #real + 8 #complex slices) n1 n2 l; the split forms run 3x that on the tensor pipe."""
    import torch
    n1, n2, l, n3 = (int(v) for v in args.gemm_shape.split(","))
    g = synth.gemm(0, n1, n2, l, n3)
    A, B = tp.to_device(g["A"], device), tp.to_device(g["B"], device)
    try:
        oracle = tprod_oracle_sample(g["A"], g["B"], args.cpu_seconds / 3)
    except Exception as e:  # a host-side baseline; the GPU legs below stand without it
        oracle = {"error": repr(e)}
    del g
    C = tp.empty(n1, l, n3, device)
    h = n3 // 2 + 1
    nreal = 2 if n3 % 2 == 0 else 1
    flops = (2.0 * nreal + 8.0 * (h - nreal)) * n1 * n2 * l
    steps = max(3, min(args.steps, 10))
    out = {"workload": f"A {n1}x{n2}x{n3} * B {n2}x{l}x{n3}, N(0,1)", "flops": flops}
    for prec in ("fp32", "bf16x3", "3xtf32"):
        for _ in range(2):
            tp.tprod(A, B, out=C, opts=tp.options(precision=prec, sync=False))
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(tp.STAGE_EVENTS)]
               for _ in range(steps)]
        for s_ in evs:
            for e in s_:
                e.record()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for i in range(steps):
            tp.tprod(A, B, out=C, opts=tp.options(precision=prec, sync=False, stage_events=evs[i]))
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
        seg = lambda a, b: sum(s_[a].elapsed_time(s_[b]) for s_ in evs) / steps
        st = [seg(0, 1), seg(3, 4), seg(4, 5)]
        gemm_tflops = flops / (st[1] / 1e3) / 1e12
        if prec == "fp32":
            roof = {"bound": "alu", "achieved": gemm_tflops, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": gemm_tflops / FP32_PEAK_TFLOPS}
        else:
            peak = BF16_PEAK_TFLOPS if prec == "bf16x3" else TF32_PEAK_TFLOPS
            pipe = 3.0 * gemm_tflops
            how = ("the forward DFT writes the BF16 hi/lo operand planes, so the stage is the "
                   "GEMM kernel alone" if prec == "bf16x3" else
                   "stage includes the hi/lo split kernels")
            roof = {"bound": "tensor", "achieved": pipe, "peak": peak, "unit": "TFLOP/s",
                    "frac": pipe / peak, "note": "3 split MMAs per useful flop; " + how}
        out[prec] = {"tflops": flops / (ms / 1e3) / 1e12, "ms_per_call": ms,
                     "stages_ms": {"rfft": st[0], "gemm": st[1], "irfft": st[2]},
                     "gemm_useful_tflops": gemm_tflops, "gemm_roofline": roof}
        if "ref" in oracle:
            try:
                out[prec]["sampled_rel_err_vs_oracle"] = sampled_rel_err(C, oracle)
            except Exception as e:
                out[prec]["sampled_rel_err_vs_oracle"] = repr(e)
    oracle.pop("idx", None)
    oracle.pop("ref", None)
    out["oracle"] = oracle
    del C
    # tran (Def. 2.2) of A: a pure permutation, one read and one write of every entry
    AT = tp.empty(n2, n1, n3, device)
    for _ in range(2):
        tp.tran(A, out=AT)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        tp.tran(A, out=AT)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    nb = 8.0 * n1 * n2 * n3
    out["tran"] = {"workload": f"tran of A {n1}x{n2}x{n3} (FP32, {nb / 2 / 2**20:.0f} MiB)",
                   "ms_per_call": ms, "bytes": nb,
                   "roofline": {"bound": "hbm", "achieved": nb / (ms / 1e3) / 1e9,
                                "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                "frac": nb / (ms / 1e3) / 1e9 / HBM_PEAK_GBS}}
    del AT
    out["dft_long"] = dft_long_leg(tp, device)
    return out


def dft_long_leg(tp, device, n3s=(61, 64, 127, 128, 251, 256), tubes=1 << 20):
    """The tube DFTs alone at long tube lengths (the mixed call stream's n3 reaches 256): a
    t-product A * B with A tubes x 1 x n3 and B 1 x 1 x n3, timed by the library's stage events
    around its forward DFT (A and the one tube of B) and its inverse DFT (C); bytes are one
    read of the real tubes and one write of the half spectrum (or the reverse)."""
    import torch
    res = {}
    for n3 in n3s:
        A = tp.empty(tubes, 1, n3, device)
        A.normal_()
        B = tp.empty(1, 1, n3, device)
        B.normal_()
        C = tp.empty(tubes, 1, n3, device)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        for e in ev:
            e.record()
        o = tp.options(stage_events=ev)
        fw, iv = [], []
        for rep in range(4):
            tp.tprod(A, B, out=C, opts=o)
            torch.cuda.synchronize()
            if rep:
                fw.append(ev[0].elapsed_time(ev[1]))
                iv.append(ev[4].elapsed_time(ev[5]))
        nb = tubes * (4.0 * n3 + 8.0 * (n3 // 2 + 1))
        res[str(n3)] = {"fwd_gbs": nb / (min(fw) / 1e3) / 1e9, "inv_gbs": nb / (min(iv) / 1e3) / 1e9,
                        "fwd_ms": min(fw), "inv_ms": min(iv)}
        del A, B, C
    return {"workload": f"{tubes} tubes per length, N(0,1); stage events include the job-table "
                        "upload (a few microseconds)", "lengths": res}


def factor_leg(args, tp, synth, device):
    """tinv on 128x128x302 and economy tqr on 128x64x302 (shifted-identity / N(0,1) inputs):
    302 tubes give 152 independent Fourier slices, one CTA per SM.  Model flops per complex
    slice: Gauss-Jordan 8 n^3; Householder QR plus the economy Q, 16 (n1 n2^2 - n2^3 / 3)
    (half that on the two real slices is not credited)."""
    import torch
    out = {}
    steps = max(3, min(args.steps, 10))
    cases = {
        "tinv": (synth.shifted_square(128, 302, 0), 8.0 * 128 ** 3,
                 lambda A, o: tp.tinv(A, opts=o)),
        "tqr": (synth.gaussian(128, 64, 302, 0), 16.0 * (128 * 64 ** 2 - 64 ** 3 / 3.0),
                lambda A, o: tp.tqr(A, econ=True, opts=o)),
    }
    for name, (host, slice_flops, call) in cases.items():
        A = tp.to_device(host, device)
        n1, n2, n3 = host.shape
        h = n3 // 2 + 1
        for _ in range(3):
            call(A, tp.options(sync=False, econ=(name == "tqr")))
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(tp.STAGE_EVENTS)]
               for _ in range(steps)]
        for s_ in evs:          # torch creates the CUDA event at its first record
            for e in s_:
                e.record()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for i in range(steps):
            call(A, tp.options(sync=False, econ=(name == "tqr"), stage_events=evs[i]))
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
        seg = lambda a, b: sum(s_[a].elapsed_time(s_[b]) for s_ in evs) / steps
        k_ms = seg(3, 4)
        tflops = slice_flops * h / (k_ms / 1e3) / 1e12
        out[name] = {"shape": [n1, n2, n3], "slices": h, "slices_per_s": h / (ms / 1e3),
                     "ms_per_call": ms,
                     "stages_ms": {"rfft": seg(0, 1), "slice_kernel": k_ms, "irfft": seg(4, 5)},
                     "roofline": {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS,
                                  "unit": "TFLOP/s", "frac": tflops / FP32_PEAK_TFLOPS}}
        del A
    return out


def trpca_problem(tp, synth, seed, device):
    """L0 = P * Q (240x320x100, rank 10) at unit RMS; X = L0 with 10% of its entries (linear
    column-major positions) shifted by U[-5, 5]."""
    import torch
    g = synth.trpca(seed)
    L0 = tp.tprod(tp.to_device(g["P"], device), tp.to_device(g["Q"], device))
    L0.mul_(1.0 / float(L0.pow(2).mean().sqrt()))
    X = L0.clone()
    flat = X.permute(2, 1, 0).reshape(-1)           # column-major element order, a view
    flat[torch.from_numpy(g["pos"]).to(device)] += torch.from_numpy(g["val"]).to(device)
    return L0, X, g["tau"]


def trpca_admm(tp, X, lam, method, iters=50, record=None):
    """ADMM for min ||L||_* + lam ||E||_1 s.t. L + E = X with the tensor nuclear norm of
    Def. 2.9: L <- prox_tnn(X - E - Y/mu, 1/mu) (the library call), E <- soft(X - L - Y/mu,
    lam/mu), Y <- Y + mu (L + E - X), mu <- min(1.1 mu, 1e10), mu0 = 1e-3."""
    import torch
    n1, n2, n3 = X.shape
    L = tp.empty(n1, n2, n3, X.device)
    E = torch.zeros_like(X)
    Y = torch.zeros_like(X)
    T = tp.empty(n1, n2, n3, X.device)
    mu = 1e-3
    flags = torch.zeros((n3 // 2 + 1,), dtype=torch.int32, device=X.device)
    fb = torch.zeros((), dtype=torch.int64, device=X.device)
    opts = tp.options(sync=False, method=method,
                      slice_flags_out=flags if method == "learned" else None)
    for _ in range(iters):
        torch.sub(X, E, out=T)
        T.sub_(Y, alpha=1.0 / mu)
        if record is not None:
            record.append((T.clone(), 1.0 / mu))
        tp.prox_tnn(T, 1.0 / mu, out=L, opts=opts)
        if method == "learned":
            fb += flags.sum()
        torch.sub(X, L, out=T)
        T.sub_(Y, alpha=1.0 / mu)
        E.copy_(torch.sign(T) * torch.clamp(T.abs() - lam / mu, min=0.0))
        Y.add_(L + E - X, alpha=mu)
        mu = min(1.1 * mu, 1e10)
    return L, int(fb) / (iters * (n3 // 2 + 1))


def trpca_leg(args, tp, synth, device):
    import torch
    L0, X, lam = trpca_problem(tp, synth, 0, device)
    n1, n2, n3 = X.shape
    h = n3 // 2 + 1
    iters = 50
    out = {"workload": "240x320x100, rank 10 at unit RMS, 10% corrupted by U[-5,5]; 50 ADMM "
                       "iterations, mu0 = 1e-3, rho = 1.1, lambda = 1/sqrt(320*100)",
           "slices_per_call": h, "iterations": iters}
    # proposer for this loop: plain-path iterates of another draw label its training set
    _, Xt, _ = trpca_problem(tp, synth, 1, device)
    rec = []
    trpca_admm(tp, Xt, lam, "jacobi", iters, record=rec)
    t0 = time.time()
    mse = tp.proposer_train([r[0] for r in rec], [r[1] for r in rec], steps=300, seed=2)
    out["train"] = {"slices": len(rec) * h, "mse": mse, "seconds": time.time() - t0}
    del rec, Xt
    for method in ("jacobi", "learned"):
        trpca_admm(tp, X, lam, method, 3)          # warm-up
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        L, fbf = trpca_admm(tp, X, lam, method, iters)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        err = float((L - L0).norm() / L0.norm())
        out[method] = {"ms": ms, "ms_per_iteration": ms / iters,
                       "slices_per_s": iters * h / (ms / 1e3), "L_rel_err": err}
        if method == "learned":
            out[method]["fallback_fraction"] = fbf
    out["learned_vs_plain"] = out["jacobi"]["ms"] / out["learned"]["ms"]
    return out


def stream_leg(args, tp, synth, device):
    """A bounded sample of the mixed call stream: the first `stream_calls` calls of the seeded
    stream (prox_tnn or tprod by a fair coin; n1, n2 up to 512, n3 up to 256, every operand a
    rank-4..40 t-product plus N(0, 0.02^2) noise), run two ways on the same tensors:
      plain     every call on its own in stream order: tp_prox_tnn (Jacobi, FP32) and
                tp_tprod (FP32 slice GEMMs);
      combined  the stream in windows of `stream_window` consecutive calls: the window's prox
                calls as one replayed batched plan (CUDA graph) with the learned method, its
                tprod calls with BF16x3 tensor-core slice GEMMs.
    Operand data is drawn on the device (seeded torch generator; sizes from the generator
    module) and formed with the library's t-product, untimed. The proposer is retrained on the
    plain path's labels for prox calls of another draw of the stream."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(20180619)

    def randn(n1, n2, n3, std=1.0):
        return (torch.randn(n3, n2, n1, generator=gen, device=device) * std).permute(2, 1, 0)

    def low_rank(sp):
        X = tp.tprod(randn(sp.n1, sp.r, sp.n3), randn(sp.r, sp.n2, sp.n3))
        X.add_(randn(sp.n1, sp.n2, sp.n3, sp.noise))
        return X

    # proposer for these sizes and ranks
    t0 = time.time()
    tcalls = [c for c in synth.stream_specs(8 * args.stream_calls, seed=1) if c.op == "prox"][:96]
    tY = [low_rank(c.a) for c in tcalls]
    mse = tp.proposer_train(tY, [c.a.tau for c in tcalls], steps=300, seed=3)
    train = {"tensors": len(tY), "slices": sum(Y.shape[2] // 2 + 1 for Y in tY), "mse": mse,
             "seconds": time.time() - t0}
    del tY

    calls = synth.stream_specs(args.stream_calls, seed=0)
    data = []
    for c in calls:
        if c.op == "prox":
            Y = low_rank(c.a)
            data.append({"Y": Y, "Xp": tp.empty(*Y.shape, device=device),
                         "Xc": tp.empty(*Y.shape, device=device)})
        else:
            A, B = low_rank(c.a), low_rank(c.b)
            data.append({"A": A, "B": B, "Cp": tp.empty(c.a.n1, c.b.n2, c.a.n3, device=device),
                         "Cc": tp.empty(c.a.n1, c.b.n2, c.a.n3, device=device)})
    torch.cuda.synchronize()
    prox_idx = [i for i, c in enumerate(calls) if c.op == "prox"]
    tprod_idx = [i for i, c in enumerate(calls) if c.op == "tprod"]
    prox_slices = sum(calls[i].a.n3 // 2 + 1 for i in prox_idx)
    tprod_flops = 0.0
    for i in tprod_idx:
        a, b = calls[i].a, calls[i].b
        h = a.n3 // 2 + 1
        nreal = 2 if a.n3 % 2 == 0 else 1
        tprod_flops += (2.0 * nreal + 8.0 * (h - nreal)) * a.n1 * a.n2 * b.n2

    o_plain_p = tp.options(sync=False)
    o_plain_t = tp.options(sync=False)
    o_tc = tp.options(precision="bf16x3", sync=False)

    def plain_pass():
        for i, c in enumerate(calls):
            d = data[i]
            if c.op == "prox":
                tp.prox_tnn(d["Y"], c.a.tau, out=d["Xp"], opts=o_plain_p)
            else:
                tp.tprod(d["A"], d["B"], out=d["Cp"], opts=o_plain_t)

    W = args.stream_window
    windows, flags = [], []
    for w0 in range(0, len(calls), W):
        w = range(w0, min(w0 + W, len(calls)))
        px = [i for i in w if calls[i].op == "prox"]
        plan = None
        if px:
            f = torch.zeros(sum(calls[i].a.n3 // 2 + 1 for i in px), dtype=torch.int32,
                            device=device)
            flags.append(f)
            plan = tp.ProxPlan([data[i]["Y"] for i in px], [calls[i].a.tau for i in px],
                               outs=[data[i]["Xc"] for i in px],
                               opts=tp.options(sync=False, method="learned", slice_flags_out=f))
        windows.append((plan, [i for i in w if calls[i].op == "tprod"]))

    def combined_pass():
        for plan, tps in windows:
            if plan is not None:
                plan.run()
            for i in tps:
                tp.tprod(data[i]["A"], data[i]["B"], out=data[i]["Cc"], opts=o_tc)

    reps = 1 if len(calls) >= 200 else 2
    out = {"workload": f"first {len(calls)} calls of the seeded mixed stream (prox_tnn or tprod "
                       "by a fair coin; n1,n2~U{16..512}, n3~U{4..256}, l~U{16..512}, tubal rank "
                       "r~U{4..40} + N(0,0.02^2) noise, tau = 2x noise level)",
           "calls": len(calls), "prox_calls": len(prox_idx), "tprod_calls": len(tprod_idx),
           "prox_slices": prox_slices, "tprod_flops": tprod_flops, "window": W,
           "proposer_train": train}
    for name, fn in (("plain", plain_pass), ("combined", combined_pass)):
        fn()  # warm-up
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        out[name] = {"ms_per_pass": ms, "calls_per_s": len(calls) / (ms / 1e3)}
    fl = torch.cat(flags).cpu() if flags else torch.zeros(0)
    out["combined"]["prox_fallback_fraction"] = float((fl == 1).float().mean()) if fl.numel() else 0.0
    out["combined"]["api"] = ("tp_prox_plan_run (learned) per window + tp_tprod BF16x3; "
                              f"{sum(1 for p, _ in windows if p is not None)} plans")
    out["plain"]["api"] = "tp_prox_tnn (Jacobi) and tp_tprod (FP32), one call each"
    out["speedup"] = out["plain"]["ms_per_pass"] / out["combined"]["ms_per_pass"]

    def reldev(x, y):
        return float(torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(y).clamp_min(1e-30))

    out["max_rel_dev_vs_plain"] = {
        "prox": max((reldev(data[i]["Xc"], data[i]["Xp"]) for i in prox_idx), default=0.0),
        "tprod": max((reldev(data[i]["Cc"], data[i]["Cp"]) for i in tprod_idx), default=0.0)}
    for plan, _ in windows:
        if plan is not None:
            plan.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_tp(args)


if __name__ == "__main__":
    sys.exit(main())
