"""Benchmark of the emulated DGEMM (Ozaki scheme II, fast mode, Algorithm 2 scaling) on GB300.

Workload: square FP64 GEMM m = n = k = 16384, entries (rand - 0.5) exp(phi randn) with phi = 1
(the paper's generator, eq. random-matrix-generation), N = 14 moduli.  One step = one
ozaki2_dgemm call: scaling, conversion, residue GEMMs, CRT.  Metric: effective TFLOPS =
2 m n k / t (eq. tflops).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (torchrun) every rank runs its own independent problem on its own GPU (weak scaling);
the only cross-rank traffic is the timing reduction.  --impl reference times the CPU oracle on a
bounded block of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIZE = 16384
PHI = 1.0
NUM_MODULI = 16
SGEMM_MODULI = 8
METRIC = "Ozaki-II DGEMM effective TFLOPS at stated error vs cuBLAS DGEMM; p50/p99 lat"
FP64_NOMINAL_TFLOPS = 1.25  # GB300's dense FP64 rate (nominal)
WORKLOAD = f"square FP64 GEMM m=n=k={SIZE}, phi={PHI}, N={NUM_MODULI} moduli"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def hbm_peak():
    """Measured HBM copy bandwidth in GB/s (the fallback figure when no measurement exists)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def stage_rooflines(m, n, k, N, esz, stages_ms, hbm_gbs, scaling="proposed", beta_reads=False):
    """Achieved GB/s of the HBM-side stages from their algorithmic bytes and the library's stage
    times: scale reads each input element once (esz bytes); convert reads it again and writes N
    bf16 residues (2N bytes); the reconstruction reads N residue bytes per entry and writes the
    entry (esz bytes, plus esz more read when beta != 0).  Accurate mode's scale stage also
    builds and multiplies A-bar and B-bar, so its bytes are not those of a stream and it is
    left out.  frac is against the measured HBM copy bandwidth."""
    elems = m * k + k * n
    out = {}
    work = {"convert": elems * (esz + 2 * N),
            "crt": m * n * (N + esz + (esz if beta_reads else 0))}
    if scaling != "accurate":
        work["scale"] = elems * esz
    for name, nbytes in work.items():
        ms = stages_ms.get(name)
        if not ms:
            continue
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"algorithmic_bytes": nbytes, "ms": ms, "achieved_gbs": gbs,
                     "frac_of_hbm": gbs / hbm_gbs}
    if "scale" in out:
        # one upward-rounded FP64 FMA per element: the stage's other bound on GB300, against
        # the nominal FP64 rate (no measured figure exists for it)
        tflops = 2.0 * elems / (out["scale"]["ms"] * 1e-3) / 1e12
        out["scale"].update(fp64_tflops=tflops, frac_of_fp64_nominal=tflops / FP64_NOMINAL_TFLOPS)
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d.get("bf16_tflops"), d.get("bf16_tflops_sustained"), "measured"
    except Exception:
        return 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.start = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up holds the driver for a while: let it finish before the timed
            # region begins, and count only the samples taken from then on
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.start = len(self.lines)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.start:] or self.lines
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() and args.impl != "reference" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ------------------------------------------------------------------------------- oracle arm
def oracle_block_tflops(A_h, B_h, m, n, k, N, rows: int, cols: int):
    """Time the CPU oracle on a rows x cols block of C (full k), return (TFLOPS, seconds)."""
    import numpy as np

    import oracle

    I = np.linspace(0, m - 1, rows).astype(np.int32)
    J = np.linspace(0, n - 1, cols).astype(np.int32)
    t0 = time.perf_counter()
    if A_h.dtype == np.float32:
        oracle.sgemm_block(A_h, B_h, k, N, I, J)
    else:
        oracle.dgemm_block(A_h, B_h, m, n, k, N, I, J)
    dt = time.perf_counter() - t0
    return 2.0 * rows * cols * k / dt / 1e12, dt


def run_reference(args, world, rank):
    """--impl reference: the oracle as it stands, on host cores, bounded blocks of the workload."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synthetic

    oracle.build()
    m = n = k = args.size
    rows = cols = min(args.ref_block, args.size)
    # The oracle needs only the sampled rows of A and columns of B; the rest is never read, so
    # draw just those lines from the paper's generator (independent streams per line).
    I = np.linspace(0, m - 1, rows).astype(np.int32)
    J = np.linspace(0, n - 1, cols).astype(np.int32)
    A_rows = synthetic.paper_matrix(rows, k, PHI, synthetic.seed_for(2, 1, 1))  # rows x k block
    B_cols = synthetic.paper_matrix(k, cols, PHI, synthetic.seed_for(2, 1, 2))
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.dgemm_block(A_rows, B_cols, rows, cols, k, args.moduli, np.arange(rows),
                           np.arange(cols))
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    total = sum(times)
    flops = 2.0 * rows * cols * k
    value = flops * len(times) / total / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (int64 residue products, 256-bit CRT)",
        "data": "synthetic",
        "config": {"workload": f"square FP64 GEMM m=n=k={m}, phi={PHI}, N={args.moduli} moduli",
                   "sample": f"{rows}x{cols} block" if rows < m else "full"},
        "cpu_baseline": {"value": value, "unit": "TFLOPS", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": (f"{rows}x{cols} block of C (full k={k}) per step" if rows < m
                                    else "the full product per step")},
        "e2e": {"value": value, "unit": "TFLOPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    del I, J
    print(json.dumps(line), flush=True)


def run_calibrate(args):
    """The accuracy table of the autotuner, measured against the double-double reference of the
    oracle (on a random 64 x 64 block of C per problem) instead of the emulation with N = 20:
    for each size class (square problems of the class edge, m = n capped at 4096) and each
    phi, the maximum relative error of the emulation for N = 8..20 and of cuBLAS DGEMM.  Writes
    the table to --calibration-out (the package's calibration file is this output)."""
    import numpy as np
    import torch

    import oracle
    from paper_2606_29129_gb300 import autotune

    oracle.build()
    rng = np.random.default_rng(17)
    torch.backends.cuda.matmul.allow_tf32 = False

    def dd_reference(A, B, m, n, k):
        I = np.sort(rng.choice(m, size=min(64, m), replace=False)).astype(np.int32)
        J = np.sort(rng.choice(n, size=min(64, n), replace=False)).astype(np.int32)
        hi, _ = oracle.dd_block(A.cpu().numpy(), B.cpu().numpy(), k, I, J)
        dev = A.device
        return (torch.from_numpy(I.astype(np.int64)).to(dev),
                torch.from_numpy(J.astype(np.int64)).to(dev), torch.from_numpy(hi).to(dev))

    t0 = time.perf_counter()
    table = autotune.calibrate(reference=dd_reference)
    out = {"table": autotune.table_to_json(table),
           "how": "bench.py --calibrate: square problems m = n = min(k, 4096) at each class edge "
                  "k, phi in {0.5, 1, 2}, maximum relative error on a random 64 x 64 block of C "
                  "against the double-double reference (TwoProd/TwoSum accumulation)",
           "seconds": time.perf_counter() - t0}
    if args.calibration_out:
        with open(args.calibration_out, "w") as fh:
            json.dump(out, fh, indent=1)
    print(json.dumps({"mode": "calibration", **out}), flush=True)


def run_tune_tiles(args):
    """Residue-GEMM configuration per size class by timing: kernel variant (128 x 256 tiles on
    one SM, or 256 x 256 on an SM pair) and K chunk, for square DGEMMs of each size."""
    from paper_2606_29129_gb300 import autotune

    with ClockSampler(0) as clocks:
        table = autotune.tune_tiles(sizes=tuple(args.tune_sizes), N=args.moduli,
                                    chunks=tuple(args.tune_chunks),
                                    groups=tuple(args.tune_groups))
    print(json.dumps({"mode": "tile_tuning", "N": args.moduli,
                      "table": autotune.tiles_to_json(table), "clocks": clocks.summary(),
                      "variants": {"1": "128 x 256 tiles, one CTA per SM",
                                   "2": "256 x 256 tiles on SM pairs"}}), flush=True)


def run_reference_batched(args):
    """--impl reference --batched: the oracle over every problem of the batched workload, full,
    on host cores (the GPU run's problem sizes, entries drawn on the host; N = 15, the moduli
    count the autotuner gives most of them)."""
    import numpy as np

    import oracle

    oracle.build()
    items = batched_problems(args.batch, seed=4, device="cpu")
    N = 15
    flops = sum(2.0 * it["m"] * it["n"] * it["k"] for it in items)
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for p in items:
            oracle.dgemm(p["A"].numpy(), p["B"].numpy(), p["m"], p["n"], p["k"], N)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = flops * len(times) / total / 1e12
    print(json.dumps({
        "impl": "reference", "mode": "batched",
        "metric": "batched Ozaki-II DGEMM effective TFLOPS (sum 2mnk / time)", "value": value,
        "unit": "TFLOPS", "steps": args.steps, "warmup": args.warmup,
        "ms_per_batch": 1e3 * total / len(times), "dtype": "f64 (int64 residue products, 256-bit CRT)",
        "config": {"workload": f"{args.batch} problems, m, n, k log-uniform in [64, 2048], phi in "
                               "{0.5, 1} alternating", "n_per_item": N},
        "cpu_baseline": {"value": value, "unit": "TFLOPS", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": "every problem, full"},
    }), flush=True)


# ------------------------------------------------------------------------------- GPU arm
def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    import synthetic
    from paper_2606_29129_gb300 import ozaki2 as oz

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, n, k = args.shape if args.shape else (args.size,) * 3
    N = args.moduli
    f32 = args.dtype == "f32"
    seed_a = synthetic.seed_for(2, 1, 1) + 100 * rank
    seed_b = synthetic.seed_for(2, 1, 2) + 100 * rank
    A = synthetic.paper_matrix_torch(m, k, PHI, seed_a, device=dev)   # column-major m x k
    B = synthetic.paper_matrix_torch(k, n, PHI, seed_b, device=dev)   # column-major k x n
    if f32:
        A, B = A.float(), B.float()
    C = torch.empty((n, m), dtype=A.dtype, device=dev)
    gemm = oz.ozaki2_sgemm if f32 else oz.ozaki2_dgemm
    h = oz.Handle()
    h.set_timing(True)
    scaling = {"proposed": oz.SCALING_PROPOSED, "fast": oz.SCALING_FAST,
               "accurate": oz.SCALING_ACCURATE}[args.scaling]
    h.set_option(oz.OPT_SCALING, scaling)

    def step():
        rc = gemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, N, h)
        if rc:
            raise oz.Ozaki2Error(gemm.__name__, rc)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if h.status():
        raise RuntimeError("device status flags raised during warm-up")

    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stage_ms = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            stage_ms.append(h.timing())   # waits for this step's events
        t1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    total_ms = t0.elapsed_time(t1)
    step_ms = sorted(a.elapsed_time(b) for a, b in ev)
    total_ms = max_over_ranks(total_ms, world)
    flops_step = 2.0 * m * n * k
    value = flops_step * world * args.steps / (total_ms * 1e-3) / 1e12
    status = h.status()

    # dominant kernel: the residue GEMMs (tensor-bound), timed live by the library's events
    gemm_ms = statistics.mean(s[2] for s in stage_ms)
    gemm_flops = 2.0 * N * m * n * k
    burst, sustained, src = peaks()
    achieved = gemm_flops / (gemm_ms * 1e-3) / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": sustained, "unit": "TFLOP/s",
                "frac": achieved / sustained if sustained else None,
                # DRAM bytes per launch from an ncu capture of the current kernel, when given
                "traffic": args.gemm_traffic,
                "algorithmic_bytes": 2.0 * N * (m * k + k * n) + N * m * n,
                "peak_source": f"bf16_tflops_sustained ({src}); kernel timed inside the step",
                "kernel": "residue_gemm_kernel (tcgen05 kind::f16, bf16 residues)"}
    stages = {name: statistics.mean(s[i] for s in stage_ms)
              for i, name in enumerate(["scale", "convert", "residue_gemm", "crt"])}
    hbm, hbm_src = hbm_peak()
    stage_bw = stage_rooflines(m, n, k, N, A.element_size(), stages, hbm, args.scaling)
    stage_bw["peak_gbs"] = hbm
    stage_bw["peak_source"] = f"hbm_gbs ({hbm_src})"

    clk = clocks.summary()
    if clk.get("sm_mhz"):
        # flops per second per SM clock: compares runs taken at different power-capped clocks
        roofline["tflops_per_ghz"] = achieved / (clk["sm_mhz"] / 1e3)
    extra = {}
    if rank == 0 and not args.profile_step:
        extra = accuracy_and_baselines(args, A, B, C, m, n, k, N, torch, np)
    e2e = (measure_e2e(args, oz, h, A, B, m, n, k, N, torch, gemm)
           if rank == 0 and not args.profile_step else None)
    if rank != 0:
        return
    square = m == n == k
    shape = f"m=n=k={m}" if square else f"m={m}, n={n}, k={k}"
    line = {
        "metric": METRIC if not f32 else METRIC.replace("DGEMM", "SGEMM"), "value": value,
        "unit": "TFLOPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("f32" if f32 else "f64") +
                 " emulated (bf16-held int8 residues on tcgen05, fp32 exact accumulate)",
        "data": "synthetic",
        "config": {"workload": f"{'square ' if square else ''}{'FP32' if f32 else 'FP64'} GEMM "
                               f"{shape}, phi={PHI}, N={N} moduli" +
                   ("" if args.scaling == "proposed" else f", {args.scaling} scaling"),
                   "m": m, "n": n, "k": k, "phi": PHI,
                   "num_moduli": N, "scaling": args.scaling,
                   "parallelism": f"replicas x{world} (independent problems)",
                   "l2": "A, B, C: {:.2f} GiB ({})".format(
                       (A.numel() + B.numel() + C.numel()) * A.element_size() / 2**30,
                       "larger than L2" if (A.numel() + B.numel() + C.numel()) *
                       A.element_size() > 129e6 else "not larger than L2")},
        "latency_ms": {"p50": step_ms[len(step_ms) // 2],
                       "p99": step_ms[min(len(step_ms) - 1, int(0.99 * len(step_ms)))],
                       "min": step_ms[0], "max": step_ms[-1]},
        "stages_ms": stages,
        "stage_bandwidth": stage_bw,
        "roofline": roofline,
        "clocks": clk,
        "gpu_launches": (9 if args.scaling == "accurate" else 5) * args.steps,
        "device_status": status,
        "e2e": e2e,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


def accuracy_and_baselines(args, A, B, C, m, n, k, N, torch, np):
    """Max relative error vs the double-double reference on a sampled block, the same for
    cuBLAS DGEMM (timed on the same inputs), and the oracle's CPU throughput on a block."""
    import oracle

    out = {}
    oracle.build()
    f32 = A.dtype == torch.float32
    A_h = A.cpu().numpy()
    B_h = B.cpu().numpy()
    C_h = C.cpu().numpy()
    rng = np.random.default_rng(1)
    I = np.sort(rng.choice(m, size=min(args.err_block, m), replace=False)).astype(np.int32)
    J = np.sort(rng.choice(n, size=min(args.err_block, n), replace=False)).astype(np.int32)
    hi, lo = oracle.dd_block(A_h.astype(np.float64), B_h.astype(np.float64), k, I, J)
    err, zeros = oracle.max_rel_error(C_h[np.ix_(J, I)], hi, lo)
    # cuBLAS DGEMM (native FP64) on the same inputs: C^T = B^T A^T in row-major terms
    At = A.view(k, m)    # row-major (k, m) = A^T
    Bt = B.view(n, k)    # row-major (n, k) = B^T
    torch.backends.cuda.matmul.allow_tf32 = False
    Cd = torch.matmul(Bt, At)   # (n, m) row-major = C column-major
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.cublas_reps):
        torch.matmul(Bt, At, out=Cd)
    e.record()
    torch.cuda.synchronize()
    cub_ms = s.elapsed_time(e) / args.cublas_reps
    cub_err, _ = oracle.max_rel_error(Cd.cpu().numpy()[np.ix_(J, I)], hi, lo)
    out["accuracy"] = {"max_rel_err": err, "zero_reference_entries": zeros,
                       "sample": f"{len(I)}x{len(J)} random block vs double-double"}
    out["cublas_sgemm" if f32 else "cublas_dgemm"] = {
        "tflops": 2.0 * m * n * k / (cub_ms * 1e-3) / 1e12, "ms": cub_ms, "max_rel_err": cub_err}
    if not args.no_cpu_baseline:
        # a block of about the same work as cpu_block^2 x 16384 (10-30 s of CPU time)
        side = max(32, int(args.cpu_block * math.sqrt(16384.0 / max(k, 1))))
        rows, cols = min(side, m), min(side, n)
        tf, dt = oracle_block_tflops(A_h, B_h, m, n, k, N, rows, cols)
        out["cpu_baseline"] = {"value": tf, "unit": "TFLOPS", "cores": oracle.num_threads(),
                               "kind": "oracle",
                               "sample": f"{rows}x{cols} block of C (full k={k}), {dt:.1f} s"}
    return out


def measure_e2e(args, oz, h, A, B, m, n, k, N, torch, gemm=None):
    """The same metric through the public API with host buffers: each step passes page-locked
    host A, B and C to the call, which by default copies A and B into device memory with a
    kernel and whose reconstruction kernel writes C straight into the host buffer
    (--host-copies 1: copy engines both ways, whose rate measured erratic on this part).  Every
    byte in and out crosses the host link inside the timed region."""
    gemm = gemm or oz.ozaki2_dgemm
    A_h = torch.empty(A.shape, dtype=A.dtype, pin_memory=True)
    B_h = torch.empty(B.shape, dtype=B.dtype, pin_memory=True)
    C_h = torch.empty((n, m), dtype=A.dtype, pin_memory=True)
    A_h.copy_(A)
    B_h.copy_(B)
    h.set_timing(False)

    def step():
        rc = gemm("N", "N", m, n, k, 1.0, A_h, m, B_h, k, 0.0, C_h, m, N, h)
        if rc:
            raise oz.Ozaki2Error(gemm.__name__, rc)

    if args.host_copies is not None:
        h.set_option(oz.OPT_HOST_COPIES, args.host_copies)
    step()
    step()
    torch.cuda.synchronize()
    reps = max(4, min(args.steps, 10))
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    t0 = time.perf_counter()
    ev[0].record(stream)
    for i in range(reps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / reps
    h.set_timing(True)
    copies = args.host_copies if args.host_copies is not None else 0
    path = ("host A, B, C (page-locked) passed to the call: inputs staged into HBM by a kernel, "
            "the result written into host memory by the reconstruction" if copies == 0 else
            "host A, B, C (page-locked) passed to the call: inputs uploaded by a copy engine, "
            "the result reconstructed in HBM and downloaded by a copy engine")
    return {"value": 2.0 * m * n * k / (ms * 1e-3) / 1e12, "unit": "TFLOPS",
            "h2d_bytes_per_step": (A.numel() + B.numel()) * A.element_size(),
            "d2h_bytes_per_step": m * n * A.element_size(), "ms_per_step": ms, "steps": reps,
            "step_ms": [ev[i].elapsed_time(ev[i + 1]) for i in range(reps)],
            "host_copies": copies, "path": path,
            "clock": "host wall clock around the steps, synchronised on both sides"}


def batched_problems(count, seed, lo=64, hi=2048, device="cuda"):
    """The batched workload: `count` problems with m, n, k each log-uniform in [lo, hi], phi in
    {0.5, 1} alternating, seeded per item; column-major device inputs."""
    import numpy as np

    import synthetic

    rng = np.random.default_rng(seed)
    items = []
    for i in range(count):
        m, n, k = (int(np.exp(rng.uniform(np.log(lo), np.log(hi + 1)))) for _ in range(3))
        phi = (0.5, 1.0)[i % 2]
        A = synthetic.paper_matrix_torch(m, k, phi, 100000 + 2 * i, device=device)
        B = synthetic.paper_matrix_torch(k, n, phi, 100001 + 2 * i, device=device)
        items.append(dict(m=m, n=n, k=k, phi=phi, A=A, B=B))
    return items


def run_batched(args):
    """512 emulated DGEMMs in one grouped call replayed from a CUDA graph, N per item from the
    accuracy autotuner (smallest N not worse than cuBLAS DGEMM for the item's size class),
    against a per-request cuBLAS DGEMM loop on the same inputs."""
    import numpy as np
    import torch

    import oracle
    from paper_2606_29129_gb300 import autotune
    from paper_2606_29129_gb300 import ozaki2 as oz

    oracle.build()
    items = batched_problems(args.batch, seed=4)
    t0 = time.perf_counter()
    table = autotune.load_calibration()
    calib_src = "committed table (double-double reference)"
    if table is None:
        table = autotune.calibrate(ks=(64, 128, 256, 512, 1024, 2048))
        calib_src = "measured now (reference: the emulation with N = 20)"
    calib_s = time.perf_counter() - t0
    for it in items:
        it["N"] = autotune.choose_n(table, it["k"], margin=args.n_margin)
        it["C"] = torch.empty((it["n"], it["m"]), dtype=torch.float64, device="cuda")
    flops = sum(2.0 * it["m"] * it["n"] * it["k"] for it in items)
    probs = oz.problems_array([dict(m=it["m"], n=it["n"], k=it["k"], A=it["A"], lda=it["m"],
                                    B=it["B"], ldb=it["k"], C=it["C"], ldc=it["m"],
                                    num_moduli=it["N"]) for it in items])
    h = oz.Handle()
    h.set_option(oz.OPT_GRAPH, 1)

    def grouped():
        rc = oz.ozaki2_dgemm_grouped(len(items), probs, h)
        if rc:
            raise oz.Ozaki2Error("ozaki2_dgemm_grouped", rc)

    def ev_loop(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            fn()
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps

    # the K chunk of the grouped residue GEMM, then the tile width and chunk per size class, by
    # timing (results identical for every configuration)
    chunk_ms, chunk_best = autotune.tune_grouped_chunk(grouped, h)
    tiles = autotune.tune_grouped_tiles(grouped, h)
    t_grouped = ev_loop(grouped, args.steps)
    status = h.status()
    # per-request loops on the same inputs
    h2 = oz.Handle()

    def per_request_ozaki():
        for it in items:
            rc = oz.ozaki2_dgemm("N", "N", it["m"], it["n"], it["k"], 1.0, it["A"], it["m"],
                                 it["B"], it["k"], 0.0, it["C"], it["m"], it["N"], h2)
            if rc:
                raise oz.Ozaki2Error("ozaki2_dgemm", rc)

    def per_request_cublas():
        for it in items:
            torch.matmul(it["B"].view(it["n"], it["k"]), it["A"].view(it["k"], it["m"]),
                         out=it["Cd"])

    for it in items:
        it["Cd"] = torch.empty((it["n"], it["m"]), dtype=torch.float64, device="cuda")
    t_loop = ev_loop(per_request_ozaki, max(1, args.steps // 2))
    torch.backends.cuda.matmul.allow_tf32 = False
    t_cublas = ev_loop(per_request_cublas, 1)
    # accuracy: every item against the double-double reference on a sampled block
    grouped()
    torch.cuda.synchronize()
    per_request_cublas()
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    worst, worst_cub, worse_than_cublas = 0.0, 0.0, 0
    per_item = []
    side = args.err_side
    for idx, it in enumerate(items[: args.err_items]):
        A_h, B_h = it["A"].cpu().numpy(), it["B"].cpu().numpy()
        I = np.sort(rng.choice(it["m"], size=min(side, it["m"]), replace=False)).astype(np.int32)
        J = np.sort(rng.choice(it["n"], size=min(side, it["n"]), replace=False)).astype(np.int32)
        hi, lo = oracle.dd_block(A_h, B_h, it["k"], I, J)
        e1 = oracle.max_rel_error(it["C"].cpu().numpy()[np.ix_(J, I)], hi, lo)[0]
        e2 = oracle.max_rel_error(it["Cd"].cpu().numpy()[np.ix_(J, I)], hi, lo)[0]
        worst, worst_cub = max(worst, e1), max(worst_cub, e2)
        worse_than_cublas += e1 > e2
        per_item.append({"item": idx, "m": it["m"], "n": it["n"], "k": it["k"],
                         "phi": it["phi"], "N": it["N"], "max_rel_err": e1,
                         "cublas_max_rel_err": e2})
    if args.items_out:
        with open(args.items_out, "w") as fh:
            json.dump({"sample": f"{side}x{side} random block per item (all rows/columns when "
                                 "smaller) vs the double-double reference of the oracle",
                       "items": per_item}, fh, indent=0)
    errs = np.array([r["max_rel_err"] for r in per_item]) if per_item else np.zeros(1)
    line = {
        "mode": "batched", "metric": "batched Ozaki-II DGEMM effective TFLOPS (sum 2mnk / time)",
        "value": flops / (t_grouped * 1e-3) / 1e12, "unit": "TFLOPS", "n_gpus": 1,
        "ms_per_batch": t_grouped, "steps": args.steps, "warmup": args.warmup,
        "config": {"workload": f"{len(items)} problems, m, n, k log-uniform in [64, 2048], "
                               "phi in {0.5, 1} alternating", "launch": "ozaki2_dgemm_grouped "
                               "replayed from a CUDA graph", "n_per_item": "autotuned per "
                               "size class to the accuracy of cuBLAS DGEMM"},
        "moduli_histogram": {str(N): sum(1 for it in items if it["N"] == N)
                             for N in sorted({it["N"] for it in items})},
        "per_request_ozaki2_ms": t_loop, "per_request_cublas_dgemm_ms": t_cublas,
        "speedup_vs_cublas_loop": t_cublas / t_grouped,
        "speedup_vs_per_request_ozaki2": t_loop / t_grouped,
        "accuracy": {"items_checked": min(args.err_items, len(items)),
                     "max_rel_err": worst, "cublas_max_rel_err": worst_cub,
                     "median_item_max_rel_err": float(np.median(errs)),
                     "items_worse_than_cublas": int(worse_than_cublas),
                     "sample": f"{side}x{side} random block per item vs double-double",
                     "per_item_file": args.items_out},
        "calibration": {"seconds": calib_s, "source": calib_src, "margin": args.n_margin,
                        "table": autotune.table_to_json(table)},
        "tile_tuning": {"chunk_k_ms": {str(c): t for c, t in chunk_ms.items()},
                        "chunk_k": chunk_best,
                        "rules_n_max_k_max_tile_n_chunk_k": tiles["rules"],
                        "auto_ms": tiles["auto_ms"], "tuned_ms": tiles["best_ms"],
                        "tile_histogram": tile_histogram(items, tiles["rules"]),
                        "tiles": "128 rows x 256, 128 or 64 columns, per problem"},
        "device_status": status,
    }
    print(json.dumps(line), flush=True)


def tile_histogram(items, rules):
    """Problems per tile width under the given rules (the library's automatic width for n
    otherwise: 64 for n <= 64, 128 for n <= 128, else 256)."""
    hist = {}
    for it in items:
        tn = next((r[2] for r in rules if it["n"] <= r[0] and it["k"] <= r[1]),
                  64 if it["n"] <= 64 else 128 if it["n"] <= 128 else 256)
        hist[str(tn)] = hist.get(str(tn), 0) + 1
    return hist


def run_serve(args):
    """Serving: Poisson streams of requests (sizes log-uniform in [64, serve_max], relative-error
    targets 1e-10 / 1e-13 / 1e-15 in turn, N from the calibration table) through the
    continuous-batching server with its residue cache, at each offered rate (0 = every request
    at once: the server's capacity); p50/p99 latency, throughput and a makespan breakdown per
    rate, and a per-request cuBLAS DGEMM loop over the same stream at saturation."""
    import numpy as np
    import torch

    import synthetic
    from paper_2606_29129_gb300 import autotune
    from paper_2606_29129_gb300.serve import GpuExecutor, Request, ResultPool, Server

    rng = np.random.default_rng(args.serve_seed)
    pool = []
    for i in range(args.serve_pool):
        m, n, k = (int(np.exp(rng.uniform(np.log(64), np.log(args.serve_max + 1))))
                   for _ in range(3))
        phi = (0.5, 1.0)[i % 2]
        A = synthetic.paper_matrix_torch(m, k, phi, 300000 + 2 * i).cpu().pin_memory()
        B = synthetic.paper_matrix_torch(k, n, phi, 300001 + 2 * i).cpu().pin_memory()
        pool.append((m, n, k, A, B))
    targets = (1e-10, 1e-13, 1e-15)
    t0 = time.perf_counter()
    table = autotune.load_calibration()
    if table is None:
        table = autotune.calibrate(ks=tuple(e for e in autotune.CLASS_EDGES
                                            if e <= args.serve_max))
    calib_s = time.perf_counter() - t0
    slot_ws = args.serve_slot_ws_gb << 30
    budget = args.serve_budget_gb << 30
    cache_bytes = args.serve_cache_gb << 30
    count = args.serve_requests
    cub_ms = None
    # page-locked result buffers, reused: the client consumes each result when it completes and
    # hands the buffer back; allocated before the timed streams (up to 64 per size bucket)
    results = ResultPool(lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True))
    picks0 = np.random.default_rng(args.serve_seed + 1).integers(0, len(pool), size=count)
    per_bucket = {}
    for p in picks0:
        b = ResultPool.bucket(pool[int(p)][0] * pool[int(p)][1])
        per_bucket[b] = per_bucket.get(b, 0) + 1
    for b, c in per_bucket.items():
        results.prewarm(b, min(c, 64))
    prewarmed = results.allocated
    for lam in args.serve_rates:
        rng_s = np.random.default_rng(args.serve_seed + 1)
        arrivals = (np.cumsum(rng_s.exponential(1.0 / lam, size=count)) if lam > 0
                    else np.zeros(count))
        picks = rng_s.integers(0, len(pool), size=count)
        ex = GpuExecutor(slots=args.serve_slots, slot_workspace_bytes=slot_ws,
                         cache_bytes=cache_bytes, result_pool=results)
        io_budget = budget - args.serve_slots * slot_ws - cache_bytes
        srv = Server(ex, io_budget_bytes=io_budget, max_batch=64, calibration=table,
                     max_batch_flops=args.serve_batch_tflop * 1e12)
        reqs = []
        start = time.perf_counter()
        i = 0
        consumed = 0
        while i < count or not srv.idle():
            now = time.perf_counter() - start
            while i < count and arrivals[i] <= now:
                p = int(picks[i])
                m, n, k, A, B = pool[p]
                r = Request(rid=i, m=m, n=n, k=k, target=targets[i % 3], A=A, B=B,
                            a_key=("A", p), b_key=("B", p), arrival=start + arrivals[i])
                srv.submit(r)
                reqs.append(r)
                i += 1
            srv.step()
            while consumed < len(srv.finished):   # the client takes each result as it completes
                ex.recycle(srv.finished[consumed])
                consumed += 1
        makespan = time.perf_counter() - start
        bd = ex.breakdown()
        lat = sorted(r.latency for r in reqs if r.error is None)
        ok = [r for r in reqs if r.error is None]
        flops = sum(2.0 * r.m * r.n * r.k for r in ok)
        line = {
            "mode": "serving", "metric": "served emulated DGEMM p50/p99 latency and throughput",
            "requests": len(reqs), "completed": len(ok), "rate_per_s": lam,
            "makespan_s": makespan, "throughput_req_per_s": len(ok) / makespan,
            "effective_tflops": flops / makespan / 1e12,
            "latency_ms": {"p50": 1e3 * lat[len(lat) // 2],
                           "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "max": 1e3 * lat[-1]},
            "moduli_histogram": {str(N): sum(1 for r in ok if r.num_moduli == N)
                                 for N in sorted({r.num_moduli for r in ok})},
            "peak_upload_gb": srv.peak_io / 2**30, "budget_gb": args.serve_budget_gb,
            "breakdown": {
                "host_scheduling_s": srv.step_seconds,
                "link_upload_gb": bd["upload_bytes"] / 1e9,
                "link_result_gb": bd["result_bytes"] / 1e9,
                "encode_device_s": bd["encode_ms"] / 1e3,
                "batch_device_s": bd["batch_ms"] / 1e3,
                "batches": bd["batches"],
                "encoded_operands": bd["encoded_operands"],
                "cache_hits": bd.get("cache_hits"), "cache_misses": bd.get("cache_misses"),
                "cache_evictions": bd.get("cache_evictions"),
                "cache_peak_gb": bd.get("cache_peak_gb"),
                "result_buffers": {"prewarmed": prewarmed, "allocated_total": results.allocated},
                "note": "batch_device_s sums the slots' grouped calls (GEMM + CRT writing C to "
                        "host memory), which overlap on the device; host_scheduling_s is the "
                        "time spent inside Server.step"},
            "config": {"sizes": f"m, n, k log-uniform in [64, {args.serve_max}]",
                       "targets": list(targets), "slots": args.serve_slots,
                       "slot_workspace_gb": args.serve_slot_ws_gb,
                       "residue_cache_gb": args.serve_cache_gb, "pool": len(pool),
                       "batch_work_cap_tflop": args.serve_batch_tflop,
                       "arrivals": "Poisson" if lam > 0 else "all at t = 0"},
            "calibration_s": calib_s,
        }
        if lam == 0:
            # a per-request cuBLAS DGEMM loop over the same stream (device-resident inputs)
            if cub_ms is None:
                torch.backends.cuda.matmul.allow_tf32 = False
                cub_ms = []
                for (m, n, k, A, B) in pool:
                    dA, dB = A.cuda(), B.cuda()
                    out = torch.empty((n, m), dtype=torch.float64, device="cuda")
                    torch.matmul(dB.view(n, k), dA.view(k, m), out=out)
                    torch.cuda.synchronize()
                    s_ev = torch.cuda.Event(enable_timing=True)
                    e_ev = torch.cuda.Event(enable_timing=True)
                    s_ev.record()
                    torch.matmul(dB.view(n, k), dA.view(k, m), out=out)
                    e_ev.record()
                    torch.cuda.synchronize()
                    cub_ms.append(s_ev.elapsed_time(e_ev))
                    del dA, dB, out
            cub_total = sum(cub_ms[int(picks[r.rid])] for r in ok) / 1e3
            line["cublas_dgemm_loop_s"] = cub_total
            line["cublas_loop_tflops"] = flops / cub_total / 1e12
            line["speedup_vs_cublas_loop"] = cub_total / makespan
        print(json.dumps(line), flush=True)
        del ex, srv
        torch.cuda.empty_cache()


def run_sweep(args):
    """Accuracy sweep: max relative error vs the double-double reference for each N, phi and
    scaled copy, beside cuBLAS on the same inputs.  f64: N = 8..20, phi in {0.5, 1, 2}, copies
    scaled by 2^+-40 and 3.7e+-20.  f32 (SGEMM): N = 3..12, phi in {0, 0.5, 1, 1.5} (the paper's
    SGEMM ranges), copies scaled by 2^+-20.  One JSON line per (size, phi, alpha)."""
    import numpy as np
    import torch

    import oracle
    import synthetic
    from paper_2606_29129_gb300 import ozaki2 as oz

    oracle.build()
    torch.backends.cuda.matmul.allow_tf32 = False
    f32 = args.dtype == "f32"
    moduli = range(3, 13) if f32 else range(8, 21)
    phis = (0.0, 0.5, 1.0, 1.5) if f32 else (0.5, 1.0, 2.0)
    alphas = (1.0, 2.0**20, 2.0**-20) if f32 else (1.0, 2.0**40, 2.0**-40, 3.7e20, 3.7e-20)
    gemm = oz.ozaki2_sgemm if f32 else oz.ozaki2_dgemm
    for size in args.sweep_sizes:
        m = n = k = size
        for pi, phi in enumerate(phis):
            A0 = synthetic.paper_matrix_torch(m, k, phi, synthetic.seed_for(2, pi, 1))
            B0 = synthetic.paper_matrix_torch(k, n, phi, synthetic.seed_for(2, pi, 2))
            if f32:
                A0, B0 = A0.float(), B0.float()
            rng = np.random.default_rng(size + pi)
            I = np.sort(rng.choice(m, size=args.err_block, replace=False)).astype(np.int32)
            J = np.sort(rng.choice(n, size=args.err_block, replace=False)).astype(np.int32)
            for alpha in alphas:
                A = A0 * alpha
                B = B0 * alpha
                A_h = A.cpu().numpy().astype(np.float64)
                B_h = B.cpu().numpy().astype(np.float64)
                hi, lo = oracle.dd_block(A_h, B_h, k, I, J)
                C = torch.empty((n, m), dtype=A.dtype, device="cuda")
                errs = {}
                for N in moduli:
                    rc = gemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, N)
                    if rc:
                        raise oz.Ozaki2Error(gemm.__name__, rc)
                    torch.cuda.synchronize()
                    errs[N] = oracle.max_rel_error(
                        C.cpu().numpy()[np.ix_(J, I)].astype(np.float64), hi, lo)[0]
                Cd = torch.matmul(B.view(n, k), A.view(k, m))
                torch.cuda.synchronize()
                cub = oracle.max_rel_error(Cd.cpu().numpy()[np.ix_(J, I)].astype(np.float64),
                                           hi, lo)[0]
                default = next((N for N in moduli if errs[N] <= cub), None)
                print(json.dumps({"dtype": args.dtype, "size": size, "phi": phi, "alpha": alpha,
                                  "sample": f"{len(I)}x{len(J)}", "max_rel_err": errs,
                                  "cublas": cub, "smallest_N_not_worse": default}),
                      flush=True)
                del A, B, C, Cd
            del A0, B0
            torch.cuda.empty_cache()


def run_scaling_study(args):
    """Figs. 1-3 on the GPU: the original fast mode (Algorithm 1) and accurate mode against the
    proposed scaling (Algorithm 2), all at N = 20, for A = 2^s A^, B = 2^s B^, s = -10..10.

    Random inputs (eq. random-matrix-generation, phi in {0.5, 1, 2}): per s, the max relative
    error of each mode against double-double on a sampled block (the block's reference is taken
    once at s = 0 and scaled by 4^s, exact for powers of two), and the fast mode's max relative
    difference over the FULL matrix from the proposed N = 20 result (which resolves every error
    above ~2e-16 and so finds the isolated entries where CRT recovery fails).  cuBLAS DGEMM is
    measured at s in {-10, 0, 10} (its error does not depend on a power-of-two scale).
    All-ones inputs: log2 (A'B')_ij from the GPU shifts against log2(P/2) (Fig. 1), and the max
    relative error of both modes against the exact k 4^s over the full matrix (Fig. 3)."""
    import numpy as np
    import torch

    import oracle
    import synthetic
    from paper_2606_29129_gb300 import ozaki2 as oz

    oracle.build()
    torch.backends.cuda.matmul.allow_tf32 = False
    N = 20
    moduli, _, _ = oz.ozaki2_constants(N)
    log2_half_P = sum(math.log2(p) for p in moduli) - 1.0
    hf = oz.Handle()
    hf.set_option(oz.OPT_SCALING, oz.SCALING_FAST)
    ha = oz.Handle()
    ha.set_option(oz.OPT_SCALING, oz.SCALING_ACCURATE)
    hp = oz.Handle()

    def emulate(A, B, C, m, n, k, h):
        rc = oz.ozaki2_dgemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, N, h)
        if rc:
            raise oz.Ozaki2Error("ozaki2_dgemm", rc)

    def full_rel(C, R):
        nz = R != 0
        d = (C - R).abs() / R.abs().where(nz, torch.ones_like(R))
        return float(d.where(nz, torch.zeros_like(d)).max())

    svals = list(range(-10, 11))
    for size in args.study_sizes:
        m = n = k = size
        Cf = torch.empty((n, m), dtype=torch.float64, device="cuda")
        Cp = torch.empty_like(Cf)
        Ca = torch.empty_like(Cf)
        for pi, phi in enumerate((0.5, 1.0, 2.0)):
            A0 = synthetic.paper_matrix_torch(m, k, phi, synthetic.seed_for(2, pi, 1))
            B0 = synthetic.paper_matrix_torch(k, n, phi, synthetic.seed_for(2, pi, 2))
            rng = np.random.default_rng(size + pi)
            I = np.sort(rng.choice(m, size=args.err_block, replace=False)).astype(np.int32)
            J = np.sort(rng.choice(n, size=args.err_block, replace=False)).astype(np.int32)
            hi0, lo0 = oracle.dd_block(A0.cpu().numpy(), B0.cpu().numpy(), k, I, J)
            Jd, Id = torch.from_numpy(J).long().cuda(), torch.from_numpy(I).long().cuda()

            def block(C):
                return C[Jd][:, Id].cpu().numpy()

            for s in svals:
                A, B = A0 * 2.0**s, B0 * 2.0**s
                hi, lo = hi0 * 4.0**s, lo0 * 4.0**s
                emulate(A, B, Cf, m, n, k, hf)
                emulate(A, B, Cp, m, n, k, hp)
                emulate(A, B, Ca, m, n, k, ha)
                torch.cuda.synchronize()
                line = {"study": "fig2", "size": size, "phi": phi, "s": s, "N": N,
                        "sample": f"{len(I)}x{len(J)}",
                        "fast_vs_dd_block": oracle.max_rel_error(block(Cf), hi, lo)[0],
                        "proposed_vs_dd_block": oracle.max_rel_error(block(Cp), hi, lo)[0],
                        "accurate_vs_dd_block": oracle.max_rel_error(block(Ca), hi, lo)[0],
                        "fast_full_vs_proposed": full_rel(Cf, Cp),
                        "accurate_full_vs_proposed": full_rel(Ca, Cp)}
                if s in (-10, 0, 10):
                    Cd = torch.matmul(B.view(n, k), A.view(k, m))
                    torch.cuda.synchronize()
                    line["cublas_vs_dd_block"] = oracle.max_rel_error(block(Cd), hi, lo)[0]
                    del Cd
                print(json.dumps(line), flush=True)
                del A, B
            del A0, B0
            torch.cuda.empty_cache()
        ones_A = torch.ones((k, m), dtype=torch.float64, device="cuda")
        ones_B = torch.ones((n, k), dtype=torch.float64, device="cuda")
        e = torch.empty(m, dtype=torch.int32, device="cuda")
        for s in svals:
            A, B = ones_A * 2.0**s, ones_B * 2.0**s
            exact = torch.full_like(Cf, k * 4.0**s)
            emulate(A, B, Cf, m, n, k, hf)
            emulate(A, B, Cp, m, n, k, hp)
            emulate(A, B, Ca, m, n, k, ha)
            rc = oz.ozaki2_scale_a("N", m, k, A, m, N, e, hf)
            if rc:
                raise oz.Ozaki2Error("ozaki2_scale_a", rc)
            torch.cuda.synchronize()
            ef = int(e[0])
            rc = oz.ozaki2_scale_a("N", m, k, A, m, N, e, hp)
            if rc:
                raise oz.Ozaki2Error("ozaki2_scale_a", rc)
            torch.cuda.synchronize()
            ep = int(e[0])
            print(json.dumps({"study": "fig1_fig3", "size": size, "s": s, "N": N,
                              "log2_half_P": log2_half_P,
                              "fast_log2_ApBp": math.log2(k) + 2 * (ef + s),
                              "proposed_log2_ApBp": math.log2(k) + 2 * (ep + s),
                              "fast_full_vs_exact": full_rel(Cf, exact),
                              "proposed_full_vs_exact": full_rel(Cp, exact),
                              "accurate_full_vs_exact": full_rel(Ca, exact)}), flush=True)
            del A, B, exact
        del ones_A, ones_B, Cf, Cp, Ca
        torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=SIZE)
    ap.add_argument("--shape", type=int, nargs=3, default=None, metavar=("M", "N", "K"),
                    help="a rectangular problem (the configurations m=n=16384, k=1024; "
                         "m=n=1024, k=65536; m=65536, n=256, k=4096) instead of --size")
    ap.add_argument("--moduli", type=int, default=None,
                    help=f"moduli count (default {NUM_MODULI} for f64, {SGEMM_MODULI} for f32)")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"],
                    help="f64: emulated DGEMM (the benchmark); f32: emulated SGEMM")
    ap.add_argument("--scaling", default="proposed", choices=["proposed", "fast", "accurate"],
                    help="scaling step: Algorithm 2 (default), Algorithm 1, or accurate mode")
    ap.add_argument("--err-block", type=int, default=96)
    ap.add_argument("--cpu-block", type=int, default=896)
    ap.add_argument("--ref-block", type=int, default=384)
    ap.add_argument("--cublas-reps", type=int, default=1)
    ap.add_argument("--gemm-traffic", type=float, default=None,
                    help="DRAM bytes per residue-GEMM launch from an ncu capture, if current")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-copies", type=int, choices=[0, 1], default=None,
                    help="e2e leg: how the call moves host data (OZAKI2_OPT_HOST_COPIES: 0 "
                         "kernels, the default; 1 copy engines)")
    ap.add_argument("--profile-step", action="store_true",
                    help="only the timed steps (no cuBLAS, accuracy, CPU or e2e legs): for "
                         "launch lists under a profiler")
    ap.add_argument("--batched", action="store_true",
                    help="the batched workload (grouped call) instead of the benchmark")
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--err-items", type=int, default=512)
    ap.add_argument("--n-margin", type=float, default=8.0,
                    help="batched mode: choose N with calibrated error <= cuBLAS's / margin")
    ap.add_argument("--calibrate", action="store_true",
                    help="measure the autotuner's accuracy table against double-double")
    ap.add_argument("--calibration-out", default=None)
    ap.add_argument("--err-side", type=int, default=48,
                    help="batched mode: rows and columns of each item's error block")
    ap.add_argument("--items-out", default=None,
                    help="batched mode: write every item's size, N and errors to this JSON file")
    ap.add_argument("--serve", action="store_true",
                    help="the serving workload (Poisson stream) instead of the benchmark")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.0, 100.0, 400.0],
                    help="offered loads in requests per second (0: every request at once)")
    ap.add_argument("--serve-cache-gb", type=int, default=60)
    ap.add_argument("--serve-batch-tflop", type=float, default=2.0,
                    help="work cap of one serving batch, in units of 10^12 flops (sum 2mnk)")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-max", type=int, default=8192)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--serve-slots", type=int, default=2)
    ap.add_argument("--serve-slot-ws-gb", type=int, default=20)
    ap.add_argument("--serve-budget-gb", type=int, default=120)
    ap.add_argument("--serve-seed", type=int, default=5)
    ap.add_argument("--sweep", action="store_true",
                    help="accuracy sweep over N, phi and alpha instead of the benchmark")
    ap.add_argument("--sweep-sizes", type=int, nargs="+", default=[8192, 16384])
    ap.add_argument("--tune-tiles", action="store_true",
                    help="time the residue-GEMM kernel variants and K chunks per size class")
    ap.add_argument("--tune-sizes", type=int, nargs="+", default=[1024, 2048, 4096, 8192, 16384])
    ap.add_argument("--tune-chunks", type=int, nargs="+", default=[960, 640, 448, 320])
    ap.add_argument("--tune-groups", type=int, nargs="+", default=[0],
                    help="tile-order group sizes to time (0: the library default, 16)")
    ap.add_argument("--scaling-study", action="store_true",
                    help="fast mode (Algorithm 1) against the proposed scaling over alpha = 2^s")
    ap.add_argument("--study-sizes", type=int, nargs="+", default=[1024, 16384])
    args = ap.parse_args()
    if args.moduli is None:
        args.moduli = SGEMM_MODULI if args.dtype == "f32" else NUM_MODULI
    if args.sweep:
        run_sweep(args)
        return
    if args.scaling_study:
        run_scaling_study(args)
        return
    if args.tune_tiles:
        run_tune_tiles(args)
        return
    if args.calibrate:
        run_calibrate(args)
        return
    if args.batched:
        if args.impl == "reference":
            run_reference_batched(args)
        else:
            run_batched(args)
        return
    if args.serve:
        run_serve(args)
        return
    full_reference = args.impl == "reference" and args.ref_block >= args.size
    if args.warmup < 3 and not full_reference:  # (a full oracle product needs no warm-up)
        log("warm-up raised to 3 steps")
        args.warmup = 3
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
