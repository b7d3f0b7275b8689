#!/usr/bin/env python
"""Benchmark of the planar split-complex DFT on GB300.

One step = one forward transform (Eq. (1) in the split form of Eq. (3)) of a
whole synthetic batch, already resident in HBM: N = 1024, batch 65536, FP32
planar, iid N(0, 1) from seed 1 (256 MiB per plane; each step reads 512 MiB
and writes 512 MiB, more than L2, so no L2 flush is needed between steps).

Prints ONE JSON line (rank 0):
  value        Gpoints/s of the forward kernel over all ranks (B*N*ranks / time)
  roofline     HBM roofline of that kernel: 16 algorithmic bytes per point
               (read xr, xi; write yr, yi) / average launch time, against the
               measured copy bandwidth of this GPU model
  adjoint      the same for the adjoint kernel (E_2N^T)
  e2e          the forward through the C ABI on pinned HOST buffers
               (host->device, transform, device->host inside the timed region)
  cpu_baseline the CPU oracle (Eq. (6) procedure, float64) on the host cores,
               timed on a bounded sample of the same workload
  clocks       SM clock and throttle reasons sampled during the timed region

--impl reference times the CPU oracle instead (the only other implementation
of the method that exists), on the same workload and metric.
Multi-GPU (torchrun): every rank transforms its own batch (weak scaling); the
transforms are independent, so there is no collective on the data path.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "planar DFT Gpts/s & %HBM peak, N=1024 B=65536: FP32 vs split-BF16, fwd+adj"
UNIT = "Gpts/s"
N_POINTS = 1024
BATCH = 65536
BYTES_PER_POINT = 16          # algorithmic: 4 B each of xr, xi read and yr, yi written

# Sources of the timed N = 1024 kernel: the traffic figure below is reported
# only while their code (comments aside) is unchanged since its ncu capture.
HEADLINE_SOURCES = ("fft_core.cuh", "kernels_rows.cuh", "rows_1024.cu", "launch.h")

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one forward
# launch of the full 65536 x 1024 workload, from one ncu capture of the
# headline command (`ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum
# -k regex:k_rows`), with the source hash of the kernel it was taken on.
NCU_TRAFFIC = {
    "fwd": {"bytes": 536916480 + 485299712, "hash": "83fbbb28fab409a3",
            "schedule": "N=1024: 32 threads/transform, radix [32,32]"},
}


def _code_only(text: str) -> str:
    """C++ source without comments and with whitespace collapsed, so that
    editing a comment does not change the hash (the sources have no string
    literals containing comment markers)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2504_07264_gb300", "csrc")
    for name in HEADLINE_SOURCES:
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode() + b"\0" + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def mark(self):
        return len(self.lines)

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self._t is not None:
            self._t.join(timeout=2)

    def summary(self, start: int = 0, end: int | None = None) -> dict:
        rows = []
        for ln in self.lines[start:end]:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                rows.append((float(p[0]), float(p[1]), p[4], p[5], p[6], p[7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------- CPU oracle --
def cpu_oracle_rate(target_s: float = 10.0, max_batch: int = BATCH) -> dict:
    """Time the CPU oracle's Eq. (6) procedure (float64, OpenMP over
    transforms, all host cores) on a bounded sample of the workload."""
    import numpy as np

    import workloads
    from oracle import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    used = oracle.thread_count(threads)
    # calibrate on a small sample, then size the timed sample to ~target_s
    cal = min(max_batch, max(64, 4 * used))
    xr, xi = workloads.normal_planes(N_POINTS, cal, seed=1)
    xr64, xi64 = xr.astype(np.float64), xi.astype(np.float64)
    t0 = time.perf_counter()
    oracle.dft_factored_dit(xr64, xi64, threads=used)
    dt = time.perf_counter() - t0
    per = dt / cal
    sample = int(min(max_batch, max(cal, target_s / max(per, 1e-9))))
    # when the whole workload is quicker than target_s, time repeated passes
    passes = max(1, int(round(target_s / max(per * sample, 1e-9)))) if sample == max_batch else 1
    xr, xi = workloads.normal_planes(N_POINTS, sample, seed=1)
    xr64, xi64 = xr.astype(np.float64), xi.astype(np.float64)
    t0 = time.perf_counter()
    for _ in range(passes):
        oracle.dft_factored_dit(xr64, xi64, threads=used)
    dt = time.perf_counter() - t0
    what = (f"all {sample} transforms, {passes} passes" if passes > 1
            else f"first {sample} of the {BATCH} transforms")
    # the same procedure on one core, on a sample sized to ~target_s / 4
    one = int(max(16, min(max_batch, (target_s / 4) / max(per * used, 1e-9))))
    t0 = time.perf_counter()
    oracle.dft_factored_dit(xr64[:one], xi64[:one], threads=1)
    dt1 = time.perf_counter() - t0
    # the binary32 instance of the same procedure, all cores, on the float32
    # inputs themselves (sample sized like the one-core leg)
    f32n = int(max(16, min(sample, (target_s / 4) / max(per, 1e-9))))
    t0 = time.perf_counter()
    oracle.dft_factored_dit_f32(xr[:f32n], xi[:f32n], threads=used)
    dt32 = time.perf_counter() - t0
    return {"value": passes * sample * N_POINTS / dt / 1e9, "unit": UNIT, "cores": used,
            "kind": "oracle",
            "sample": f"{what} (N={N_POINTS}, seed 1), Eq. (6) procedure in float64, {dt:.1f} s",
            "one_core": {"value": one * N_POINTS / dt1 / 1e9, "unit": UNIT,
                         "sample": f"first {one} transforms, {dt1:.1f} s"},
            "float32": {"value": f32n * N_POINTS / dt32 / 1e9, "unit": UNIT, "cores": used,
                        "sample": f"first {f32n} transforms, Eq. (6) procedure in float32, "
                                  f"{dt32:.1f} s"}}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import workloads
    from oracle import oracle
    oracle.build()
    used = oracle.thread_count(os.cpu_count() or 1)
    # size each step so that warmup + steps take a few minutes at most
    cal = 256
    xr, xi = workloads.normal_planes(N_POINTS, cal, seed=1)
    t0 = time.perf_counter()
    oracle.dft_factored_dit(xr.astype(np.float64), xi.astype(np.float64), threads=used)
    per = (time.perf_counter() - t0) / cal
    budget = 120.0 / max(1, args.steps + args.warmup)
    sample = int(max(16, min(BATCH, budget / max(per, 1e-9))))
    xr, xi = workloads.normal_planes(N_POINTS, sample, seed=1)
    xr64, xi64 = xr.astype(np.float64), xi.astype(np.float64)
    for _ in range(args.warmup):
        oracle.dft_factored_dit(xr64, xi64, threads=used)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.dft_factored_dit(xr64, xi64, threads=used)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = sample * N_POINTS / dt / 1e9
    desc = (f"{sample} of the {BATCH} transforms (N={N_POINTS}, seed 1) per step, "
            f"Eq. (6) procedure in float64")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"bandwidth: N={N_POINTS} x {BATCH} planar, iid N(0,1) seed 1 "
                               f"(CPU oracle on a bounded sample)", "n": N_POINTS, "batch": BATCH},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------ GPU arm --
def _time_steps(fn, steps: int, stream) -> float:
    """Milliseconds per step over `steps` calls, CUDA events on `stream`."""
    import torch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / steps


def _err_sums(gr, gi, xr_rows, xi_rows):
    """Squared error of GPU rows (gr, gi) against a float64 FFT (numpy.fft) of
    the input rows, and the squared norm of that reference, per row."""
    import numpy as np
    ref = np.fft.fft(np.asarray(xr_rows, np.float64) + 1j * np.asarray(xi_rows, np.float64))
    er = np.asarray(gr, np.float64) - ref.real
    ei = np.asarray(gi, np.float64) - ref.imag
    return (er ** 2 + ei ** 2).sum(-1), (ref.real ** 2 + ref.imag ** 2).sum(-1)


def _rel_l2(num, den) -> dict:
    """Relative L2 error over the sample and of its worst transform."""
    import numpy as np
    num, den = np.atleast_1d(num), np.atleast_1d(den)
    return {"rel_l2": float(np.sqrt(num.sum() / den.sum())),
            "worst_transform": float(np.sqrt(num / den).max())}


def _sample_rows(plan_run, xr_h, xi_h, yr, yi, count: int, seed: int = 8) -> dict:
    """Run `plan_run` once (it writes yr, yi) and compare `count` sampled rows
    of a uniform batch with a float64 FFT."""
    import numpy as np
    import torch
    plan_run()
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(seed).choice(xr_h.shape[0], count, replace=False))
    sel = torch.from_numpy(idx).to(yr.device)
    out = _rel_l2(*_err_sums(yr.index_select(0, sel).cpu().numpy(),
                             yi.index_select(0, sel).cpu().numpy(), xr_h[idx], xi_h[idx]))
    out["sample"] = f"{count} transforms vs a float64 FFT (numpy.fft)"
    return out


def _step_stats(fn, n: int, stream) -> dict:
    """Median and best of `n` individually timed steps (CUDA events around
    each call on `stream`), milliseconds."""
    import statistics

    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(n)]
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    evs[-1][1].synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    return {"median_ms": statistics.median(ms), "best_ms": min(ms), "samples": n}


def run_ours(args) -> None:
    import numpy as np
    import torch

    import workloads
    from paper_2504_07264_gb300 import SDFT_ADJOINT, SDFT_FORWARD, Plan
    from paper_2504_07264_gb300 import build as cuda_build
    from paper_2504_07264_gb300.sharding import max_over_ranks

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cuda_build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    batch = args.batch or BATCH
    xr_h, xi_h = workloads.bandwidth(batch)
    points = N_POINTS * batch
    xr = torch.from_numpy(xr_h).cuda()
    xi = torch.from_numpy(xi_h).cuda()
    yr = torch.empty_like(xr)
    yi = torch.empty_like(xi)
    plan = Plan(N_POINTS, batch)
    launches_per_step = plan.launches(SDFT_FORWARD)

    fwd = lambda: plan.execute(SDFT_FORWARD, xr, xi, yr, yi, stream)  # noqa: E731
    adj = lambda: plan.execute(SDFT_ADJOINT, xr, xi, yr, yi, stream)  # noqa: E731
    for _ in range(args.warmup):
        fwd()
        adj()

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = None
    with ClockSampler(gpu_id if rank == 0 else None) as clk:
        barrier()
        m0 = clk.mark()
        ms_fwd = _time_steps(fwd, args.steps, stream)
        m1 = clk.mark()
        barrier()
        ms_adj = _time_steps(adj, args.steps, stream)
        barrier()
        # outside the timed region: 20 individually timed forward steps
        fwd_stats = _step_stats(fwd, 20, stream)
        # practical ceiling: a same-shape planar copy (both planes)
        copy = lambda: (yr.copy_(xr), yi.copy_(xi))  # noqa: E731
        for _ in range(3):
            copy()
        ms_copy = _time_steps(copy, max(10, args.steps // 4), stream)
        barrier()
        # the metric's second arithmetic path: split-BF16 tensor cores, same shape
        with Plan(N_POINTS, batch, 1) as splan:
            sf = lambda: splan.execute(SDFT_FORWARD, xr, xi, yr, yi, stream)  # noqa: E731
            sa = lambda: splan.execute(SDFT_ADJOINT, xr, xi, yr, yi, stream)  # noqa: E731
            for _ in range(3):
                sf()
                sa()
            split_steps = max(10, min(args.steps, 500))
            ms_sf = _time_steps(sf, split_steps, stream)
            ms_sa = _time_steps(sa, split_steps, stream)
            split_desc = splan.describe()
            # after the timed regions: sampled accuracy of both forward paths
            acc_split = _sample_rows(sf, xr_h, xi_h, yr, yi, 64)
    acc_f32 = _sample_rows(fwd, xr_h, xi_h, yr, yi, 64)
    clocks = clk.summary(m0, m1 if m1 > m0 else None)
    ms_fwd = max_over_ranks(ms_fwd, dist)
    ms_adj = max_over_ranks(ms_adj, dist)

    # end to end through the C ABI on pinned host buffers: the default mode
    # (zero copy for page-locked buffers) and the staged copy pipeline
    e2e_s = None
    e2e_modes = {}
    if not args.no_e2e:
        from paper_2504_07264_gb300.sdft import SDFT_HOST_STAGED, SDFT_HOST_ZERO_COPY
        hxr = torch.from_numpy(xr_h).pin_memory()
        hxi = torch.from_numpy(xi_h).pin_memory()
        hyr = torch.empty_like(hxr).pin_memory()
        hyi = torch.empty_like(hxi).pin_memory()
        e2e_steps = max(1, min(args.steps, 10))
        for mode_name, mode in (("staged", SDFT_HOST_STAGED), ("zero_copy", SDFT_HOST_ZERO_COPY)):
            plan.set_host_mode(mode)
            plan.execute_host(SDFT_FORWARD, hxr, hxi, hyr, hyi, stream)   # first call sets up
            barrier()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                plan.execute_host(SDFT_FORWARD, hxr, hxi, hyr, hyi, stream)
            barrier()
            sec = (time.perf_counter() - t0) / e2e_steps
            e2e_modes[mode_name] = max_over_ranks(sec, dist)
        e2e_s = e2e_modes["zero_copy"]
    describe = plan.describe()
    plan.destroy()

    # The other measured configurations, on rank 0's GPU after every timed
    # region of the headline (each with its own warm-up and CUDA-event
    # timing; none of it is in `value`): the differentiation, precision and
    # batching workloads, each against the plain FP32 kernel on this GPU.
    extra = {}
    if rank == 0 and not args.no_extra:
        del xr, xi, yr, yi
        torch.cuda.empty_cache()
        xsteps = max(10, min(args.steps, 50))
        xwarm = max(3, min(args.warmup, 5))
        with ClockSampler(gpu_id) as xclk:
            extra["autograd"] = autograd_block(xsteps, xwarm, stream)
            torch.cuda.empty_cache()
            extra["precision"] = precision_block(xsteps, xwarm, stream, with_n1024=False)
            torch.cuda.empty_cache()
            extra["ragged"] = ragged_block(xsteps, xwarm, stream)
            torch.cuda.empty_cache()
        extra["extra_clocks"] = xclk.summary()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks = _peaks()
    achieved = BYTES_PER_POINT * points / (ms_fwd * 1e-3) / 1e9
    achieved_adj = BYTES_PER_POINT * points / (ms_adj * 1e-3) / 1e9
    src_hash = _kernel_source_hash()
    tr = NCU_TRAFFIC.get("fwd")
    traffic = (tr["bytes"] if tr and tr.get("hash") == src_hash
               and describe.startswith(tr["schedule"]) else None)
    cpu = None if args.no_cpu_baseline else cpu_oracle_rate()
    line = {
        "metric": METRIC,
        "value": world * points / (ms_fwd * 1e-3) / 1e9,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_fwd,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"bandwidth: N={N_POINTS} x {batch} FP32 planar forward, "
                               "iid N(0,1) seed 1",
                   "n": N_POINTS, "batch": batch, "per_gpu_points": points,
                   "l2": "inputs larger than L2 (1 GiB moved per step), no flush",
                   "schedule": describe, "parallelism": f"dp{world} (independent batches)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_source": f"{peaks['source']} (burst copy)",
                     "frac_of_nominal_8tbs": achieved / 8000.0},
        "adjoint": {"value": world * points / (ms_adj * 1e-3) / 1e9, "unit": UNIT,
                    "ms_per_step": ms_adj, "achieved_gbs": achieved_adj,
                    "frac": achieved_adj / peaks["hbm_gbs"]},
        "forward_step_stats": {
            **fwd_stats,
            "median_value": points / (fwd_stats["median_ms"] * 1e-3) / 1e9,
            "best_value": points / (fwd_stats["best_ms"] * 1e-3) / 1e9, "unit": UNIT,
            "what": "rank 0, forward steps timed one by one after the timed region"},
        "copy_ceiling": {"gbs": BYTES_PER_POINT * points / (ms_copy * 1e-3) / 1e9,
                         "what": "torch copy_ of both planes, same shape"},
        "split_bf16": {
            "forward": {"value": points / (ms_sf * 1e-3) / 1e9, "unit": UNIT, "ms": ms_sf,
                        "frac": BYTES_PER_POINT * points / (ms_sf * 1e-3) / 1e9 / peaks["hbm_gbs"]},
            "adjoint": {"value": points / (ms_sa * 1e-3) / 1e9, "unit": UNIT, "ms": ms_sa,
                        "frac": BYTES_PER_POINT * points / (ms_sa * 1e-3) / 1e9 / peaks["hbm_gbs"]},
            "steps": split_steps, "schedule": split_desc, "accuracy": acc_split,
            "what": "rank 0's GPU, same inputs, timed after the FP32 region"},
        "accuracy": acc_f32,
        "e2e": None if e2e_s is None else {
            "value": world * points / e2e_s / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": 2 * points * 4, "d2h_bytes_per_step": 2 * points * 4,
            "api": "sdft_execute_host, pinned host buffers, default mode (zero copy: the kernel "
                   "reads and writes host memory over NVLink-C2C)",
            "staged_pipeline": {"value": world * points / e2e_modes["staged"] / 1e9,
                                "unit": UNIT}},
        "cpu_baseline": cpu,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "kernel_source_hash": src_hash,
        **extra,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _measure_uniform(n: int, batch: int, xr_h, xi_h, steps: int, warmup: int, stream,
                     dtype: int = 0, accuracy_sample: int = 0) -> dict:
    """Forward and adjoint kernel times of one uniform plan (one GPU); with
    accuracy_sample > 0 also the relative L2 error of that many sampled
    transforms against a float64 FFT (numpy.fft; the tests pin it to the
    oracle and check every kernel against the oracle itself)."""
    import numpy as np
    import torch

    from paper_2504_07264_gb300 import SDFT_ADJOINT, SDFT_FORWARD, Plan
    xr = torch.from_numpy(xr_h).cuda()
    xi = torch.from_numpy(xi_h).cuda()
    yr = torch.empty_like(xr)
    yi = torch.empty_like(xi)
    points = n * batch
    peak = _peaks()["hbm_gbs"]
    acc = None
    with Plan(n, batch, dtype) as plan:
        if accuracy_sample:
            plan.execute(SDFT_FORWARD, xr, xi, yr, yi, stream)
            idx = np.sort(np.random.default_rng(8).choice(batch, accuracy_sample, replace=False))
            sel = torch.from_numpy(idx).cuda()
            gr = yr.index_select(0, sel).cpu().numpy().astype(np.float64)
            gi = yi.index_select(0, sel).cpu().numpy().astype(np.float64)
            ref = np.fft.fft(xr_h[idx].astype(np.float64) + 1j * xi_h[idx].astype(np.float64), axis=1)
            rr, ri = ref.real, ref.imag
            rows = np.sqrt(((gr - rr) ** 2 + (gi - ri) ** 2).sum(1) / (rr ** 2 + ri ** 2).sum(1))
            acc = {"rel_l2": float(np.sqrt(((gr - rr) ** 2 + (gi - ri) ** 2).sum()
                                           / (rr ** 2 + ri ** 2).sum())),
                   "rel_l2_worst_transform": float(rows.max()),
                   "sample": f"{accuracy_sample} transforms vs a float64 FFT (numpy.fft)"}
        fwd = lambda: plan.execute(SDFT_FORWARD, xr, xi, yr, yi, stream)  # noqa: E731
        adj = lambda: plan.execute(SDFT_ADJOINT, xr, xi, yr, yi, stream)  # noqa: E731
        for _ in range(warmup):
            fwd()
            adj()
        torch.cuda.synchronize()
        ms_f = _time_steps(fwd, steps, stream)
        ms_a = _time_steps(adj, steps, stream)
        out = {"n": n, "batch": batch, "dtype": dtype, "schedule": plan.describe(),
               "launches_per_call": plan.launches(SDFT_FORWARD)}
        if acc is not None:
            out["accuracy"] = acc
    for name, ms in (("forward", ms_f), ("adjoint", ms_a)):
        gbs = BYTES_PER_POINT * points / (ms * 1e-3) / 1e9
        out[name] = {"gpts": points / (ms * 1e-3) / 1e9, "ms": ms, "gbs": gbs, "frac": gbs / peak}
    return out


def autograd_block(steps: int, warmup: int, stream) -> dict:
    """The differentiation workload: N = 4096, batch 16384, iid N(0,1) seed 1;
    forward and adjoint kernels, and the whole autograd step (split_dft,
    loss sum(w_r yr^2 + w_i yi^2) with w iid U[0,1) seed 2, backward)."""
    import torch

    import workloads
    from paper_2504_07264_gb300 import split_dft
    cfg = workloads.AUTOGRAD
    n, batch = cfg["n"], cfg["batch"]
    xr_h, xi_h = workloads.normal_planes(n, batch, cfg["seed"])
    out = _measure_uniform(n, batch, xr_h, xi_h, steps, warmup, stream, accuracy_sample=32)
    wr_h, wi_h = workloads.loss_weights(n, batch, cfg["weight_seed"])
    xr = torch.from_numpy(xr_h).cuda().requires_grad_(True)
    xi = torch.from_numpy(xi_h).cuda().requires_grad_(True)
    wr, wi = torch.from_numpy(wr_h).cuda(), torch.from_numpy(wi_h).cuda()

    def step():
        xr.grad = None
        xi.grad = None
        yr, yi = split_dft(xr, xi)
        (wr * yr ** 2 + wi * yi ** 2).sum().backward()
    for _ in range(warmup):
        step()
    ms = _time_steps(step, max(5, steps // 10), stream)
    out["autograd_step"] = {"ms": ms, "gpts": n * batch / (ms * 1e-3) / 1e9,
                            "what": "split_dft forward + weighted-square loss + backward "
                                    "(adjoint kernel), torch elementwise ops included"}
    out["workload"] = (f"differentiation: N={n} x {batch} FP32 planar, iid N(0,1) seed 1; "
                       "loss weights U[0,1) seed 2")
    return out


def precision_block(steps: int, warmup: int, stream, with_n1024: bool = True) -> dict:
    """The precision workload: N = 256, batch 262144, |x| = 10^U(-3,3) with
    uniform phase (seed 3), on the FP32 kernel and on the split-BF16 and
    split-FP16 tensor-core paths, each with its error on 256 sampled
    transforms; optionally the same three paths on the N = 1024 x 65536
    bandwidth workload."""
    import workloads
    cfg = workloads.PRECISION
    n, batch = cfg["n"], cfg["batch"]
    xr_h, xi_h = workloads.precision()
    paths = {}
    for name, dt in (("f32", 0), ("split_bf16", 1), ("split_fp16", 2)):
        paths[name] = _measure_uniform(n, batch, xr_h, xi_h, steps, warmup, stream,
                                       dtype=dt, accuracy_sample=256)
    del xr_h, xi_h
    if with_n1024:
        br, bi = workloads.bandwidth()
        for name, dt in (("f32_n1024", 0), ("split_bf16_n1024", 1), ("split_fp16_n1024", 2)):
            paths[name] = _measure_uniform(1024, 65536, br, bi, steps, warmup, stream,
                                           dtype=dt, accuracy_sample=64)
    for name in ("split_bf16", "split_fp16"):
        paths[name]["vs_f32_forward"] = paths[name]["forward"]["gpts"] / paths["f32"]["forward"]["gpts"]
    return {"paths": paths,
            "workload": (f"precision: N={n} x {batch}, |x| = 10^U(-3,3), phase U[0,2pi), seed 3; "
                         "FP32 kernel vs split-BF16 vs split-FP16 tensor cores")}


def ragged_block(steps: int, warmup: int, stream, tune: bool = True) -> dict:
    """The batching workload: 10000 transforms of lengths 2^k, k uniform in
    {3..16} (seed 4), iid N(0,1): one persistent launch per call replayed from
    a CUDA graph (forward and adjoint), the plan's tuner run first; the same
    transforms as one uniform FP32 plan per length for comparison."""
    import numpy as np
    import torch

    import workloads
    from paper_2504_07264_gb300 import SDFT_ADJOINT, SDFT_FORWARD, Plan
    peak = _peaks()["hbm_gbs"]
    lengths, off, xr_h, xi_h = workloads.ragged_planes()
    points = int(off[-1])
    xr = torch.from_numpy(xr_h).cuda()
    xi = torch.from_numpy(xi_h).cuda()
    yr = torch.empty_like(xr)
    yi = torch.empty_like(xi)
    line = {}
    with Plan(lengths=lengths) as plan:
        if tune:
            # every length on its form 0 first (the library's default), then
            # each length's form chosen on this batch by the plan's tuner
            for logn in range(2, 17):
                if (lengths == (1 << logn)).any():
                    plan.set_ragged_form(1 << logn, 0)
            fwd0 = lambda: plan.execute(SDFT_FORWARD, xr, xi, yr, yi, stream)  # noqa: E731
            for _ in range(warmup):
                fwd0()
            ms0 = _time_steps(fwd0, steps, stream)
            line["default_forms"] = {"gpts": points / (ms0 * 1e-3) / 1e9, "ms": ms0,
                                     "what": "forward, every length on its form 0, before tuning"}
            line["ragged_tuning"] = plan.ragged_autotune(xr, xi, yr, yi, reps=5, stream=stream)
        line["forms"] = {str(1 << l): plan.ragged_form(1 << l)
                         for l in range(2, 17) if (lengths == (1 << l)).any()}
        fwd = lambda: plan.execute(SDFT_FORWARD, xr, xi, yr, yi, stream)  # noqa: E731
        adj = lambda: plan.execute(SDFT_ADJOINT, xr, xi, yr, yi, stream)  # noqa: E731
        for _ in range(warmup):
            fwd()
            adj()
        torch.cuda.synchronize()
        ms_f = _time_steps(fwd, steps, stream)
        ms_a = _time_steps(adj, steps, stream)
        line["schedule"] = plan.describe()
        line["launches_per_call"] = plan.launches(SDFT_FORWARD)
        # after the timed region: 64 sampled transforms against a float64 FFT
        fwd()
        torch.cuda.synchronize()
        yr_h, yi_h = yr.cpu().numpy(), yi.cpu().numpy()
        pick = np.sort(np.random.default_rng(8).choice(lengths.size, 64, replace=False))
        sums = [_err_sums(yr_h[off[t]:off[t + 1]], yi_h[off[t]:off[t + 1]],
                          xr_h[off[t]:off[t + 1]], xi_h[off[t]:off[t + 1]]) for t in pick]
        line["accuracy"] = dict(_rel_l2(np.array([a for a, _ in sums]),
                                        np.array([b for _, b in sums])),
                                sample="64 transforms (all lengths) vs a float64 FFT (numpy.fft)")
    for name, ms in (("forward", ms_f), ("adjoint", ms_a)):
        gbs = BYTES_PER_POINT * points / (ms * 1e-3) / 1e9
        line[name] = {"gpts": points / (ms * 1e-3) / 1e9, "ms": ms, "gbs": gbs,
                      "frac": gbs / peak}
    del xr, xi, yr, yi
    # the same transforms as one uniform plan per length (one launch each),
    # on per-length contiguous copies of the data
    plans, bufs = [], []
    for logn in range(2, 17):
        sel = np.nonzero(lengths == (1 << logn))[0]
        if sel.size == 0:
            continue
        rows_r = np.concatenate([xr_h[off[t]:off[t + 1]] for t in sel])
        rows_i = np.concatenate([xi_h[off[t]:off[t + 1]] for t in sel])
        a = torch.from_numpy(rows_r).cuda()
        b = torch.from_numpy(rows_i).cuda()
        bufs.append((a, b, torch.empty_like(a), torch.empty_like(b)))
        plans.append(Plan(1 << logn, int(sel.size)))

    def per_length():
        for pl, (a, b, c, d) in zip(plans, bufs):
            pl.execute(SDFT_FORWARD, a, b, c, d, stream)
    for _ in range(warmup):
        per_length()
    ms_u = _time_steps(per_length, steps, stream)
    for pl in plans:
        pl.destroy()
    gbs = BYTES_PER_POINT * points / (ms_u * 1e-3) / 1e9
    line["per_length_uniform_kernels"] = {
        "gpts": points / (ms_u * 1e-3) / 1e9, "ms": ms_u, "gbs": gbs, "frac": gbs / peak,
        "launches": len(plans), "what": "one uniform FP32 plan per length, data pre-sorted"}
    line["vs_per_length_uniform"] = line["forward"]["gpts"] / line["per_length_uniform_kernels"]["gpts"]
    if "default_forms" in line:
        line["tuned_vs_default_forms"] = line["forward"]["gpts"] / line["default_forms"]["gpts"]
    line["points"] = points
    line["workload"] = (f"batching: {lengths.size} transforms, lengths 2^U{{3..16}} (seed 4), "
                        f"{points} points, iid N(0,1); one persistent launch in a CUDA graph")
    return line


def run_workload(args) -> None:
    """Single-GPU measurements of the other configurations (one JSON line)."""
    import torch

    import workloads
    from paper_2504_07264_gb300 import build as cuda_build
    cuda_build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    peak = _peaks()["hbm_gbs"]
    line = {"workload": args.workload, "unit": UNIT, "peak_gbs": peak, "steps": args.steps,
            "warmup": args.warmup}
    if args.workload == "autograd":
        line.update(autograd_block(args.steps, args.warmup, stream))
        line["metric"] = "planar DFT Gpts/s, N=4096 B=16384, fwd + adj kernels and autograd step"
        line["value"] = line["forward"]["gpts"]
    elif args.workload == "precision":
        line.update(precision_block(args.steps, args.warmup, stream))
        line["metric"] = ("planar DFT Gpts/s, N=256 B=262144 |x| log-uniform: FP32 vs split-BF16 vs "
                          "split-FP16 tensor cores (and N=1024 B=65536)")
        line["value"] = line["paths"]["split_bf16"]["forward"]["gpts"]
    elif args.workload == "ragged":
        line.update(ragged_block(args.steps, args.warmup, stream))
        line["metric"] = ("planar DFT Gpts/s, ragged batch of 10000 transforms, lengths 2^U{3..16} "
                          "(seed 4), one persistent launch in a CUDA graph")
        line["value"] = line["forward"]["gpts"]
    elif args.workload == "uniform":
        n = args.n
        batch = args.batch or max(1, (1 << 26) // n)
        xr_h, xi_h = workloads.normal_planes(n, batch, seed=1)
        if args.schedule is not None:
            from paper_2504_07264_gb300 import sdft as S
            if S.sdft_schedule_select(n, args.dtype, args.schedule) != S.SDFT_OK:
                raise SystemExit(f"no schedule {args.schedule} for N={n} dtype {args.dtype}")
        line.update(_measure_uniform(n, batch, xr_h, xi_h, args.steps, args.warmup, stream,
                                     dtype=args.dtype))
        line["metric"] = f"planar DFT Gpts/s, N={n} B={batch} dtype {args.dtype}"
        line["value"] = line["forward"]["gpts"]
    elif args.workload == "sizes":
        rows = []
        for logn in range(1, 17):
            n = 1 << logn
            batch = (1 << 26) // n
            xr_h, xi_h = workloads.normal_planes(n, batch, seed=1)
            r = _measure_uniform(n, batch, xr_h, xi_h, max(20, args.steps // 10), args.warmup,
                                 stream)
            rows.append({k: r[k] for k in ("n", "batch", "forward", "adjoint", "schedule")})
            del xr_h, xi_h
        line["sizes"] = rows
        line["metric"] = "planar DFT Gpts/s per N, 2^26 points per step"
        line["value"] = None
    elif args.workload == "plain":
        # 1024 transforms of N = 16 (256 KiB moved): a latency-bound call,
        # reported in microseconds, with its error against a float64 FFT
        # (the tests check the same configuration against the oracle)
        import numpy as np

        from paper_2504_07264_gb300 import SDFT_FORWARD, Plan
        cfg = workloads.PLAIN
        n, batch = cfg["n"], cfg["batch"]
        xr_h, xi_h = workloads.plain()
        xr = torch.from_numpy(xr_h).cuda()
        xi = torch.from_numpy(xi_h).cuda()
        yr = torch.empty_like(xr)
        yi = torch.empty_like(xi)
        with Plan(n, batch) as plan:
            plan.execute(SDFT_FORWARD, xr, xi, yr, yi, stream)
            torch.cuda.synchronize()
            gr = yr.cpu().numpy().astype(np.float64)
            gi = yi.cpu().numpy().astype(np.float64)
            ref = np.fft.fft(xr_h.astype(np.float64) + 1j * xi_h.astype(np.float64), axis=1)
            rr, ri = ref.real, ref.imag
            rows = np.sqrt(((gr - rr) ** 2 + (gi - ri) ** 2).sum(1) / (rr ** 2 + ri ** 2).sum(1))
            fwd = lambda: plan.execute(SDFT_FORWARD, xr, xi, yr, yi, stream)  # noqa: E731
            for _ in range(args.warmup):
                fwd()
            torch.cuda.synchronize()
            ms = _time_steps(fwd, args.steps, stream)
            line.update({"n": n, "batch": batch, "schedule": plan.describe(),
                         "us_per_call": ms * 1e3, "gpts": n * batch / (ms * 1e-3) / 1e9,
                         "rel_l2_worst_transform": float(rows.max()),
                         "accuracy_reference": "float64 numpy.fft"})
        line["metric"] = "planar DFT, 1024 transforms of N=16 (uniform [-1,1), seed 0): us per call"
        line["value"] = ms * 1e3
        line["unit"] = "us"
        line["higher_is_better"] = False
    print(json.dumps(line), flush=True)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description="planar DFT benchmark (one JSON line)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the CPU oracle timing (it is on by default)")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the host-buffer end-to-end leg (it is on by default)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the differentiation, precision and batching configurations "
                         "measured after the headline (they are on by default)")
    ap.add_argument("--workload",
                    choices=("bandwidth", "autograd", "precision", "ragged", "sizes", "uniform",
                             "plain"),
                    default="bandwidth",
                    help="bandwidth (default) is the headline line; the others print one "
                         "single-GPU line of their own")
    ap.add_argument("--n", type=int, default=1024, help="length for --workload uniform")
    ap.add_argument("--dtype", type=int, default=0,
                    help="arithmetic path for --workload uniform (0 FP32, 1 split-BF16, 2 split-FP16)")
    ap.add_argument("--schedule", type=int, default=None,
                    help="compiled schedule index for --workload uniform (default: the tuned one)")
    ap.add_argument("--batch", type=int, default=None,
                    help="transforms per step (default: the workload's own batch, 65536 for "
                         "the headline; smaller only for profiling captures)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "bandwidth":
        run_workload(args)
    else:
        run_ours(args)
    return 0


if __name__ == "__main__":
    sys.exit(main())
