"""Autotuner for the per-length schedules of libsdft.so.

Every transform length has one or more compiled schedules (radix split,
threads per transform, transforms per CTA, register-DFT order).  ``tune``
times each of them on the GPU through the C ABI's ``sdft_autotune`` (CUDA
events, the caller's buffers) and records the fastest; ``apply`` selects the
recorded schedules for the plans created afterwards.  Results are kept as JSON
keyed by GPU name, dtype and N:

    {"NVIDIA GB300": {"0": {"1024": {"index": 0, "ms": [...], "schedules": [...]}},
                      "ragged": {"32768": 1, ...}}}

The "ragged" entry holds the form of every length in the persistent kernel of
ragged plans (``tune_ragged``: the plan tuner of the C ABI run on the ragged
workload), applied with ``sdft_ragged_form_select``.

At import of the package nothing is changed; ``ensure_applied()`` (called by
``Plan``) loads the file named by the environment variable SDFT_TUNE_CACHE, or
else the table shipped with the package (``tuned_schedules.json``), once.

CLI:  python -m paper_2504_07264_gb300.autotune [--out FILE] [--points P] [--reps R]
                                               [--sizes N [N ...]] [--ragged]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading

from . import sdft as S

HERE = os.path.dirname(os.path.abspath(__file__))
SHIPPED = os.path.join(HERE, "tuned_schedules.json")

_applied = False
_lock = threading.Lock()


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


MARGIN = 0.01   # a schedule replaces the default only if it is >1 % faster


def pick(ms: list[float]) -> int:
    """The fastest schedule, unless it beats schedule 0 by no more than MARGIN
    (timing noise): then schedule 0."""
    best = min(range(len(ms)), key=lambda i: ms[i])
    return best if ms[best] < (1.0 - MARGIN) * ms[0] else 0


def tune_one(n: int, dtype: int = S.SDFT_F32, points: int = 1 << 26, reps: int = 20,
             stream=None) -> dict:
    """Time every schedule of length n on ``points`` complex values of random
    data (forward); selects the fastest (see ``pick``) and returns its record."""
    import ctypes

    import torch
    batch = max(1, points // n)
    count = S.sdft_schedule_count(n, dtype)
    if count < 0:
        raise S.SdftError(-count, f"sdft_schedule_count({n})")
    g = torch.Generator(device="cuda").manual_seed(n)
    xr = torch.randn(batch * n, device="cuda", generator=g)
    xi = torch.randn(batch * n, device="cuda", generator=g)
    yr = torch.empty_like(xr)
    yi = torch.empty_like(xi)
    ms = (ctypes.c_float * count)()
    st = int((stream or torch.cuda.current_stream()).cuda_stream)
    best = S.sdft_autotune(n, batch, dtype, xr.data_ptr(), xi.data_ptr(), yr.data_ptr(),
                           yi.data_ptr(), reps, ctypes.addressof(ms), st)
    if best < 0:
        raise S.SdftError(-best, f"sdft_autotune({n})")
    times = [float(v) for v in ms]
    best = pick(times)
    S.lib().sdft_schedule_select(n, dtype, best)
    return {"index": int(best), "ms": times, "batch": batch,
            "schedules": [S.sdft_schedule_describe(n, dtype, i) for i in range(count)]}


def tune(sizes=None, dtype: int = S.SDFT_F32, points: int = 1 << 26, reps: int = 20) -> dict:
    """Tune every length in ``sizes`` (default 2 .. 65536); returns the table
    for this GPU: {str(dtype): {str(n): record}}."""
    sizes = [1 << m for m in range(1, 17)] if sizes is None else sizes
    out = {}
    for n in sizes:
        if S.sdft_schedule_count(n, dtype) <= 1:
            continue
        out[str(n)] = tune_one(n, dtype, points, reps)
    return {str(dtype): out}


def tune_ragged(reps: int = 5, stream=None) -> dict:
    """Run the work-queue plan tuner (``sdft_plan_ragged_autotune``) on the
    ragged workload (10000 transforms, lengths 2^U{3..16}, seed 4) and select
    the forms it keeps for later plans; returns {"ragged": {str(n): form}}
    for every length 4 .. 65536 (lengths the workload lacks keep form 0)."""
    import torch
    root = os.path.dirname(HERE)
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads
    lengths, _, xr_h, xi_h = workloads.ragged_planes()
    xr = torch.from_numpy(xr_h).cuda()
    xi = torch.from_numpy(xi_h).cuda()
    yr, yi = torch.empty_like(xr), torch.empty_like(xi)
    with S.Plan(lengths=lengths) as plan:
        plan.ragged_autotune(xr, xi, yr, yi, reps=reps, stream=stream)
        forms = {}
        for logn in range(2, 17):
            n = 1 << logn
            forms[str(n)] = plan.ragged_form(n) if (lengths == n).any() else 0
    for n, f in forms.items():
        S.lib().sdft_ragged_form_select(int(n), int(f))
    return {"ragged": forms}


def apply(table: dict, name: str | None = None) -> int:
    """Select the recorded schedules (and work-queue forms) of GPU ``name``
    (default: the current one); returns how many lengths were set."""
    if name is None:
        name = gpu_name()
    applied = 0
    for dtype, per_n in table.get(name, {}).items():
        if dtype == "ragged":
            for n, form in per_n.items():
                if 0 <= int(form) < max(0, S.sdft_ragged_form_count(int(n))) and \
                        S.lib().sdft_ragged_form_select(int(n), int(form)) == S.SDFT_OK:
                    applied += 1
            continue
        for n, rec in per_n.items():
            idx = int(rec["index"])
            if idx < S.sdft_schedule_count(int(n), int(dtype)) and \
                    S.lib().sdft_schedule_select(int(n), int(dtype), idx) == S.SDFT_OK:
                applied += 1
    return applied


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)


def save(table: dict, path: str, name: str | None = None) -> None:
    """Merge this GPU's ``table`` into the JSON file at ``path``."""
    if name is None:
        name = gpu_name()
    full = load(path) if os.path.exists(path) else {}
    mine = full.setdefault(name, {})
    for dtype, per_n in table.items():
        mine.setdefault(dtype, {}).update(per_n)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(full, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def ensure_applied() -> None:
    """Apply the tuning file once per process (SDFT_TUNE_CACHE, else the
    shipped table); silently does nothing if neither exists."""
    global _applied
    with _lock:
        if _applied:
            return
        _applied = True
        path = os.environ.get("SDFT_TUNE_CACHE") or SHIPPED
        if os.path.exists(path):
            try:
                apply(load(path))
            except Exception:
                pass


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description="time every schedule and record the fastest")
    ap.add_argument("--out", default=os.environ.get("SDFT_TUNE_CACHE") or SHIPPED)
    ap.add_argument("--points", type=int, default=1 << 26)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--sizes", type=int, nargs="+", default=None,
                    help="lengths to tune (default: every power of two 2 .. 65536); the "
                         "others keep their entries in --out")
    ap.add_argument("--ragged", action="store_true",
                    help="tune only the work-queue forms of ragged plans, on the ragged workload")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    if a.ragged:
        ensure_applied()
        table = tune_ragged()
        save(table, a.out)
        print("ragged forms:", table["ragged"])
        print(f"wrote {a.out}")
        return 0
    table = tune(sizes=a.sizes, points=a.points, reps=a.reps)
    save(table, a.out)
    for dtype, per_n in table.items():
        for n, rec in sorted(per_n.items(), key=lambda kv: int(kv[0])):
            times = ", ".join(f"{t * 1e3:.1f}" for t in rec["ms"])
            print(f"N={n:>6}: best {rec['index']}  (us/launch: {times})")
    print(f"wrote {a.out}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
