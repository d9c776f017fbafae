"""Benchmark: FP32 extended-stencil FDTD on a 256^3 periodic grid (plane wave, Courant 0.95
of the scheme's limit) -- forward and adjoint Gcell-updates/s, FP64 forward for comparison,
roofline fraction of the dominant kernel, end-to-end rate through the C ABI with host buffers,
and the FP64 CPU oracle as the reported baseline.

One "step" = one leapfrog step (B half step + E step) over the whole grid.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own replica (weak scaling, no collective on the
data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS = 256
LAMBDA = 16.0
COURANT = 0.95
SEED = 0
WORKLOAD = "3D FDTD 256^3 periodic, FP32 fields, extended curl-E stencil (seeded coefficient set 0), " \
           "plane wave lambda=16 along x, Courant 0.95 of the scheme's limit"
BYTES_FWD32 = 48.0    # E, B read once and written once per cell-update (FP32)
BYTES_FWD64 = 96.0
BYTES_ADJ32 = 60.0    # lambda (6) read+write, E^n (3) read
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the FP32 step
# kernel at 256^3, from one ncu capture of that kernel version; reported only
# while the kernel sources still hash to the captured version.
# PIC cycle workload (the paper's Sec. 6 setting): 512 x 256 x 256 FP32, 16-cell absorbing
# layers on +-y, +-z, a gamma = 10 electron bunch of 2^22 macro-particles along +x
PIC_SHAPE = (512, 256, 256)
PIC_N = 1 << 22
PIC_WORKLOAD = ("PIC cycle 512x256x256 FP32, 16-cell absorbing layers on y and z, extended "
                "stencil (seeded coefficient set 0), Courant 0.95; gamma=10 electron bunch, "
                "2^22 macro-particles, sigma_par=4, sigma_perp=8 cells, along +x")
STEP_TRAFFIC = {"sources_sha256_16": "7920d8a126534ed8", "bytes_per_launch": 828902144}
STEP_SOURCES = ["fdtd_fused32.cu", "fdtd_seg.cuh", "fdtd_tma.cuh", "fdtd_internal.cuh", "fdtd_tmem.cuh"]


def step_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1710_06829_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def step_traffic(n):
    """Captured DRAM bytes per launch of the step kernel, or None if stale or another size."""
    if n != N_CELLS or STEP_TRAFFIC["bytes_per_launch"] is None:
        return None
    if step_sources_sha() != STEP_TRAFFIC["sources_sha256_16"]:
        return None
    return STEP_TRAFFIC["bytes_per_launch"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_CELLS)
    p.add_argument("--slab", type=int, default=32, help="slab length of the temporally blocked leg")
    p.add_argument("--pipes", type=int, default=3, help="host-streaming pipelines of the e2e leg")
    p.add_argument("--part-e2e", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--part", default="all", choices=["all", "fwd32", "fwd32t2", "adj32", "pic", "fwd64", "norm"],
                   help="run one leg only (profiling driver: fwd32, adj32, pic, fwd64 = the FP64 "
                        "step, norm = the dispersion norm + gradient over the n^3 k-grid); prints "
                        "a short line that is not a bench result")
    return p.parse_args()


def coeffs():
    """Seeded coefficient set 0: first admissible draw of the seeded generator."""
    from paper_1710_06829_gb300 import inputs
    from paper_1710_06829_gb300 import sim as S
    s = SEED
    while True:
        beta, delta = inputs.random_theta(s, 3)
        _, smin, _ = S.dt_max(beta, delta, [1, 1, 1], 3)
        if smin >= 0:
            return beta, delta
        s += 1000


def coeffs_oracle():
    from oracle import dispersion as D
    from paper_1710_06829_gb300 import inputs
    s = SEED
    while True:
        beta, delta = inputs.random_theta(s, 3)
        smin, _ = D.S_extremes(beta, delta, [1, 1, 1], 3)
        if smin >= 0:
            return beta, delta
        s += 1000


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """SM clock and clock-event-reason samples inside [mark_start, mark_end].

    Samples come from NVML (libnvidia-ml through ctypes) every 2 ms on a background thread, so
    that a timed region of a few milliseconds still holds samples; where NVML cannot be loaded
    the sampler falls back to nvidia-smi at 50 ms (and, for a region shorter than that, to the
    samples nearest to it).  Nothing here changes a GPU setting: clocks and reasons are read."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    def __init__(self, index=0):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"fdtd_bench_clocks_{os.getpid()}.csv")
        self.index = index
        self.t0 = self.t1 = None
        self.nvml = None
        self.samples = []
        self.stop = False
        self.thread = None

    def _nvml_open(self):
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = C.c_void_p()
        ok = False
        try:   # the NVML device of this process's CUDA device, by PCI bus id
            import torch
            pr = torch.cuda.get_device_properties(self.index)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
            ok = lib.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(bus), C.byref(h)) == 0
        except Exception:  # noqa: BLE001
            ok = False
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.index), C.byref(h)) != 0:
            raise RuntimeError("no NVML handle")
        mx = C.c_uint()
        lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx))   # 1 = NVML_CLOCK_SM
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.nvml = (C, lib, h, reasons_fn, mx.value)

    def _poll(self):
        C, lib, h, reasons_fn, _ = self.nvml
        clk = C.c_uint()
        rs = C.c_ulonglong()
        while not self.stop:
            t = time.time()
            if lib.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0 and reasons_fn(h, C.byref(rs)) == 0:
                self.samples.append((t, clk.value, rs.value))
            time.sleep(0.002)

    def __enter__(self):
        try:
            import threading
            self._nvml_open()
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return self
        except Exception:  # noqa: BLE001
            self.nvml = None
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
            deadline = time.time() + 5.0
            while time.time() < deadline and os.path.getsize(self.path) == 0:
                time.sleep(0.05)
        except Exception:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        time.sleep(0.15)

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop = True
            self.thread.join(timeout=2)
            try:
                self.nvml[1].nvmlShutdown()
            except Exception:  # noqa: BLE001
                pass
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.nvml is not None:
            inside = [(c, r) for t, c, r in self.samples if self.t0 <= t <= self.t1]
            window = "timed region (NVML, 2 ms period)"
            if len(inside) < 2:
                mid = 0.5 * (self.t0 + self.t1)
                near = sorted(self.samples, key=lambda x: abs(x[0] - mid))[:3]
                inside = [(c, r) for _, c, r in near]
                window = "nearest samples (NVML)"
            reasons = sorted({n for _, r in inside for b, n in self.REASONS.items() if r & b})
            sm = [c for c, _ in inside]
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.nvml[4],
                    "reasons": reasons, "samples": len(inside), "window": window}
        import datetime as _dt
        try:
            rows = []
            for line in open(self.path).read().strip().splitlines():
                r = [x.strip() for x in line.split(",")]
                try:
                    ts = _dt.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, r))
                except ValueError:
                    continue
            inside = [r for ts, r in rows if self.t0 is not None and self.t0 <= ts <= self.t1]
            window = "timed region"
            if len(inside) < 2:
                # region shorter than the sampling period: take the samples closest to it
                mid = 0.5 * (self.t0 + self.t1)
                inside = [r for _, r in sorted(rows, key=lambda x: abs(x[0] - mid))[:3]]
                window = "nearest samples (timed region shorter than the sampling period)"
            sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
            mx = max(float(r[2]) for r in inside)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = sorted({names[i] for r in inside for i in range(4)
                              if r[5 + i].lower() == "active"})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                    "reasons": reasons, "samples": len(inside), "window": window}
        except Exception as e:  # noqa: BLE001
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": str(e)[:80]}


def dist_init(args, backend="nccl"):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier_max(x, world, device="cuda"):
    """Max of a per-rank time over all ranks (the job's time is its slowest replica)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------- reference arm


def _oracle_setup(n_cells):
    from oracle import dispersion as D
    from oracle import fdtd as F
    from paper_1710_06829_gb300 import inputs
    beta, delta = coeffs_oracle()
    dt = COURANT * D.dt_max(beta, delta, [1, 1, 1], 3)
    shape = (n_cells, n_cells, n_cells)
    kx = 2 * math.pi * round(n_cells / LAMBDA) / n_cells
    fields = inputs.plane_wave(shape, (kx, 0, 0), (0, 0, 1), [1, 1, 1])
    return F.State(fields[:3], fields[3:]), F.Coeffs(beta, delta, [1, 1, 1], dt)


def _oracle_worker(args):
    """One process: whole FP64 oracle steps on its own copy of the workload until the budget
    is spent (at least one step); returns (steps, seconds)."""
    n_cells, budget_s, max_steps = args
    from oracle import fdtd as F
    s, c = _oracle_setup(n_cells)
    steps = 0
    t0 = time.perf_counter()
    while True:
        F.step(s, c)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= max_steps:
            return steps, el


def cpu_oracle_rate(n_cells, budget_s=12.0, n_all=128):
    """FP64 numpy oracle forward rate on this host: one process on the full grid (whole steps,
    bounded sample), and one process per host core, each stepping its own n_all^3 copy of the
    workload (aggregate rate).  numpy's elementwise arithmetic is single-threaded, so one
    process uses one core."""
    import multiprocessing as mp
    steps, el = _oracle_worker((n_cells, budget_s, 20))
    one = steps * float(n_cells) ** 3 / el / 1e9
    cores = os.cpu_count() or 1
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, [(n_all, budget_s, 1000)] * cores)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    wall = max(e for _, e in res)
    allc = sum(st for st, _ in res) * float(n_all) ** 3 / wall / 1e9
    return {"value": allc, "unit": "Gcell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes (one per host core), each stepping its own {n_all}^3 copy "
                      f"of the workload with the FP64 numpy oracle for ~{budget_s:.0f} s",
            "single_core": {"value": one, "unit": "Gcell-updates/s", "cores": 1,
                            "sample": f"{steps} FP64 numpy oracle steps on the full {n_cells}^3 grid "
                                      f"in {el:.1f} s, one process"}}


def run_reference(args):
    """The paper ships no code, so the reference arm is the FP64 numpy oracle: one step = one
    leapfrog step of the oracle on a 64^3 sample of the same workload (same coefficients,
    Courant number and plane wave), timed on the host cores.  Under torchrun only rank 0 runs."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import dispersion as D
    from oracle import fdtd as F
    from paper_1710_06829_gb300 import inputs
    ns = 64
    beta, delta = coeffs_oracle()
    dt = COURANT * D.dt_max(beta, delta, [1, 1, 1], 3)
    kx = 2 * math.pi * round(ns / LAMBDA) / ns
    fields = inputs.plane_wave((ns, ns, ns), (kx, 0, 0), (0, 0, 1), [1, 1, 1])
    s = F.State(fields[:3], fields[3:])
    c = F.Coeffs(beta, delta, [1, 1, 1], dt)
    for _ in range(args.warmup):
        F.step(s, c)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        F.step(s, c)
    el = time.perf_counter() - t0
    cells = float(ns) ** 3
    value = args.steps * cells / el / 1e9
    line = {"impl": "reference", "metric": "Gcell-updates/s", "value": value,
            "unit": "Gcell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_grid": [ns, ns, ns]},
            "cpu_baseline": {"value": value, "unit": "Gcell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} FP64 numpy oracle steps on a {ns}^3 sample of "
                                       f"the workload ({el:.1f} s, single thread)"},
            "e2e": {"value": value, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------- our arm


REPEATS = 5   # each timed region is repeated; the median per-step time is reported


def time_median(fn, steps, stream, repeats=REPEATS):
    """Median over `repeats` CUDA-event timings of `steps` calls, and the individual times."""
    ts = [time_events(fn, steps, stream) for _ in range(repeats)]
    return statistics.median(ts), ts


def time_events(fn, steps, stream):
    import torch
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(steps):
        fn()
    stop.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(stop) / 1e3


def pic_leg(S, inputs, beta, delta, dt, stream, world, args):
    """PIC cycles (fdtd_pic_step) of the bunch workload: whole cycles timed with CUDA events,
    and the same cycles without particles (the field part) for the split."""
    import numpy as np
    import torch
    nx, ny, nz = PIC_SHAPE
    sm = S.Simulation(PIC_SHAPE, [1, 1, 1], dt, beta, delta, dims=3, dtype="f32",
                      absorb_cells=16, absorb_sigma=0.5, stream=stream)
    sm.set_state([None] * 6)
    x, u = inputs.gaussian_bunch(PIC_N, (64.0, ny / 2, nz / 2), (4.0, 8.0), (1.0, 0.0, 0.0), 10.0,
                                 seed=21)
    sp = S.Species(torch.from_numpy(x.astype(np.float32)).cuda(),
                   torch.from_numpy(u.astype(np.float32)).cuda(), -1.0 / PIC_N, -1.0)
    empty = S.Species(torch.empty((3, 0), device="cuda"), torch.empty((3, 0), device="cuda"), 0.0,
                      1.0)
    for _ in range(max(3, args.warmup)):
        sm.pic_step(1, [sp])
    k = max(5, min(args.steps, 50))
    t_cyc = barrier_max(time_events(lambda: sm.pic_step(1, [sp]), k, stream), world)
    t_fld = barrier_max(time_events(lambda: sm.pic_step(1, [empty]), k, stream), world)
    sm.sync()
    sm.close()
    cells = float(nx * ny * nz)
    peak, peak_kind = peaks()
    t_push = max(t_cyc - t_fld, 1e-12) / k
    push_gbs = 48.0 * PIC_N / t_push / 1e9   # particle state read + written, FP32
    return {"value": world * PIC_N * k / t_cyc / 1e9, "unit": "Gparticle-pushes/s",
            "push_roofline": {"bound": "latency (gathers) and same-address reductions in L2, "
                                       "not HBM", "algorithmic_bytes_per_push": 48,
                              "achieved": push_gbs, "peak": peak, "unit": "GB/s",
                              "frac": push_gbs / peak, "peak_kind": peak_kind},
            "workload": PIC_WORKLOAD, "particles": PIC_N, "cycles": k,
            "ms_per_cycle": t_cyc / k * 1e3, "field_ms_per_cycle": t_fld / k * 1e3,
            "push_ms_per_cycle": (t_cyc - t_fld) / k * 1e3,
            "push_rate": {"value": PIC_N * k / max(t_cyc - t_fld, 1e-12) / 1e9,
                          "unit": "Gparticle-pushes/s", "note": "gather + Boris + Esirkepov "
                          "deposit alone (cycle minus the particle-free cycle)"},
            "cycle_cell_rate": {"value": world * cells * k / t_cyc / 1e9, "unit": "Gcell-updates/s"}}


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    from paper_1710_06829_gb300 import _lib as L
    from paper_1710_06829_gb300 import inputs
    from paper_1710_06829_gb300 import sim as S

    n = args.n
    shape = (n, n, n)
    cells = float(n) ** 3
    beta, delta = coeffs()
    dtm, _, _ = S.dt_max(beta, delta, [1, 1, 1], 3)
    dt = COURANT * dtm
    kx = 2 * math.pi * round(n / LAMBDA) / n
    fields64 = inputs.plane_wave(shape, (kx, 0, 0), (0, 0, 1), [1, 1, 1])
    fields = [torch.from_numpy(f.astype(np.float32)) for f in fields64]
    stream = torch.cuda.current_stream()

    if args.part == "norm":
        for _ in range(max(1, args.warmup)):
            S.disp_norm(beta, delta, dt, [1, 1, 1], 3, (n, n, n))
        t = time_events(lambda: S.disp_norm(beta, delta, dt, [1, 1, 1], 3, (n, n, n)), args.steps, stream)
        if rank == 0:
            print(json.dumps({"part": "norm", "gpoints_per_s": cells * args.steps / t / 1e9,
                              "ms_per_call": t / args.steps * 1e3}))
        return
    if args.part == "fwd64":
        sm64 = S.Simulation(shape, [1, 1, 1], dt, beta, delta, dims=3, dtype="f64", stream=stream)
        sm64.set_state([torch.from_numpy(f) for f in fields64])
        for _ in range(max(1, args.warmup)):
            sm64.step(1)
        t = time_events(lambda: sm64.step(1), args.steps, stream)
        sm64.close()
        if rank == 0:
            print(json.dumps({"part": "fwd64", "gcells_per_s": cells * args.steps / t / 1e9,
                              "ms_per_step": t / args.steps * 1e3}))
        return

    # --- forward FP32
    sm = S.Simulation(shape, [1, 1, 1], dt, beta, delta, dims=3, dtype="f32", stream=stream)
    sm.set_state(fields)
    for _ in range(max(3, args.warmup)):
        sm.step(1)
    barrier(world)
    with Clocks(local) as clk:
        clk.mark_start()
        t_fwd, t_fwd_all = time_median(lambda: sm.step(1), args.steps, stream)
        clk.mark_end()
    t_fwd = barrier_max(t_fwd, world)
    fwd = world * cells * args.steps / t_fwd / 1e9
    if args.part == "fwd32":
        sm.close()
        if rank == 0:
            print(json.dumps({"part": "fwd32", "gcells_per_s": fwd, "ms_per_step": t_fwd / args.steps * 1e3}))
        return

    # --- the same steps temporally blocked (pairs slab by slab through L2)
    sm.set_temporal_blocking(2, args.slab)
    for _ in range(2):
        sm.step(2)
    k2 = max(1, args.steps // 2)
    t_t2, _ = time_median(lambda: sm.step(2), k2, stream)
    t_t2 = barrier_max(t_t2, world)
    sm.set_temporal_blocking(1)
    fwd_t2 = world * cells * 2 * k2 / t_t2 / 1e9
    if args.part == "fwd32t2":
        sm.close()
        if rank == 0:
            print(json.dumps({"part": "fwd32t2", "slab": args.slab, "gcells_per_s": fwd_t2,
                              "ms_per_step": t_t2 / (2 * k2) * 1e3}))
        return

    # --- adjoint FP32 (record a segment, then reverse it)
    seg = min(args.steps, 20)
    sm.step(seg, record=True)
    sm.set_adjoint([f for f in fields])
    grad = torch.zeros(12, dtype=torch.float64, device="cuda")
    sm.step_adjoint(2, grad)    # warm-up
    t_adj_all = []
    for _ in range(REPEATS):    # each repetition reverses a freshly recorded segment
        sm.step(seg, record=True)
        torch.cuda.synchronize()
        t_adj_all.append(time_events(lambda: sm.step_adjoint(seg, grad), 1, stream))
    t_adj = barrier_max(statistics.median(t_adj_all), world)
    adj = world * cells * seg / t_adj / 1e9
    if args.part == "adj32":
        sm.close()
        if rank == 0:
            print(json.dumps({"part": "adj32", "gcells_per_s": adj, "ms_per_step": t_adj / seg * 1e3}))
        return

    # --- PIC cycle: bunch of macro-particles on the 512 x 256 x 256 absorbing-layer grid
    pic = pic_leg(S, inputs, beta, delta, dt, stream, world, args) if not args.part_e2e else None
    if args.part == "pic":
        sm.close()
        if rank == 0:
            print(json.dumps({"part": "pic", **pic}))
        return

    # --- end to end through the C ABI with host buffers: upload, 20 steps, download
    n_inner = 20
    pinned_in = [f.pin_memory() for f in fields]
    pinned_out = [torch.empty_like(f).pin_memory() for f in fields]

    def e2e_step():
        sm.set_state_host(pinned_in)
        sm.step(n_inner)
        sm.get_state_host(pinned_out)
    e2e_step()
    e2e_reps = 10
    times = []
    for _ in range(e2e_reps):   # each repetition ends with the host read-back (synchronous)
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t_e2e1 = barrier_max(statistics.median(times), world)
    e2e_single = world * cells * n_inner / t_e2e1 / 1e9
    sm.close()
    # several pipelines: one handle per pipeline on its own stream, each driven by its own host
    # thread through the same calls (upload, 20 steps, download), so that one pipeline's copies
    # overlap the others' kernels; every e2e step still uploads its inputs and downloads its result
    import threading
    npipe, reps_p = max(1, args.pipes), 6
    sims = [S.Simulation(shape, [1, 1, 1], dt, beta, delta, dims=3, dtype="f32",
                         stream=torch.cuda.Stream()) for _ in range(npipe)]
    p_in = [[f.pin_memory() for f in fields] for _ in range(npipe)]
    p_out = [[torch.empty_like(f).pin_memory() for f in fields] for _ in range(npipe)]

    def pipe_step(k):
        sims[k].set_state_host(p_in[k])
        sims[k].step(n_inner)
        sims[k].get_state_host(p_out[k])

    def pipe_run(k, reps):
        for _ in range(reps):
            pipe_step(k)
    for k in range(npipe):
        pipe_step(k)          # warm-up (creates each handle's copy stream)
    torch.cuda.synchronize()
    # the pipelined region, repeated; the median is reported (the host link is shared with the
    # rest of the machine, and a transient slowdown of one repetition should not set the figure)
    t_pipes = []
    for _ in range(REPEATS):
        barrier(world)
        t0 = time.perf_counter()
        threads = [threading.Thread(target=pipe_run, args=(k, reps_p)) for k in range(npipe)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        torch.cuda.synchronize()
        t_pipes.append(time.perf_counter() - t0)
    t_pipe = barrier_max(statistics.median(t_pipes), world)
    e2e = world * cells * n_inner * npipe * reps_p / t_pipe / 1e9
    ok_pipe = all(torch.equal(a, b) for k in range(1, npipe) for a, b in zip(p_out[0], p_out[k]))
    for x in sims:
        x.close()
    if args.part_e2e:
        if rank == 0:
            print(json.dumps({"part": "e2e", "pipelines": npipe, "e2e": e2e, "single": e2e_single,
                              "agree": ok_pipe}))
        return
    # the host link alone: plain copies of the same pinned buffers; with the step time this gives
    # the rate an upload + steps + download cannot exceed on this link
    dev_bufs = [torch.empty_like(f, device="cuda") for f in fields]
    for d, h in zip(dev_bufs, pinned_in):
        d.copy_(h, non_blocking=True)
    t_h2d = statistics.median(
        time_events(lambda: [d.copy_(h, non_blocking=True) for d, h in zip(dev_bufs, pinned_in)], 1,
                    stream) for _ in range(REPEATS))
    t_d2h = statistics.median(
        time_events(lambda: [h.copy_(d, non_blocking=True) for d, h in zip(dev_bufs, pinned_out)], 1,
                    stream) for _ in range(REPEATS))
    del dev_bufs
    link_bytes = 6 * 4 * cells
    # one pipeline cannot beat upload + steps + download in sequence; overlapped pipelines cannot
    # beat the busiest of the link directions and the GPU
    e2e_ceiling = world * cells * n_inner / (t_h2d + n_inner * t_fwd / args.steps + t_d2h) / 1e9
    e2e_ceiling_pipe = world * cells * n_inner / max(t_h2d, t_d2h, n_inner * t_fwd / args.steps) / 1e9

    # --- FP64 forward for comparison
    sm64 = S.Simulation(shape, [1, 1, 1], dt, beta, delta, dims=3, dtype="f64", stream=stream)
    sm64.set_state([torch.from_numpy(f) for f in fields64])
    for _ in range(3):
        sm64.step(1)
    k64 = max(3, args.steps // 50)
    t64 = barrier_max(time_median(lambda: sm64.step(1), k64, stream)[0], world)
    fwd64 = world * cells * k64 / t64 / 1e9
    sm64.close()

    # --- dispersion norm + gradient over the 256^3 k-grid (FP64 per point and accumulation)
    t_norm = time_events(lambda: S.disp_norm(beta, delta, dt, [1, 1, 1], 3, (n, n, n)), 3, stream)
    norm_rate = cells * 3 / t_norm / 1e9

    if rank != 0:
        return
    peak, peak_kind = peaks()
    achieved = BYTES_FWD32 * cells / (t_fwd / args.steps) / 1e9
    line = {
        "metric": "Gcell-updates/s", "value": fwd, "unit": "Gcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_fwd / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [n, n, n], "l2": "inputs larger than L2 "
                   "(state 6 x 4 B x 256^3 = 403 MB per copy)", "parallelism": f"replicas x{world}"},
        "timing": {"repeats": REPEATS, "forward_region_ms": [t * 1e3 for t in t_fwd_all],
                   "adjoint_region_ms": [t * 1e3 for t in t_adj_all],
                   "note": "value, adjoint and fp64_forward are medians over the repetitions"},
        "adjoint": {"value": adj, "unit": "Gcell-updates/s", "steps": seg,
                    "roofline_frac": BYTES_ADJ32 * cells * seg / t_adj / 1e9 / peak},
        "temporal_blocking": {"value": fwd_t2, "unit": "Gcell-updates/s", "slab_planes": args.slab,
                              "ms_per_step": t_t2 / (2 * k2) * 1e3,
                              "effective_frac": BYTES_FWD32 * cells * 2 * k2 / t_t2 / 1e9 / peak,
                              "note": "pairs of steps slab by slab through L2 "
                                      "(fdtd_set_temporal_blocking); off by default: slower"},
        "dispersion_norm": {"value": norm_rate, "unit": "Gpoint/s", "grid": [n, n, n],
                            "note": "value and 13-entry gradient, FP64"},
        "fp64_forward": {"value": fwd64, "unit": "Gcell-updates/s",
                         "roofline_frac": BYTES_FWD64 * cells * k64 / t64 / 1e9 / peak},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": step_traffic(n),
                     "traffic_unit": "DRAM bytes per launch (ncu)", "peak_kind": peak_kind,
                     "kernel": "forward step (48 B/cell-update algorithmic)"},
        "pic": pic,
        "e2e": {"value": e2e, "unit": "Gcell-updates/s",
                "h2d_bytes_per_step": int(6 * 4 * cells), "d2h_bytes_per_step": int(6 * 4 * cells),
                "step": f"host upload + {n_inner} leapfrog steps + host download, through the C ABI "
                        f"with pinned host buffers; {npipe} pipelines ({npipe} handles on their own "
                        f"streams, one host thread each) x {reps_p} steps, wall clock, median of "
                        f"{REPEATS} repetitions of that region",
                "region_ms": [t * 1e3 for t in t_pipes],
                "pipelines": npipe, "pipelines_agree": ok_pipe,
                "ceiling": e2e_ceiling_pipe, "frac_of_ceiling": e2e / e2e_ceiling_pipe,
                "link_h2d_gbs": link_bytes / t_h2d / 1e9, "link_d2h_gbs": link_bytes / t_d2h / 1e9,
                "single_pipeline": {"value": e2e_single, "unit": "Gcell-updates/s",
                                    "step": f"one handle, median of {e2e_reps} repetitions",
                                    "ceiling": e2e_ceiling,
                                    "frac_of_ceiling": e2e_single / e2e_ceiling}},
        "gpu_launches": REPEATS * args.steps * (1 if (n % 64 == 0 and n % 8 == 0) else 2),
        "clocks": clk.summary(),
    }
    if world == 1:
        line["cpu_baseline"] = cpu_oracle_rate(n)
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
