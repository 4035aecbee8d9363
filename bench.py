"""Benchmark of the MultiFab time-step sweep (FillBoundary + flux-form stencil) on GB300.

One bench step = one call of mf_advance over the whole workload: 100 forward-Euler time
steps of the periodic 256^3 heat equation in 64 boxes of 64^3 with one ghost cell (the
paper's Sec. 4.1 test scaled to one GPU), every time step a FillBoundary launch and a
persistent stencil launch, replayed as one CUDA graph.  Metric: cell-updates per second
including the ghost fill.  The headline runs FP32 storage/arithmetic; the same line also
reports the FP64 batched sweep and the FP64 plain per-box sweep (Sec. 3.1 untiled MFIter
baseline) and their ratio.

Timing: CUDA events on the launching stream, W untimed warm-ups, K timed steps, the L2 cache
flushed (a 512 MB write) before every timed step; max over ranks.  Under torchrun every rank
runs an independent replica (weak scaling; the sweep has no cross-GPU exchange here).

--impl reference times the FP64 CPU oracle (the plain definition the GPU path is checked
against) on the host cores: one bench step = one oracle time step of the same 256^3 grid.
"""
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "c2"
METRIC = "cell-updates/s per step incl. ghost fill"
UNIT = "cell-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--dtype", default="f32", choices=["f32", "f64", "bf16"])
    p.add_argument("--no-extras", action="store_true", help="headline only (no FP64, e2e, CPU baseline)")
    p.add_argument("--tile", default=None, help="fixed tile 'x,y,z' instead of the autotuner (0 = whole box)")
    p.add_argument("--kernel", default="tma", choices=["tma", "global"], help="stencil kernel variant")
    p.add_argument("--only", default=None,
                   choices=["bf16_batched", "rk3_8th", "amr2lev_reflux", "manybox512", "fp64_fixed", "diff8th512"],
                   help="run only this secondary line (for profiling) and print it")
    p.add_argument("--schedule", default=None,
                   help="fixed schedule 'x,y,z,rows,stages,group_bytes' instead of the autotuner")
    p.add_argument("--fixed", action="store_true",
                   help="headline with --dtype f64: fixed-point differences (MF_FIXED_DIFF)")
    p.add_argument("--c3-n", type=int, default=None,
                   help="with --only diff8th512: domain edge N instead of 512 (a smaller level to profile)")
    p.add_argument("--c3-dtype", default="f32,f64", help="with --only diff8th512: storage types to run")
    p.add_argument("--c5", default=None,
                   help="with --only manybox512: run one level, 'boxes,storage[,max_region]' (storage f32 or "
                        "f64fixed), for profiling")
    p.add_argument("--plain", action="store_true",
                   help="headline as the untiled per-box sweep (MF_PLAIN_PER_BOX), for profiling the baseline")
    a = p.parse_args()
    if a.fixed and a.dtype != "f64":
        p.error("--fixed needs --dtype f64")
    if a.plain and (a.fixed or not a.no_extras):
        p.error("--plain profiles the headline alone: with --no-extras, without --fixed")
    return a


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def level_bytes(N, mgs, g, C, S):
    """Bytes of one time level of the N^3 domain chopped into boxes of mgs^3: each FArrayBox
    spans its grown box in rows of whole 32-byte sectors (the low side padded so that valid x = 0
    starts a sector) and starts on a 256-byte boundary."""
    e = 32 // S
    fpad = (e - g % e) % e
    px = -(-(fpad + mgs + 2 * g) // e) * e
    fab = px * (mgs + 2 * g) ** 2 * C
    fab = -(-fab // (256 // S)) * (256 // S)
    return (N // mgs) ** 3 * fab * S


def workload_config(cfg):
    N = cfg["N"]
    ws_mb = 2 * level_bytes(N, cfg["max_grid_size"], cfg["ngrow"], cfg["ncomp"], 4) / 1e6
    return {"workload": "%s: periodic %d^3, %d boxes of %d^3, ngrow %d, %d comp, 7-point flux-form heat "
                        "stencil, %d time steps per bench step" % (cfg["name"], N, (N // cfg["max_grid_size"]) ** 3,
                                                                   cfg["max_grid_size"], cfg["ngrow"], cfg["ncomp"],
                                                                   cfg["nsteps"]),
            "domain": N, "max_grid_size": cfg["max_grid_size"], "ngrow": cfg["ngrow"], "ncomp": cfg["ncomp"],
            "stencil_radius": cfg["R"], "time_steps_per_bench_step": cfg["nsteps"],
            "initial_data": "8 seeded sine modes, |k_d| in 1..16",
            "l2": "flushed (512 MB write, then 512 MB read) before every timed bench step; per-step working "
                  "set (two FP32 time levels incl. ghosts) %.0f MB, larger than the 129 MB L2" % ws_mb}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ reference arm (oracle on the host)

def run_reference(args, cfg):
    import oracle
    N = cfg["N"]
    lo, hi = [0, 0, 0], [N - 1] * 3
    L = oracle.Level(oracle.chop(lo, hi, cfg["max_grid_size"]), lo, hi, cfg["ngrow"], cfg["ncomp"])
    u = L.from_dense(synth.initial_field(cfg))
    lam = 1.0 * synth.dt_for(cfg) * float(N * N)
    for _ in range(args.warmup):
        u = oracle.advance(L, u, cfg["R"], lam, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u = oracle.advance(L, u, cfg["R"], lam, 1)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    V = N ** 3
    value = V * args.steps / total
    sample = "one FP64 oracle time step (FillBoundary + flux-form stencil) of the %d^3 / %d-box grid per bench " \
             "step, single-threaded C (gcc -O2)" % (N, (N // cfg["max_grid_size"]) ** 3)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(cfg),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def cpu_baseline(cfg, target_s=15.0):
    """The oracle as it stands on the host cores: single-threaded (the reported baseline), and
    with the paper's threaded loop over boxes (Sec. 3.3) on every core, on the same steps, with
    a check that both give the same bits."""
    import oracle
    N = cfg["N"]
    lo, hi = [0, 0, 0], [N - 1] * 3
    L = oracle.Level(oracle.chop(lo, hi, cfg["max_grid_size"]), lo, hi, cfg["ngrow"], cfg["ncomp"])
    u = L.from_dense(synth.initial_field(cfg))
    lam = 1.0 * synth.dt_for(cfg) * float(N * N)
    t0 = time.perf_counter()
    u = oracle.advance(L, u, cfg["R"], lam, 1)
    t1 = time.perf_counter() - t0
    n = max(1, min(cfg["nsteps"], int(target_s / max(t1, 1e-3)) - 1))
    t0 = time.perf_counter()
    serial = oracle.advance(L, u, cfg["R"], lam, n)
    t = time.perf_counter() - t0
    threads = oracle.omp_threads()
    t0 = time.perf_counter()
    threaded = oracle.advance_omp(L, u, cfg["R"], lam, n)
    t_omp = time.perf_counter() - t0
    nbox = (N // cfg["max_grid_size"]) ** 3
    return {"value": N ** 3 * n / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d of the %d FP64 time steps of the %d^3 / %d-box workload, single-threaded C oracle "
                      "(gcc -O2 -ffp-contract=off) on the GPU host" % (n, cfg["nsteps"], N, nbox),
            "openmp": {"value": N ** 3 * n / t_omp, "unit": UNIT, "cores": threads, "nproc": os.cpu_count(),
                       "kind": "oracle, boxes of each phase shared among OpenMP threads (Sec. 3.3)",
                       "sample": "the same %d steps" % n,
                       "bitwise_equal_to_single_thread": bool(np.array_equal(serial, threaded))}}


# ------------------------------------------------------------------ our arm

KERNEL_SOURCES = {
    "k_stencil_tma": ["stencil_tma_kernel.cuh", "stencil_tma.cu", "stencil_tma_fix.cu", "fixed_diff.cuh",
                      "stencil_common.cuh", "mf_internal.h"],
    "k_stencil": ["mf_kernels.cu", "stencil_common.cuh", "mf_internal.h"],
}


def src_hash(kernel):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1604_03570_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel, workload_key, dtype):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    rec = t.get("%s|%s|%s" % (kernel, workload_key, dtype))
    if not rec or rec.get("src_sha") != src_hash(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


# floating-point operations per cell of one flux-form update: 3 face fluxes per cell (each face
# is shared by two cells; radius 1: one subtraction, radius R > 1: R subtractions, R
# multiplications, R - 1 additions), 5 additions for the divergence, one multiply-add
FLOPS_PER_CELL = {1: 3 * 1 + 5 + 2, 2: 3 * (3 * 2 - 1) + 5 + 2, 4: 3 * (3 * 4 - 1) + 5 + 2}


def fp64_peak_tflops():
    """FP64 FMA throughput of this GPU, measured by the library's DFMA loop."""
    import paper_1604_03570_gb300 as mf
    return mf.mf_fp64_fma_rate()


def time_advances(mfab, R, D, dt, nsteps, K, flush, flags=0):
    import torch
    import paper_1604_03570_gb300 as mf
    s = mfab.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        flush()
        ev[k][0].record(s)
        mf.mf_advance(mfab.h, R, D, dt, nsteps, flags)
        ev[k][1].record(s)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself on one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, units_per_rank, seconds):
    """Units all ranks processed per second of the slowest rank (weak scaling: every rank
    processes the same units)."""
    return ws * units_per_rank / seconds


RK3_CFG = dict(N=256, max_grid_size=64, ngrow=4, ncomp=1, R=4, nsteps=20, dtype="f32", nmodes=8, kmax=8)


def stencil_phase(mfab, R, D, dt, nsteps, flags, steps, flush):
    """Device time of the stencil launches of one advance, from the events the graph records
    wherever the kind of launch changes: (average stencil launch in s, fill ms per advance,
    launch counts)."""
    import paper_1604_03570_gb300 as mf
    mf.mf_set_timing(mfab.h, 1)
    for _ in range(2):
        mf.mf_advance(mfab.h, R, D, dt, nsteps, flags)
    fill_ms = st_ms = 0.0
    for _ in range(steps):
        time_advances(mfab, R, D, dt, nsteps, 1, flush, flags)
        a, b = mf.mf_phase_ms(mfab.h)
        fill_ms += a
        st_ms += b
    mf.mf_set_timing(mfab.h, 0)
    launches = mf.mf_launch_count(mfab.h)
    return st_ms * 1e-3 / (launches["stencil"] * steps), fill_ms / steps, launches


def fixed_line(mf, torch, flush, args, hbm):
    """The headline grid stored in FP64 and stepped as 64-bit fixed point, exact integer
    differences and an integer update (MF_FIXED_DIFF): FP64-accurate results (<= 1e-12 of the oracle, checked by
    the full-size tests) at memory speed.  Reports the step's fraction of the HBM roofline on
    the FP64 step bytes, the stencil kernel's own fraction, and the speedup over the plain
    per-box FP64 sweep (the untiled MFIter loop, FP64 arithmetic) and the batched FP64 one."""
    cfg = dict(synth.WORKLOADS[WORKLOAD])
    N, R, nsteps, C = cfg["N"], cfg["R"], cfg["nsteps"], cfg["ncomp"]
    lo, hi = [0, 0, 0], [N - 1] * 3
    D = [1.0] * C
    dt = synth.dt_for(cfg)
    V = N ** 3
    dense = synth.initial_field(cfg)
    FIX = mf.MF_FIXED_DIFF

    def level():
        m = mf.MultiFab(lo, hi, max_grid_size=cfg["max_grid_size"], ncomp=C, ngrow=cfg["ngrow"], dtype="f64")
        m.from_host(dense)
        return m

    g = level()
    for _ in range(2):
        mf.mf_advance(g.h, R, D, dt, nsteps, FIX)
    K = max(3, args.steps // 2)
    t = time_advances(g, R, D, dt, nsteps, K, flush, FIX)
    v = V * nsteps * K / (sum(t) * 1e-3)
    step_bytes = mf.mf_step_bytes(g.h, R)
    st_s, fill_ms, launches = stencil_phase(g, R, D, dt, nsteps, FIX, K, flush)
    b = cfg["max_grid_size"]
    nbox = (N // b) ** 3
    st_bytes = 8 * C * (2 * V + nbox * 6 * R * b * b)
    sched = mf.mf_get_schedule(g.h)
    del g
    torch.cuda.empty_cache()
    f64 = level()
    for _ in range(2):
        mf.mf_advance(f64.h, R, D, dt, nsteps)
    t64 = time_advances(f64, R, D, dt, nsteps, 2, flush)
    v64 = V * nsteps * 2 / (sum(t64) * 1e-3)
    del f64
    plain = level()
    mf.mf_advance(plain.h, R, D, dt, nsteps, mf.MF_PLAIN_PER_BOX)
    tp = time_advances(plain, R, D, dt, nsteps, 2, flush, mf.MF_PLAIN_PER_BOX)
    vplain = V * nsteps * 2 / (sum(tp) * 1e-3)
    del plain
    torch.cuda.empty_cache()
    return {"value": v, "unit": UNIT, "workload": WORKLOAD + ", FP64 storage, MF_FIXED_DIFF",
            "ms_per_bench_step": sum(t) / K, "step_bytes": step_bytes,
            "step_frac": step_bytes * nsteps * K / (sum(t) * 1e-3) / 1e9 / hbm,
            "kernel": {"name": "k_stencil_tma<f64,fixed,R=%d>" % R, "avg_launch_us": st_s * 1e6,
                       "algorithmic_bytes_per_launch": st_bytes, "achieved_gbs": st_bytes / st_s / 1e9,
                       "frac": st_bytes / st_s / 1e9 / hbm},
            "fill_phase_us_per_bench_step": fill_ms * 1e3,
            "launches_per_bench_step": launches, "schedule": sched,
            "fp64_batched_value": v64, "fp64_plain_per_box_value": vplain,
            "speedup_vs_fp64_plain_per_box": v / vplain, "speedup_vs_fp64_batched": v / v64}


def diff8th_line(mf, torch, flush, args, hbm):
    """The 8th-order workload (Sec. 4.2's 25-point operator on 5 components): periodic 512^3 in 64
    boxes of 128^3, 4 ghost cells, per-component diffusivities, 20 forward-Euler steps per bench
    step, FP32 and FP64 storage.  The initial field (8 seeded modes per component plus 1e-6
    noise) is evaluated on the device by the same generator as the host's (synth)."""
    cfg = dict(synth.WORKLOADS["c3"])
    if args.only == "diff8th512" and args.c3_n:
        cfg["N"] = args.c3_n
    N, R, C, n, mgs = cfg["N"], cfg["R"], cfg["ncomp"], cfg["nsteps"], cfg["max_grid_size"]
    D = [float(d) for d in synth.diffusivities(cfg)]
    dt = synth.dt_for(cfg)
    dense = synth.initial_field_device(cfg, "cuda", N=N).cpu().pin_memory()
    torch.cuda.empty_cache()
    V, nbox = N ** 3, (N // mgs) ** 3
    out = {"workload": "diff8th512_c5: periodic %d^3, %d boxes of 128^3, ngrow 4, 5 components, 25-point "
                       "8th-order stencil, D_c in [0.5, 2], %d forward-Euler steps per bench step"
                       % (N, (N // mgs) ** 3, n)}
    K = max(2, args.steps // 4)
    dtypes = args.c3_dtype.split(",") if args.only == "diff8th512" else ["f32", "f64"]
    for dtype, S in (("f32", 4), ("f64", 8)):
        if dtype not in dtypes:
            continue
        g = mf.MultiFab([0, 0, 0], [N - 1] * 3, max_grid_size=mgs, ncomp=C, ngrow=cfg["ngrow"], dtype=dtype)
        g.from_host(dense)
        if args.only == "diff8th512" and args.schedule:
            v = [int(x) for x in args.schedule.split(",")]
            g.set_tile(tuple(v[:3]))
            mf.mf_set_schedule(g.h, *v[3:6])
        g.advance(R, D, dt, n)  # autotune and capture
        t = time_advances(g, R, D, dt, n, K, flush)
        ms = sum(t) / len(t)
        step_bytes = g.step_bytes(R)
        st_s, fill_ms, _ = stencil_phase(g, R, D, dt, n, 0, 2, flush)
        out[dtype] = {"value": V * n / (ms * 1e-3), "unit": UNIT, "ms_per_bench_step": ms,
                      "cell_comp_updates_per_s": V * C * n / (ms * 1e-3), "step_bytes": step_bytes,
                      "step_frac": step_bytes * n / (ms * 1e-3) / 1e9 / hbm,
                      "stencil_launch_us": st_s * 1e6, "fill_phase_us_per_step": fill_ms * 1e3 / n,
                      "stencil_frac": S * C * (2 * V + nbox * 6 * R * mgs * mgs) / st_s / 1e9 / hbm,
                      "launches_per_bench_step": mf.mf_launch_count(g.h), "schedule": mf.mf_get_schedule(g.h)}
        del g
        torch.cuda.empty_cache()
    if "f32" in out and "f64" in out:
        out["speedup_f32_vs_f64"] = out["f32"]["value"] / out["f64"]["value"]
    return out


def manybox_step_bytes(S, C, boxes, R):
    """Compulsory bytes of one time step of a level: every valid cell read and written once,
    and the face halo of radius R read (the stencil's x halos come from the neighbour boxes and
    its y/z face ghosts are written by the producing tiles, so no ghost region is copied as
    such)."""
    ext = boxes[:, 3:] - boxes[:, :3] + 1
    V = int(ext.prod(axis=1).sum())
    face = int((2 * (ext[:, 0] * ext[:, 1] + ext[:, 1] * ext[:, 2] + ext[:, 0] * ext[:, 2])).sum())
    return S * C * (2 * V + R * face)


def manybox_line(mf, torch, flush, args, hbm):
    """512^3 with 2 components in 4096, 8192, 16384 and 32768 uneven boxes of 8^3-32^3, 2 ghost
    cells, the 13-point stencil, 50 time steps per bench step: the whole level in one launch per
    phase of a captured graph, whatever the box count.  FP32 at every box count, and FP64-accurate
    (fixed-point steps, MF_FIXED_DIFF) at the two ends; the field is evaluated on the device by
    the seeded generator."""
    cfg = synth.WORKLOADS["c5"]
    N, R, C, n = cfg["N"], cfg["R"], cfg["ncomp"], cfg["nsteps"]
    dense = synth.initial_field_device(cfg, "cuda").cpu().pin_memory()
    torch.cuda.empty_cache()
    dt = synth.dt_for(cfg)
    out = {}
    # (boxes, storage, flags, regions of at most this many cells per side or 0 for one FArrayBox
    # per box)
    runs = ([(t, "f32", 0, 0) for t in cfg["targets"]] + [(t, "f64fixed", mf.MF_FIXED_DIFF, 0) for t in (4096, 32768)]
            + [(t, "f32", 0, 128) for t in (4096, 32768)] + [(32768, "f64fixed", mf.MF_FIXED_DIFF, 128)])
    if args.only == "manybox512" and args.c5:
        v = args.c5.split(",")
        runs = [r for r in runs if r[0] == int(v[0]) and r[1] == v[1] and r[3] == (int(v[2]) if len(v) > 2 else 0)]
    for target, dtype, flags, max_region in runs:
        boxes = synth.uneven_boxes(N, target)
        g = mf.MultiFab([0, 0, 0], [N - 1] * 3, boxes=boxes, ncomp=C, ngrow=cfg["ngrow"],
                        dtype="f64" if flags else dtype, max_region=max_region or None)
        g.from_host(dense)
        if args.only == "manybox512" and args.c5 and args.schedule:
            v = [int(x) for x in args.schedule.split(",")]
            g.set_tile(tuple(v[:3]))
            mf.mf_set_schedule(g.h, *v[3:6])
        for _ in range(max(1, args.warmup)):
            g.advance(R, [1.0] * C, dt, n, flags)
        K = max(2, args.steps // 2)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            flush()
            ev[k][0].record(g.stream)
            g.advance(R, [1.0] * C, dt, n, flags)
            ev[k][1].record(g.stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / K
        # compulsory bytes of the storage: the regions' faces for a regional level
        step_bytes = manybox_step_bytes(8 if flags else 4, C, g.regions, R)
        key = "%d_%s%s" % (target, dtype, "_regional" if max_region else "")
        out[key] = {
            "value": N ** 3 * n / (ms * 1e-3), "unit": UNIT, "ms_per_bench_step": ms,
            "cell_comp_updates_per_s": N ** 3 * C * n / (ms * 1e-3), "boxes": target, "dtype": dtype,
            "regions": mf.mf_nregions(g.h), "step_bytes": step_bytes,
            "step_frac": step_bytes * n / (ms * 1e-3) / 1e9 / hbm,
            "launches_per_bench_step": mf.mf_launch_count(g.h), "schedule": mf.mf_get_schedule(g.h)}
        del g
        torch.cuda.empty_cache()
    out["workload"] = ("manybox512_c2: periodic 512^3, 2 components, 4096-32768 uneven boxes of 8^3-32^3, "
                       "ngrow 2, 13-point stencil, FP32 and FP64-accurate fixed-point steps, %d steps per bench "
                       "step; *_regional: the same boxes stored in regions of at most 128^3 (mf_create_regional)"
                       % n)
    return out


def bf16_line(mf, torch, flush, args, hbm):
    """The headline grid (256^3 in 64 boxes of 64^3, 7-point, 100 steps per bench step) stored in
    BF16 with FP32 arithmetic: throughput, compulsory bytes per step (valid cells read and
    written, face halo read) and their fraction of the measured peak."""
    cfg = synth.WORKLOADS["c2"]
    N, R, n, mgs = cfg["N"], cfg["R"], cfg["nsteps"], cfg["max_grid_size"]
    dt = synth.dt_for(cfg)
    g = mf.MultiFab([0, 0, 0], [N - 1] * 3, max_grid_size=mgs, ncomp=1, ngrow=cfg["ngrow"], dtype="bf16")
    g.from_host(synth.initial_field(cfg))
    for _ in range(max(1, args.warmup)):
        g.advance(R, [1.0], dt, n)
    t = time_advances(g, R, [1.0], dt, n, args.steps, flush)
    ms = sum(t) / len(t)
    step_bytes = 2 * (2 * N ** 3 + (N // mgs) ** 3 * 6 * R * mgs * mgs)
    return {"value": N ** 3 * n / (ms * 1e-3), "unit": UNIT, "ms_per_bench_step": ms, "step_bytes": step_bytes,
            "step_frac": step_bytes * n / (ms * 1e-3) / 1e9 / hbm, "schedule": mf.mf_get_schedule(g.h),
            "workload": "heat256_64x64 in BF16 storage (FP32 arithmetic), %d steps per bench step" % n}


def rk3_line(mf, torch, flush, args, hbm):
    """The third-order Runge-Kutta advance with the 25-point 8th-order stencil (Sec. 4.2's
    integrator and operator): 256^3 in 64 boxes of 64^3, 4 ghost cells, FP32, 20 steps of 3
    stencil launches per bench step."""
    c = RK3_CFG
    N, R, n = c["N"], c["R"], c["nsteps"]
    dense = synth.eval_modes((N, N, N), synth.sine_modes(synth.FIELD_SEED, 300, c["nmodes"], c["kmax"]))[None]
    m = mf.MultiFab([0, 0, 0], [N - 1] * 3, max_grid_size=c["max_grid_size"], ncomp=1, ngrow=c["ngrow"],
                    dtype=c["dtype"])
    m.from_host(dense)
    if args.only and args.schedule:
        v = [int(x) for x in args.schedule.split(",")]
        m.set_tile(tuple(v[:3]))
        mf.mf_set_schedule(m.h, *v[3:6])
    dt = synth.heat_dt(N, R)
    for _ in range(2):
        m.rk3_advance(R, [1.0], dt, n)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush()
        ev[k][0].record(m.stream)
        mf.mf_rk3_advance(m.h, R, [1.0], dt, n)
        ev[k][1].record(m.stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    V, nbox, b, S = N ** 3, (N // c["max_grid_size"]) ** 3, c["max_grid_size"], 4
    # per step: 3 stencil launches (read V + face halo, write V) and 2 reads of u0
    step_bytes = S * (3 * (2 * V + nbox * 6 * R * b * b) + 2 * V)
    launches = mf.mf_launch_count(m.h)
    return {"value": V * n / (ms * 1e-3), "unit": "cell-updates/s (RK3 steps)", "ms_per_bench_step": ms,
            "workload": "rk3_8th256: periodic 256^3, 64 boxes of 64^3, ngrow 4, 25-point 8th-order stencil, "
                        "3-stage SSP Runge-Kutta, FP32, %d steps per bench step" % n,
            "step_bytes": step_bytes, "step_frac": step_bytes * n / (ms * 1e-3) / 1e9 / hbm,
            "stencil_launches_per_bench_step": launches["stencil"], "fill_launches_per_bench_step": launches["fill"],
            "schedule": mf.mf_get_schedule(m.h)}


def amr_step_bytes(S, Nc, mgs, fboxes, r, nsub, g_interp):
    """Algorithmic bytes of one coarse step of the two-level advance: each level's stencil reads
    and writes its valid cells once and reads its face halo (radius 1), the fine level nsub
    times; each interpolation writes its ghost cells and reads the coarse cells under them at
    two time levels (1/r^3 as many); the average-down reads every fine cell and writes one
    coarse cell per r^3."""
    ext = fboxes[:, 3:] - fboxes[:, :3] + 1
    Vf = int(ext.prod(axis=1).sum())
    face_f = int((2 * (ext[:, 0] * ext[:, 1] + ext[:, 1] * ext[:, 2] + ext[:, 0] * ext[:, 2])).sum())
    nb = (Nc // mgs) ** 3
    coarse = 2 * Nc ** 3 + nb * 6 * mgs * mgs
    fine = nsub * (2 * Vf + face_f)
    interp = nsub * (g_interp + 2 * g_interp / r ** 3)
    avg = Vf + Vf / r ** 3
    return S * (coarse + fine + interp + avg)


def amr_line(mf, torch, flush, args, hbm):
    """The two-level workload with refluxing: coarse 256^3 in 64 boxes of 64^3, a fine level at
    ratio 2 on the seeded sphere boxes, 2 fine substeps per coarse step, FP32, 50 coarse steps
    per bench step; cells counted once per coarse step on the coarse level and once per
    substep on the fine level."""
    cfg = synth.WORKLOADS["c4"]
    Nc, r, nsub, n = cfg["N"], cfg["ratio"], cfg["nsub"], cfg["nsteps"]
    fboxes = synth.sphere_fine_boxes(Nc, ratio=r)
    modes = synth.sine_modes(synth.FIELD_SEED, 100, cfg["nmodes"], cfg["kmax"])
    lo = fboxes[:, :3].min(axis=0)
    hi = fboxes[:, 3:].max(axis=0)
    fden = np.zeros((1, r * Nc, r * Nc, r * Nc))
    fden[0, lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = synth.eval_modes_box(
        r * Nc, lo, tuple(int(v) for v in (hi - lo + 1)[::-1]), modes)
    gc = mf.MultiFab([0, 0, 0], [Nc - 1] * 3, max_grid_size=cfg["max_grid_size"], ngrow=1, dtype="f32")
    gf = mf.MultiFab([0, 0, 0], [r * Nc - 1] * 3, boxes=fboxes, ngrow=1, dtype="f32")
    gc.from_host(synth.initial_field(cfg))
    gf.from_host(fden)
    mf.mf_average_down(gf.h, gc.h, r)
    dt = synth.dt_for(cfg)
    for _ in range(2):
        mf.mf_amr_advance(gc.h, gf.h, 1, [1.0], dt, n, nsub, r, mf.MF_REFLUX)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush()
        ev[k][0].record(gc.stream)
        mf.mf_amr_advance(gc.h, gf.h, 1, [1.0], dt, n, nsub, r, mf.MF_REFLUX)
        ev[k][1].record(gc.stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    Vc = Nc ** 3
    ext = fboxes[:, 3:] - fboxes[:, :3] + 1
    Vf = int(ext.prod(axis=1).sum())
    g_interp = mf.mf_interp_cells(gf.h, gc.h, r)[0]  # interpolated fine ghost cells per substep
    step_bytes = amr_step_bytes(4, Nc, cfg["max_grid_size"], fboxes, r, nsub, g_interp)
    return {"value": (Vc + nsub * Vf) * n / (ms * 1e-3), "unit": "cell-updates/s (coarse per step + fine per substep)",
            "ms_per_bench_step": ms, "interp_ghost_cells": g_interp,
            "step_bytes": step_bytes, "step_frac": step_bytes * n / (ms * 1e-3) / 1e9 / hbm,
            "schedule": {"coarse": mf.mf_get_schedule(gc.h), "fine": mf.mf_get_schedule(gf.h)},
            "workload": "amr2lev256_sphere: coarse 256^3 (64 boxes of 64^3) + %d fine boxes (%d cells) at ratio 2, "
                        "2 substeps, refluxing, FP32, %d coarse steps per bench step" % (len(fboxes), Vf, n),
            "launches_per_bench_step": mf.mf_launch_count(gc.h),
            "launches_per_coarse_step": sum(mf.mf_launch_count(gc.h).values()) / n}


def run_ours(args, cfg, ws, rank, local):
    import torch
    import paper_1604_03570_gb300 as mf

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    N, R, nsteps = cfg["N"], cfg["R"], cfg["nsteps"]
    lo, hi = [0, 0, 0], [N - 1] * 3
    D = [1.0] * cfg["ncomp"]
    dt = synth.dt_for(cfg)
    V = N ** 3
    dense = synth.initial_field(cfg)
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    flush_rd = torch.ones(512 << 20, dtype=torch.uint8, device=dev)

    def flush():
        # write a buffer four times the L2, then read another: the timed region starts with no
        # line of its own data in L2 and no dirty line of the flush left to write back
        flush_buf.fill_(1)
        flush_rd.max()

    def level(dtype):
        m = mf.MultiFab(lo, hi, max_grid_size=cfg["max_grid_size"], ncomp=cfg["ncomp"], ngrow=cfg["ngrow"],
                        dtype=dtype)
        m.from_host(dense)
        return m

    # ---- headline: batched, graph-captured sweep
    head = level(args.dtype)
    if args.tile:
        head.set_tile(tuple(int(v) for v in args.tile.split(",")))
    if args.schedule:
        v = [int(x) for x in args.schedule.split(",")]
        head.set_tile(tuple(v[:3]))
        mf.mf_set_schedule(head.h, *v[3:6])
    mf.mf_set_kernel(head.h, mf.MF_KERNEL_TMA if args.kernel == "tma" else mf.MF_KERNEL_GLOBAL)
    hflags = mf.MF_FIXED_DIFF if args.fixed else mf.MF_PLAIN_PER_BOX if args.plain else 0
    for _ in range(args.warmup):
        mf.mf_advance(head.h, R, D, dt, nsteps, hflags)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = time_advances(head, R, D, dt, nsteps, args.steps, flush, hflags)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(times), dist, dev)
    if dist:
        dist.barrier()
    value = whole_job_rate(ws, V * nsteps * args.steps, total_ms * 1e-3)
    tile, _ = mf.mf_get_tile(head.h)

    launches = mf.mf_launch_count(head.h)  # of one mf_advance (the graph replayed every bench step)
    sched = mf.mf_get_schedule(head.h)
    kname = "k_stencil_tma" if sched["kernel"] == "tma" else "k_stencil"
    kvar = "%s,fixed" % args.dtype if args.fixed else args.dtype

    # ---- roofline of the dominant kernel (stencil): events inside the graph wherever the kind
    # of launch changes, so the back-to-back stencil launches are timed without nodes between
    fill_ms, st_ms = 0.0, 0.0
    t_timed = []
    if args.plain:  # eager per-box launches: no graph events; the whole step stands in for the stencil
        t_timed = list(times)
        st_ms = sum(times)
    else:
        mf.mf_set_timing(head.h, 1)
        for _ in range(2):
            mf.mf_advance(head.h, R, D, dt, nsteps, hflags)
        for _ in range(args.steps):
            t_timed += time_advances(head, R, D, dt, nsteps, 1, flush, hflags)
            a, b = mf.mf_phase_ms(head.h)
            fill_ms += a
            st_ms += b
        mf.mf_set_timing(head.h, 0)
    st_avg_s = st_ms * 1e-3 / (max(1, launches["stencil"]) * args.steps)
    if args.plain:
        st_avg_s = st_ms * 1e-3 / (nsteps * args.steps)  # one time step of all per-box launches
    S = {"f64": 8, "f32": 4, "bf16": 2}[args.dtype]
    nbox = (N // cfg["max_grid_size"]) ** 3
    b = cfg["max_grid_size"]
    G = mf.mf_fb_regions(head.h)[1]
    C = cfg["ncomp"]
    # compulsory bytes of one stencil launch: every valid cell read and written once, plus the
    # face halo of radius R of every box (the ghost push into neighbouring boxes is not counted)
    st_bytes = S * C * (2 * V + nbox * 6 * R * b * b)
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    achieved = st_bytes / st_avg_s / 1e9
    step_bytes = mf.mf_step_bytes(head.h, R)
    roof = {"bound": "hbm", "kernel": "%s<%s,R=%d>" % (kname, kvar, R), "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind + " (STREAM-style copy)",
            "traffic": traffic_for(kname, WORKLOAD, kvar),
            "algorithmic_bytes_per_launch": st_bytes, "avg_launch_us": st_avg_s * 1e6,
            "stencil_launches_per_bench_step": launches["stencil"],
            "fill_launches_per_bench_step": launches["fill"],
            "fill_phase_us_per_bench_step": fill_ms * 1e3 / args.steps,
            "step_bytes": step_bytes,
            "step_frac": step_bytes * nsteps * args.steps / (total_ms * 1e-3) / 1e9 / hbm,
            "step_frac_of_8tbs": step_bytes * nsteps * args.steps / (total_ms * 1e-3) / 1e9 / 8000.0,
            "timed_with_events_ms_per_step": sum(t_timed) / len(t_timed)}

    # ---- the full FillBoundary kernel alone (every ghost cell, edges and corners included)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(3):
        mf.mf_fill_boundary(head.h)
    fb_us = []
    for _ in range(args.steps):
        flush()
        ev[0].record(head.stream)
        mf.mf_fill_boundary(head.h)
        ev[1].record(head.stream)
        torch.cuda.synchronize()
        fb_us.append(ev[0].elapsed_time(ev[1]) * 1e3)
    fb_bytes = 2 * S * C * G
    fb_avg = statistics.median(fb_us)
    roof["fill_kernel"] = {"kernel": "k_fill<%s>" % args.dtype, "achieved": fb_bytes / fb_avg / 1e3, "unit": "GB/s",
                           "frac": fb_bytes / fb_avg / 1e3 / hbm, "algorithmic_bytes_per_launch": fb_bytes,
                           "avg_launch_us": fb_avg, "ghost_cells": G}
    # ---- the compensated domain sum: mf_sum synchronises, so this is the host-visible call
    # latency (kernels, the 8-byte read-back and the wake-up of the calling thread)
    for _ in range(2):
        mf.mf_sum(head.h, 0)
    sm_us = []
    for _ in range(args.steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mf.mf_sum(head.h, 0)
        sm_us.append((time.perf_counter() - t0) * 1e6)
    sm_avg = statistics.median(sm_us)
    roof["sum_call"] = {"kernels": "k_reduce_partial<sum>+k_reduce_final", "achieved": S * V / sm_avg / 1e3,
                        "unit": "GB/s", "frac": S * V / sm_avg / 1e3 / hbm, "algorithmic_bytes_per_call": S * V,
                        "median_call_us": sm_avg}
    mx_us = []
    for _ in range(args.steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mf.mf_reduce(head.h, 0, "max")
        mx_us.append((time.perf_counter() - t0) * 1e6)
    mx_avg = statistics.median(mx_us)
    roof["max_call"] = {"kernels": "k_reduce_partial<max>+k_reduce_final", "achieved": S * V / mx_avg / 1e3,
                        "unit": "GB/s", "frac": S * V / mx_avg / 1e3 / hbm, "algorithmic_bytes_per_call": S * V,
                        "median_call_us": mx_avg}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
           "config": workload_config(cfg), "roofline": roof,
           "gpu_launches": (launches["fill"] + launches["stencil"]) * args.steps,
           "tile": list(tile), "schedule": sched}
    out["clocks"] = clk.summary()

    if not args.no_extras:
        # ---- e2e through the public API with pinned host buffers
        pin_in = torch.from_numpy(dense).pin_memory()
        pin_out = torch.empty(dense.shape, dtype=torch.float64).pin_memory()
        e2e_t = []
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mf.mf_copy_from_host(head.h, pin_in)
            mf.mf_advance(head.h, R, D, dt, nsteps, hflags)
            mf.mf_copy_to_host(head.h, pin_out)
            t1 = time.perf_counter()
            if k >= args.warmup:
                e2e_t.append(t1 - t0)
        e2e_s = max_over_ranks(sum(e2e_t), dist, dev)
        out["e2e"] = {"value": whole_job_rate(ws, V * nsteps * args.steps, e2e_s), "unit": UNIT,
                      "h2d_bytes_per_step": int(dense.nbytes), "d2h_bytes_per_step": int(dense.nbytes)}
        del head
        # ---- FP64 batched and FP64 plain per box
        k2 = max(2, args.steps // 2)
        f64 = level("f64")
        for _ in range(2):
            mf.mf_advance(f64.h, R, D, dt, nsteps)
        t64 = time_advances(f64, R, D, dt, nsteps, k2, flush)
        v64 = V * nsteps * k2 / (sum(t64) * 1e-3)
        tile64, _ = mf.mf_get_tile(f64.h)
        del f64
        plain = level("f64")
        mf.mf_advance(plain.h, R, D, dt, nsteps, mf.MF_PLAIN_PER_BOX)
        tp = time_advances(plain, R, D, dt, nsteps, 2, flush, mf.MF_PLAIN_PER_BOX)
        vplain = V * nsteps * 2 / (sum(tp) * 1e-3)
        del plain
        dpk = fp64_peak_tflops()
        flops = FLOPS_PER_CELL[R] * V * nsteps * k2 / (sum(t64) * 1e-3) / 1e12
        out["fp64_batched"] = {"value": v64, "unit": UNIT, "tile": list(tile64),
                               "frac_of_hbm": 8 * C * (2 * V + 2 * G + nbox * 6 * b * b) * nsteps * k2
                               / (sum(t64) * 1e-3) / 1e9 / hbm,
                               "roofline": {"bound": "alu", "achieved": flops, "peak": dpk, "unit": "TFLOP/s",
                                            "frac": flops / dpk if dpk else None,
                                            "peak_kind": "measured: mf_fp64_fma_rate (DFMA chains, best of 3)",
                                            "flops_per_cell": FLOPS_PER_CELL[R]}}
        out["fp64_plain_per_box"] = {"value": vplain, "unit": UNIT,
                                     "launches_per_time_step": 2 * nbox}
        # secondary lines, on one GPU only (the scaling runs compare the headline); a failure is
        # reported in its own entry and does not void the headline
        secondary = (("fp64_fixed", fixed_line), ("bf16_batched", bf16_line), ("rk3_8th", rk3_line),
                     ("diff8th512", diff8th_line), ("amr2lev_reflux", amr_line), ("manybox512", manybox_line))
        for key, line in (secondary if ws == 1 else ()):
            try:
                out[key] = line(mf, torch, flush, args, hbm)
            except Exception as e:  # noqa: BLE001
                out[key] = {"error": "%s: %s" % (type(e).__name__, e)}
                torch.cuda.synchronize()
        out["speedup_batched_vs_fp64_plain_per_box"] = value / vplain
        if rank == 0 and ws == 1:
            out["cpu_baseline"] = cpu_baseline(cfg)
    elif "e2e" not in out:
        out["e2e"] = None
    if dist:
        dist.destroy_process_group()
    return out if rank == 0 else None


def main():
    args = parse()
    ws, rank, local = dist_env()
    cfg = dict(synth.WORKLOADS[WORKLOAD])
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, cfg)))
        return 0
    if args.only:
        import torch
        import paper_1604_03570_gb300 as mf
        torch.cuda.set_device(local)
        flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        flush_rd = torch.ones(512 << 20, dtype=torch.uint8, device="cuda")

        def flush():
            flush_buf.fill_(1)
            flush_rd.max()

        peaks, _ = measured_peaks()
        hbm = float(peaks["hbm_gbs"])
        line = {"bf16_batched": bf16_line, "rk3_8th": rk3_line, "amr2lev_reflux": amr_line,
                "manybox512": manybox_line, "fp64_fixed": fixed_line, "diff8th512": diff8th_line}[args.only](
            mf, torch, flush, args, hbm)
        print(json.dumps({args.only: line}))
        return 0
    out = run_ours(args, cfg, ws, rank, local)
    if out is not None:
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
