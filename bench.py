"""Benchmark of the GKE Parseval path on GB300.

One step = one whole pass of the hot path over one batch of snapshots:
Step-1 ensemble mean, fluctuations and in-plane products, per-wavenumber
contractions over snapshots, inverse transforms to separation space and the
Step-3 stencils, i.e. every GKE term for every (Y1 <= Y2) pair and every
separation.  Throughput is counted in pair-snapshots per second:
(number of pairs Y1 <= Y2) x (snapshots in the batch) / step time.

Default workload: the Re_tau~200-shaped synthetic channel (nx = nz = 256,
ny = 129 Chebyshev points, 16 snapshots), plain FP64 path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f64|bf16x3]
                    [--workload NAME] [--impl ours|reference]

--impl reference times the CPU oracle (direct averages, C/OpenMP) on the host
cores on a bounded sample of the same workload.

--step1 times Step 1 for velocity-vorticity databases (u, w from v and the
wall-normal vorticity, Poisson pressure) on the workload's snapshots and prints
its own JSON line (snapshots/s).

--passes P runs P untimed passes of the workload at --precision and prints the
number of kernel launches per pass, nothing else: the program that ncu launch
lists and single-kernel captures are taken on.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "GKE (y,y')-pair correlations/s & tensor-pipe %, split-BF16 vs FP64 at 1e-6 rel err"
UNIT = "pair-snapshots/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA rate: the nominal 1.25 TFLOP/s of GB300 over 152 SMs at the 2070 MHz
# maximum clock is 3.97 flop/clk/SM, i.e. 2 DFMA per clock per SM.
FP64_FLOP_PER_CLK_SM = 4.0
FP32_FLOP_PER_CLK_SM = 256.0
N_SM = 152


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def correlator_cmac(wl, ns):
    """Complex multiply-adds of the per-wavenumber contractions of one pass.

    D (Hermitian, pairs y <= y'): K = 3 ns; square jobs over all ordered
    pairs: E, F, QV (K = ns), X (3 ns), Gx, Gz (4 ns each)."""
    Nk = wl.nz * wl.nxh
    return Nk * ns * (3 * wl.npair + 14 * wl.ny * wl.ny)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per pass of each
# stage's kernels at 256 x 256 x 129 x 16 (GB): ncu captures of the small
# cases profile_256x256x17_s16 and profile_32x32x129_s16, scaled by pairs,
# wall-normal planes or wavenumbers to the full size
# (profiles/dram_small_cases_split_and_f64.md); a stage missing here reports
# null (not captured since its kernels changed).
NCU_TRAFFIC_GB = {
    "f64": {"correlate": 96.7, "combine": 93.0, "terms": 104.0, "stencil": 38.0, "products": 27.8},
    "bf16x3": {"correlate": 36.6, "terms": 55.9, "stencil": 20.5, "products": 16.4},
}


def ncu_traffic(wl, precision, stage):
    """Captured DRAM bytes of a stage (only for the workload the capture ran)."""
    if wl.name != S.RETAU200.name:
        return None
    gb = NCU_TRAFFIC_GB.get(precision, {}).get(stage)
    return None if gb is None else int(gb * 1e9)


def stage_rooflines(wl, ns, precision, stage_ms, pk, pk_kind):
    """Algorithmic work of each stage of one pass, and its roofline.

    Bytes count each stage's essential inputs read once and outputs written
    once (workspaces between kernels of a stage are not counted); the
    contraction stage counts flops (tensor BF16 on the split path, FP64 DFMA
    on the plain path)."""
    f32 = precision != "f64"
    cz = 8 if f32 else 16                          # bytes of one complex operand / spectrum value
    tz = 4 if f32 else 8                           # bytes of one term value
    Nk, ny, N = wl.nz * wl.nxh, wl.ny, wl.nx * wl.nz
    yb = (ny + 7) // 8
    raw = 7 * yb * yb * 64 * Nk * cz
    comb = wl.npair * 7 * Nk * cz
    terms = 7 * wl.npair * N * tz
    spec_arr = wl.npair * N * 4
    # split-BF16 plans with one 128-row tile write six plane spectra per
    # (wavenumber, pair) from the tensor-core epilogue: no raw contractions,
    # no combine stage; the transforms read the planes
    planes = precision == "bf16x3" and (ny <= 128 or ny == 129)
    pl_bytes = 6 * Nk * (4 * ((wl.npair + 3) // 4)) * cz
    # FP32 paths: the row pass writes five terms and the spectral parts of A,
    # Phi_y, phi; the first stencil pass reads those three parts, writes Phi_y
    # and phi and updates two parts, the second reads the two and updates the
    # residual (11 values per pair and separation)
    hbm = {
        "products": ns * 4 * ny * Nk * 16 + 11 * Nk * ns * ny * cz,
        "terms": (pl_bytes if planes else comb) + (5 * terms // 7 + 3 * spec_arr if f32 else terms),
        "stencil": (11 * spec_arr) if f32 else (9 * wl.npair * N * 8),
    }
    if not planes:
        hbm["combine"] = raw + comb
    peak_bw = pk["hbm_gbs"]
    out = {}
    for st, b in hbm.items():
        if st.endswith("_bytes") or st not in stage_ms or stage_ms[st] <= 0:
            continue
        ach = b / (stage_ms[st] / 1e3) / 1e9
        out[st] = {"bound": "hbm", "achieved": ach, "peak": peak_bw, "unit": "GB/s", "frac": ach / peak_bw,
                   "bytes": b, "launch_ms": stage_ms[st], "traffic": ncu_traffic(wl, precision, st),
                   "peak_source": f"hbm_gbs ({pk_kind})"}
    cm = correlator_cmac(wl, ns)
    ms = stage_ms.get("correlate", 0.0)
    if ms > 0:
        if precision == "f32":
            flops = 8.0 * cm
            peak = N_SM * FP32_FLOP_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            out["correlate"] = {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak,
                                "unit": "TFLOP/s", "flops": flops, "launch_ms": ms,
                                "traffic": ncu_traffic(wl, precision, "correlate"),
                                "peak_source": "derived: 152 SM x 128 FFMA/clk x 2 flop x max SM clock"}
        elif f32:
            flops = 48.0 * cm                      # 6 BF16 slice products x 8 real flops per complex MAC
            peak = pk["bf16_tflops"]
            out["correlate"] = {"bound": "tensor", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak,
                                "unit": "TFLOP/s", "flops": flops, "launch_ms": ms,
                                "traffic": ncu_traffic(wl, precision, "correlate"),
                                "peak_source": f"bf16_tflops ({pk_kind})",
                                "note": "stage = operand split + tcgen05 contractions + edge row"}
        else:
            flops = 8.0 * cm
            peak = N_SM * FP64_FLOP_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            out["correlate"] = {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak,
                                "unit": "TFLOP/s", "flops": flops, "launch_ms": ms,
                                "traffic": ncu_traffic(wl, precision, "correlate"),
                                "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x max SM clock "
                                               "(nominal 1.25 TFLOP/s FP64)"}
        out["correlate"]["frac"] = out["correlate"]["achieved"] / out["correlate"]["peak"]
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r[1:]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------- CPU oracle
def oracle_sample(wl, phys, npts, nplanes, seed=0):
    """Time the oracle on npts sampled (pair, separation) points of the workload.

    Returns (pair-snapshots/s extrapolated from points to whole pairs, seconds,
    description)."""
    import oracle
    rng = np.random.default_rng(seed)
    planes = sorted(rng.choice(wl.ny, size=nplanes, replace=False).tolist())
    pts = []
    for _ in range(npts):
        a, b = sorted(rng.choice(planes, 2))
        pts.append((a, b, int(rng.integers(wl.nz)), int(rng.integers(wl.nx))))
    t0 = time.perf_counter()
    oracle.points(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu, pts)
    dt = time.perf_counter() - t0
    pair_equiv = npts / float(wl.nx * wl.nz)
    rate = pair_equiv * wl.nsnap / dt
    desc = (f"{npts} (pair, separation) points on {nplanes} wall-normal planes of {wl.name}, "
            f"all terms but the residual; rate = points/(nx nz) x snapshots / time")
    return rate, dt, desc


def run_reference(args, world, rank):
    if rank != 0:
        return
    wl = S.WORKLOADS[args.workload]
    phys = S.physical(wl)
    import oracle
    oracle.build()
    cores = os.cpu_count()
    npts, nplanes = args.ref_points, 2
    for _ in range(args.warmup):
        oracle_sample(wl, phys, max(8, npts // 8), nplanes, seed=99)
    times, rates = [], []
    for k in range(args.steps):
        r, dt, desc = oracle_sample(wl, phys, npts, nplanes, seed=k)
        times.append(dt)
        rates.append(r)
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(wl, args.precision),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(wl, precision):
    return {"workload": wl.name, "nx": wl.nx, "nz": wl.nz, "ny": wl.ny, "snapshots": wl.nsnap,
            "pairs": wl.npair, "precision": precision, "Lx": round(wl.Lx, 6), "Lz": round(wl.Lz, 6),
            "nu": wl.nu, "l2": "inputs and accumulators larger than L2 (no flush)"}


# ------------------------------------------------------- input generation
def _gen_snapshot(job):
    """Worker: coefficients of snapshot s written into the shared array."""
    from multiprocessing import shared_memory
    name, s, shm_name, shape = job
    wl = S.WORKLOADS[name]
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        arr = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
        arr[s] = S.snapshot_coefficients(wl, s)
    finally:
        shm.close()
    return s


def coefficients_parallel(wl, dev):
    """The workload's coefficients, generated snapshot by snapshot in spawned
    worker processes (large grids), copied to the device `dev`."""
    import torch
    from multiprocessing import get_context, shared_memory
    shape = (wl.nsnap, 4, wl.ny, wl.nz, wl.nxh)
    nbytes = int(np.prod(shape)) * 16
    shm = shared_memory.SharedMemory(create=True, size=nbytes)
    try:
        with get_context("spawn").Pool(min(16, os.cpu_count() or 1, wl.nsnap)) as pool:
            pool.map(_gen_snapshot, [(wl.name, s, shm.name, shape) for s in range(wl.nsnap)])
        arr = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
        out = torch.empty(shape, dtype=torch.complex128, device=dev)
        for s in range(wl.nsnap):
            out[s].copy_(torch.from_numpy(arr[s]))
        del arr
        return out
    finally:
        shm.close()
        shm.unlink()


# ------------------------------------------------------------------ ours
def run_stream(args, world, rank, local):
    """Streaming mode: the snapshots accumulated args.batch at a time, optional
    mirror sampling on the wedge and uniform undersampling by args.stride (the
    memory-bounded mode of large grids)."""
    import torch
    import paper_1910_06409_gb300._native as N

    torch.cuda.set_device(local)
    wl = S.WORKLOADS[args.workload]
    if args.nsnap:
        wl = S.Workload(wl.name, wl.wid, wl.nx, wl.nz, wl.ny, args.nsnap, wl.Lx, wl.Lz, wl.nu)
    ns = wl.nsnap
    B = args.batch or ns
    prec = {"f64": N.GKE_PREC_F64, "bf16x3": N.GKE_PREC_BF16X3, "f32": N.GKE_PREC_F32}[args.precision]
    dom = N.GKE_DOMAIN_WEDGE if args.pair_domain == "wedge" else N.GKE_DOMAIN_TRIANGLE
    st_opt = (0, 0, 0, args.stride) if args.stride > 1 else (0, 0, 0, 0)
    f_dev = coefficients_parallel(wl, "cuda")
    stream = torch.cuda.current_stream()
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), B, prec,
                      stream=stream.cuda_stream, pair_domain=dom, under_x=st_opt, under_z=st_opt)
    npair = N.gke_npair(plan)
    mz, mx = N.gke_separation_labels(plan)
    tdt = torch.float64 if args.precision == "f64" else torch.float32
    terms = torch.empty((N.GKE_NTERM, npair, len(mz), len(mx)), dtype=tdt, device="cuda")

    def step(pl=plan, out=terms):
        N.gke_reset(pl)
        for b in range(0, ns, B):
            N.gke_accumulate_mean(pl, f_dev[b:b + B], min(B, ns - b))
        for b in range(0, ns, B):
            N.gke_accumulate_snapshot(pl, f_dev[b:b + B], min(B, ns - b))
        N.gke_finalize_terms(pl, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    N.gke_set_timing(plan, True)
    N.gke_stage_times(plan)
    l0 = N.gke_launch_count(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    launches = N.gke_launch_count(plan) - l0
    stage_ms = {k: v / args.steps for k, v in N.gke_stage_times(plan).items()}
    N.gke_destroy(plan)
    ms = e0.elapsed_time(e1) / args.steps
    # accuracy of a reduced-precision run: the same snapshots through an FP64
    # plan with the same options (untimed), per-term max |x - f64| / max |f64|
    err = None
    if args.precision != "f64" and not args.no_f64_check:
        plan64 = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), B, N.GKE_PREC_F64,
                            stream=stream.cuda_stream, pair_domain=dom, under_x=st_opt, under_z=st_opt)
        terms64 = torch.empty(terms.shape, dtype=torch.float64, device="cuda")
        step(plan64, terms64)
        torch.cuda.synchronize()
        N.gke_destroy(plan64)
        err = {}
        for t, name in enumerate(TERM_NAMES):
            scale = float(terms64[t].abs().max())
            diff = float((terms[t].double() - terms64[t]).abs().max())
            err[name] = float("%.3g" % (diff / scale if scale > 0 else diff))
        del terms64
    pk, pk_kind = peaks()
    rl = stage_rooflines(wl, ns, args.precision, {"correlate": stage_ms.get("correlate", 0.0)}, pk, pk_kind)
    cfg = config_of(wl, args.precision)
    cfg.update({"pair_domain": args.pair_domain, "stride": args.stride, "batch": B, "output_pairs": npair,
                "separations": [int(len(mz)), int(len(mx))]})
    line = {"metric": METRIC, "value": npair * ns / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"f64": "f64", "bf16x3": "bf16x3/f32", "f32": "f32"}[args.precision],
            "data": "synthetic", "config": cfg,
            "max_rel_err_vs_f64": err, "tolerance": 1e-6 if err is not None else None,
            "within_tolerance": None if err is None else all(e <= 1e-6 for e in err.values()),
            "stage_ms": stage_ms, "gpu_launches": launches,
            "clocks": clk.summary(), "e2e": None, "roofline": rl.get("correlate"), "cpu_baseline": None,
            "note": "streaming mode: outputs are output_pairs x separations; value counts output pairs"}
    if rank == 0:
        print(json.dumps(line), flush=True)


GROUP = (("group_128x128x65_s32", 1), ("group_256x256x129_s16", 1), ("group_384x384x193_s8", 2))


def run_group(args, world, rank, local):
    """The three channel-shaped datasets of the grouped configuration, each
    with its own plan, back to back on one stream; the 384 x 384 x 193 one at
    separation stride 2 (its full-resolution triangle needs ~282 GB)."""
    import torch
    import paper_1910_06409_gb300._native as N

    torch.cuda.set_device(local)
    prec = {"f64": N.GKE_PREC_F64, "bf16x3": N.GKE_PREC_BF16X3, "f32": N.GKE_PREC_F32}[args.precision]
    tdt = torch.float64 if args.precision == "f64" else torch.float32
    stream = torch.cuda.current_stream()
    sets = []
    for name, stride in GROUP:
        wl = S.WORKLOADS[name]
        f = coefficients_parallel(wl, "cuda")
        st = (0, 0, 0, stride) if stride > 1 else (0, 0, 0, 0)
        plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), wl.nsnap, prec,
                          stream=stream.cuda_stream, under_x=st, under_z=st)
        mz, mx = N.gke_separation_labels(plan)
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), len(mz), len(mx)), dtype=tdt, device="cuda")
        sets.append((wl, stride, plan, f, terms))
    for _ in range(args.warmup):
        for wl, _, plan, f, terms in sets:
            N.gke_compute(plan, f, wl.nsnap, terms)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in sets]
    l0 = sum(N.gke_launch_count(s[2]) for s in sets)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per = [0.0] * len(sets)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            for i, (wl, _, plan, f, terms) in enumerate(sets):
                ev[i][0].record(stream)
                N.gke_compute(plan, f, wl.nsnap, terms)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            for i in range(len(sets)):
                per[i] += ev[i][0].elapsed_time(ev[i][1])
        e1.record(stream)
        torch.cuda.synchronize()
    launches = sum(N.gke_launch_count(s[2]) for s in sets) - l0
    ms = e0.elapsed_time(e1) / args.steps
    units = sum(N.gke_npair(s[2]) * s[0].nsnap for s in sets)
    detail = [{"workload": wl.name, "stride": stride, "pairs": N.gke_npair(plan), "snapshots": wl.nsnap,
               "ms_per_step": per[i] / args.steps} for i, (wl, stride, plan, _, _) in enumerate(sets)]
    for s_ in sets:
        N.gke_destroy(s_[2])
    line = {"metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"f64": "f64", "bf16x3": "bf16x3/f32", "f32": "f32"}[args.precision],
            "data": "synthetic", "config": {"workload": "group of three channel datasets", "datasets": detail,
                                            "precision": args.precision},
            "gpu_launches": launches, "clocks": clk.summary(), "e2e": None, "roofline": None,
            "cpu_baseline": None,
            "note": "datasets run as separate plans back to back (no grouped launch); the 384x384x193 set runs "
                    "at separation stride 2 in the chunked mode (exact aliasing onto a 192x192 separation grid) "
                    "because its full-resolution outputs and accumulators exceed one GPU's memory"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_passes(args):
    """P untimed passes of one plan (no tuning runs, no FP64 run beside it)."""
    import torch
    import paper_1910_06409_gb300._native as N

    wl = S.WORKLOADS[args.workload]
    prec = {"f64": N.GKE_PREC_F64, "bf16x3": N.GKE_PREC_BF16X3, "f32": N.GKE_PREC_F32}[args.precision]
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), wl.nsnap, prec,
                      stream=torch.cuda.current_stream().cuda_stream)
    f_dev = torch.from_numpy(S.coefficients(wl)).cuda()
    tdt = torch.float64 if args.precision == "f64" else torch.float32
    terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), wl.nz, wl.nx), dtype=tdt, device="cuda")
    for p in range(args.passes):
        l0 = N.gke_launch_count(plan)
        N.gke_compute(plan, f_dev, wl.nsnap, terms)
        torch.cuda.synchronize()
        print(f"pass {p}: {N.gke_launch_count(plan) - l0} launches", flush=True)
    N.gke_destroy(plan)


def run_step1(args, world, rank, local):
    """Step 1 for velocity-vorticity databases: all snapshots of the workload
    per step, inputs resident on the device; e2e through pinned host buffers."""
    import torch
    import paper_1910_06409_gb300._native as N

    torch.cuda.set_device(local)
    wl = S.WORKLOADS[args.workload]
    ns = wl.nsnap
    v_eta, mean_uw = S.vorticity_inputs(wl)
    stream = torch.cuda.current_stream()
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), ns, N.GKE_PREC_F64,
                      stream=stream.cuda_stream)
    v_dev, m_dev = torch.from_numpy(v_eta).cuda(), torch.from_numpy(mean_uw).cuda()
    out = torch.empty((ns, 4) + v_eta.shape[2:], dtype=torch.complex128, device="cuda")
    for _ in range(args.warmup):
        N.gke_velocity_vorticity(plan, v_dev, m_dev, ns, out)
    torch.cuda.synchronize()
    l0 = N.gke_launch_count(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            N.gke_velocity_vorticity(plan, v_dev, m_dev, ns, out)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = N.gke_launch_count(plan) - l0
    ms = e0.elapsed_time(e1) / args.steps
    e2e = None
    if not args.no_e2e:
        v_h = torch.from_numpy(v_eta).pin_memory()
        m_h = torch.from_numpy(mean_uw).pin_memory()
        o_h = torch.empty(out.shape, dtype=torch.complex128).pin_memory()
        N.gke_velocity_vorticity(plan, v_h, m_h, ns, o_h)
        t0 = time.perf_counter()
        N.gke_velocity_vorticity(plan, v_h, m_h, ns, o_h)
        ms_e2e = (time.perf_counter() - t0) * 1e3
        e2e = {"value": ns / (ms_e2e / 1e3), "unit": "snapshots/s", "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": int(v_h.numel() * 16 + m_h.numel() * 8),
               "d2h_bytes_per_step": int(o_h.numel() * 16)}
    N.gke_destroy(plan)
    # FP64 work of the transforms (5 N log2 N per complex length-N DFT): per
    # snapshot 3 + 6 column DFTs of length nz per (y, kx), 5 row DFTs of
    # length nx per (y, z)
    lg = lambda n: float(np.log2(n))
    flops = ns * wl.ny * ((3 + 6) * wl.nxh * 5 * wl.nz * lg(wl.nz) + wl.nz * 5 * 5 * wl.nx * lg(wl.nx))
    pk, pk_kind = peaks()
    peak = N_SM * FP64_FLOP_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    ach = flops / (ms / 1e3) / 1e12
    io_bytes = ns * 6 * wl.ny * wl.nz * wl.nxh * 16
    line = {"metric": "Step-1 velocity-vorticity -> u, v, w, p snapshots/s", "value": ns / (ms / 1e3),
            "unit": "snapshots/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "nx": wl.nx, "nz": wl.nz, "ny": wl.ny, "snapshots": ns,
                       "l2": "inputs and outputs larger than L2 (no flush)"},
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "flops": flops, "note": "FP64 DFT work, 5 N log2 N per transform",
                         "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x max SM clock"},
            "hbm": {"bytes": io_bytes, "achieved_gbs": io_bytes / (ms / 1e3) / 1e9, "peak_gbs": pk["hbm_gbs"],
                    "note": "inputs read once and outputs written once"},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------- one homogeneous direction
METRIC_1H = "GKE one-homogeneous-direction (p1,p2)-pair correlations/s, FP64"


# DRAM bytes of one k1_correlate launch on the small case duct_256x17x17_s16
# (41,905 pairs), scaled in proportion to the pairs of the workload run
# (profiles/k1_correlate_profile_duct_256x17x17_s16.md)
NCU_CORR_1H = (0.749e9, 41905)


def correlator_cmac_1h(wl, ns):
    """Complex multiply-adds of the one-direction correlator per pass: 37
    contractions over the snapshots for every pair p1 <= p2 and wavenumber
    (nine velocity pairs, eight for Phi_x, ten each for the y and z fluxes)."""
    return 37 * ns * wl.npair * wl.nxh


def oracle_sample_1h(wl, phys, npts, seed=0):
    """Time the one-direction oracle on npts sampled (pair, separation) points.
    Returns (pair-snapshots/s, seconds, description)."""
    from oracle import one_homog as O1
    rng = np.random.default_rng(seed)
    P = wl.npoint
    pts = []
    for _ in range(npts):
        a, b = sorted(rng.integers(0, P, 2).tolist())
        pts.append((a, b, int(rng.integers(wl.nx))))
    t0 = time.perf_counter()
    O1.points(phys, S.cgl_grid(wl.ny), S.cgl_grid(wl.nz), wl.Lx, wl.nu, pts)
    dt = time.perf_counter() - t0
    rate = npts / float(wl.nx) * wl.nsnap / dt
    desc = (f"{npts} (pair, separation) points of {wl.name}, all terms but the residual, including the "
            f"oracle's per-call set-up; rate = points/nx x snapshots / time")
    return rate, dt, desc


def config_1h(wl):
    return {"workload": wl.name, "nx": wl.nx, "ny": wl.ny, "nz": wl.nz, "snapshots": wl.nsnap,
            "pairs": wl.npair, "precision": "f64", "Lx": round(wl.Lx, 6), "nu": wl.nu,
            "l2": "operands, spectra and terms larger than L2 (no flush)"}


def run_one_homog(args, world, rank, local):
    """The GKE of a flow homogeneous in x only (a duct): all snapshots per
    step, inputs resident on the device; e2e through pinned host buffers."""
    import torch
    import paper_1910_06409_gb300._native as N

    torch.cuda.set_device(local)
    wl = S.DUCT_WORKLOADS[args.workload]
    ns = wl.nsnap
    coef = S.duct_coefficients(wl)
    stream = torch.cuda.current_stream()
    y, z = S.cgl_grid(wl.ny), S.cgl_grid(wl.nz)
    plan = N.gke1h_plan(wl.nx, wl.ny, wl.nz, wl.Lx, wl.nu, y, z, ns, stream=stream.cuda_stream)
    f_dev = torch.from_numpy(coef).cuda()
    terms = torch.empty((N.GKE1H_NTERM, wl.npair, wl.nx), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        N.gke1h_compute(plan, f_dev, ns, terms)
    torch.cuda.synchronize()
    l0 = N.gke1h_launch_count(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            N.gke1h_compute(plan, f_dev, ns, terms)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = N.gke1h_launch_count(plan) - l0
    ms = e0.elapsed_time(e1) / args.steps
    # per-stage device times of one more pass (events on the plan's stream)
    N.gke1h_set_timing(plan, True)
    N.gke1h_compute(plan, f_dev, ns, terms)
    stage_ms = N.gke1h_stage_times(plan)
    N.gke1h_set_timing(plan, False)
    e2e = None
    if not args.no_e2e:
        f_h = torch.from_numpy(coef).pin_memory()
        t_h = torch.empty(tuple(terms.shape), dtype=torch.float64).pin_memory()
        N.gke1h_compute(plan, f_h, ns, t_h)
        t0 = time.perf_counter()
        for _ in range(2):
            N.gke1h_compute(plan, f_h, ns, t_h)
        ms_e2e = (time.perf_counter() - t0) * 1e3 / 2
        e2e = {"value": wl.npair * ns / (ms_e2e / 1e3), "unit": UNIT, "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": int(f_h.numel() * 16), "d2h_bytes_per_step": int(t_h.numel() * 8)}
        del t_h
    f32 = None
    if not args.no_split:
        f32 = run_f32_beside_1h(wl, ns, f_dev, terms, ms, y, z, stream)
    del terms
    N.gke1h_destroy(plan)
    pk, pk_kind = peaks()
    peak = N_SM * FP64_FLOP_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    cms = stage_ms.get("correlate", 0.0)
    flops = 8.0 * correlator_cmac_1h(wl, ns)
    ach = flops / (cms / 1e3) / 1e12 if cms > 0 else 0.0
    roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "flops": flops, "launch_ms": cms, "stage": "correlate",
            "traffic": int(NCU_CORR_1H[0] * wl.npair / NCU_CORR_1H[1]) if ns == 16 else None,
            "traffic_note": "small-case ncu capture scaled by pairs",
            "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x max SM clock (nominal 1.25 TFLOP/s FP64)"}
    cpu = None
    if not args.no_cpu:
        phys = S.duct_physical(wl)
        rate, dt, desc = oracle_sample_1h(wl, phys, args.cpu_points // 8)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": desc,
               "seconds": dt}
    line = {"metric": METRIC_1H, "value": wl.npair * ns / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_1h(wl),
            "f32": f32, "roofline": roof, "stage_ms": {k: round(v, 3) for k, v in stage_ms.items()}, "e2e": e2e,
            "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def one_homog_compact(steps=3, warmup=2):
    """The duct workload's FP64 pass and the FP32 variant beside it, as a
    compact summary for the channel benchmark's line (device-resident inputs,
    CUDA events on the plan's stream)."""
    import torch
    import paper_1910_06409_gb300._native as N

    wl = S.DUCT
    ns = wl.nsnap
    stream = torch.cuda.current_stream()
    y, z = S.cgl_grid(wl.ny), S.cgl_grid(wl.nz)
    f_dev = torch.from_numpy(S.duct_coefficients(wl)).cuda()
    plan = N.gke1h_plan(wl.nx, wl.ny, wl.nz, wl.Lx, wl.nu, y, z, ns, stream=stream.cuda_stream)
    terms = torch.empty((N.GKE1H_NTERM, wl.npair, wl.nx), dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        N.gke1h_compute(plan, f_dev, ns, terms)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        N.gke1h_compute(plan, f_dev, ns, terms)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    N.gke1h_set_timing(plan, True)
    N.gke1h_compute(plan, f_dev, ns, terms)
    stage_ms = N.gke1h_stage_times(plan)
    N.gke1h_destroy(plan)
    f32 = run_f32_beside_1h(wl, ns, f_dev, terms, ms, y, z, stream, steps=steps, warmup=1)
    del terms, f_dev
    torch.cuda.empty_cache()
    pk, _ = peaks()
    peak = N_SM * FP64_FLOP_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    cms = stage_ms.get("correlate", 0.0)
    frac = 8.0 * correlator_cmac_1h(wl, ns) / (cms / 1e3) / 1e12 / peak if cms > 0 else None
    return {"metric": METRIC_1H, "workload": wl.name, "value": wl.npair * ns / (ms / 1e3), "unit": UNIT,
            "ms_per_step": round(ms, 3), "correlator_fp64_frac": None if frac is None else round(frac, 4),
            "stage_ms": {k: round(v, 3) for k, v in stage_ms.items()},
            "f32": {"value": f32["value"], "ms_per_step": f32["ms_per_step"],
                    "speedup_vs_f64": f32["speedup_vs_f64"], "max_rel_err_vs_f64": f32["max_rel_err_vs_f64"]}}


def run_f32_beside_1h(wl, ns, f_dev, terms64, ms64, y, z, stream, steps=5, warmup=2):
    """The FP32 variant on the same inputs: device time per pass, speed-up
    over FP64, per-term maximum deviation from the FP64 result (relative to
    each FP64 term's largest magnitude) and its correlator roofline."""
    import torch
    import paper_1910_06409_gb300._native as N

    plan = N.gke1h_plan(wl.nx, wl.ny, wl.nz, wl.Lx, wl.nu, y, z, ns, stream=stream.cuda_stream,
                        precision=N.GKE_PREC_F32)
    t32 = torch.empty(tuple(terms64.shape), dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        N.gke1h_compute(plan, f_dev, ns, t32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        N.gke1h_compute(plan, f_dev, ns, t32)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    N.gke1h_set_timing(plan, True)
    N.gke1h_compute(plan, f_dev, ns, t32)
    stage_ms = N.gke1h_stage_times(plan)
    N.gke1h_destroy(plan)
    err = {}
    for t, name in enumerate(N.TERMS_1H):
        ref = terms64[t]
        err[name] = float("%.3g" % float((t32[t].double() - ref).abs().max() / ref.abs().max()))
    del t32
    pk, _ = peaks()
    peak = N_SM * FP32_FLOP_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    cms = stage_ms.get("correlate", 0.0)
    flops = 8.0 * correlator_cmac_1h(wl, ns)
    ach = flops / (cms / 1e3) / 1e12 if cms > 0 else 0.0
    return {"value": wl.npair * ns / (ms / 1e3), "unit": UNIT, "ms_per_step": round(ms, 3),
            "speedup_vs_f64": round(ms64 / ms, 2), "max_rel_err_vs_f64": err,
            "stage_ms": {k: round(v, 3) for k, v in stage_ms.items()},
            "roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                         "frac": round(ach / peak, 4), "launch_ms": round(cms, 3), "stage": "correlate",
                         "peak_source": "derived: 152 SM x 128 FFMA/clk x 2 flop x max SM clock"}}


def run_reference_1h(args, world, rank):
    if rank != 0:
        return
    wl = S.DUCT_WORKLOADS[args.workload]
    phys = S.duct_physical(wl)
    from oracle import one_homog as O1
    O1.build()
    npts = max(8, args.ref_points // 8)
    for _ in range(args.warmup):
        oracle_sample_1h(wl, phys, 8, seed=99)
    times, rates = [], []
    for k in range(args.steps):
        r, dt, desc = oracle_sample_1h(wl, phys, npts, seed=k)
        times.append(dt)
        rates.append(r)
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC_1H, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_1h(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_passes_1h(args):
    """P untimed passes of the one-direction plan (profiling target)."""
    import torch
    import paper_1910_06409_gb300._native as N

    wl = S.DUCT_WORKLOADS[args.workload]
    plan = N.gke1h_plan(wl.nx, wl.ny, wl.nz, wl.Lx, wl.nu, S.cgl_grid(wl.ny), S.cgl_grid(wl.nz), wl.nsnap,
                        stream=torch.cuda.current_stream().cuda_stream)
    f_dev = torch.from_numpy(S.duct_coefficients(wl)).cuda()
    terms = torch.empty((N.GKE1H_NTERM, wl.npair, wl.nx), dtype=torch.float64, device="cuda")
    for p in range(args.passes):
        l0 = N.gke1h_launch_count(plan)
        N.gke1h_compute(plan, f_dev, wl.nsnap, terms)
        torch.cuda.synchronize()
        print(f"pass {p}: {N.gke1h_launch_count(plan) - l0} launches", flush=True)
    N.gke1h_destroy(plan)


def run_ours(args, world, rank, local):
    import torch
    import paper_1910_06409_gb300._native as N

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = S.WORKLOADS[args.workload]
    ns = wl.nsnap
    prec = {"f64": N.GKE_PREC_F64, "bf16x3": N.GKE_PREC_BF16X3, "f32": N.GKE_PREC_F32}[args.precision]
    coef = S.coefficients(wl)
    in_bytes = coef.nbytes
    stream = torch.cuda.current_stream()
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), ns, prec,
                      stream=stream.cuda_stream)
    npair = N.gke_npair(plan)
    f_dev = torch.from_numpy(coef).cuda()
    tdt = torch.float64 if args.precision == "f64" else torch.float32      # terms element type
    terms = torch.empty((N.GKE_NTERM, npair, wl.nz, wl.nx), dtype=tdt, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        N.gke_compute(plan, f_dev, ns, terms)
    torch.cuda.synchronize()
    N.gke_set_timing(plan, True)
    N.gke_stage_times(plan)            # clear
    l0 = N.gke_launch_count(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            N.gke_compute(plan, f_dev, ns, terms)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = N.gke_launch_count(plan) - l0
    stage = N.gke_stage_times(plan)
    N.gke_set_timing(plan, False)
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * npair * ns / (ms / 1e3)

    # end to end through the public call with host buffers (pinned); the
    # split run beside reuses the same pinned buffers
    e2e = None
    pinned = None
    if not args.no_e2e:
        f_host = torch.from_numpy(coef).pin_memory()
        tshape = (N.GKE_NTERM, npair, wl.nz, wl.nx)
        out_raw = torch.empty(int(np.prod(tshape)) * (8 if tdt == torch.float64 else 4), dtype=torch.uint8).pin_memory()
        out_host = out_raw.view(tdt).view(tshape)
        pinned = (f_host, out_raw)
        N.gke_compute(plan, f_host, ns, out_host)     # warm-up (allocates staging once)
        torch.cuda.synchronize()
        ke = max(1, min(args.steps, 3))
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ke):
            N.gke_compute(plan, f_host, ns, out_host)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_e2e = e0.elapsed_time(e1) / ke
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms_e2e], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e = float(t.item())
        e2e = {"value": world * npair * ns / (ms_e2e / 1e3), "unit": UNIT, "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": int(out_host.numel() * out_host.element_size())}
        del out_host
    N.gke_destroy(plan)

    # split-BF16 path on the same inputs: throughput, speed-up and per-term error vs the FP64 GPU path
    split = f32v = None
    if args.precision == "f64" and not args.no_split:
        split = run_split_beside(args, wl, ns, f_dev, terms, ms, barrier, world, "bf16x3", pinned)
        f32v = run_split_beside(args, wl, ns, f_dev, terms, ms, barrier, world, "f32")
    pinned = None
    # the one-homogeneous-direction variant on its duct workload, compact
    one_h = None
    if args.precision == "f64" and not args.no_split and world == 1:
        try:
            one_h = one_homog_compact()
        except Exception as e:          # a failure here must not lose the channel line
            one_h = {"error": str(e)[:200]}

    # rooflines: every stage against its bound, the dominant stage reported as "roofline"
    pk, pk_kind = peaks()
    clocks = clk.summary()
    stage_ms = {k: v / args.steps for k, v in stage.items()}
    rl = stage_rooflines(wl, ns, args.precision, stage_ms, pk, pk_kind)
    dominant = max(rl, key=lambda k: rl[k]["launch_ms"])
    roof = dict(rl[dominant], stage=dominant)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        phys = S.physical(wl)
        r, dt, desc = oracle_sample(wl, phys, args.cpu_points, 2, seed=123)
        cpu = {"value": r, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": desc,
               "seconds": dt}
    if rank == 0:
        # the split-BF16 result (the metric's subject) first and compact, the
        # per-stage tables last, so a truncated tail of the line keeps it
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"f64": "f64", "bf16x3": "bf16x3/f32", "f32": "f32"}[args.precision],
                "data": "synthetic",
                "split_bf16x3": compact(split), "one_homog": one_h, "config": config_of(wl, args.precision),
                "roofline": roof, "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "cpu_baseline": cpu,
                "parallelism": f"replicas{world}", "fp32_cuda_cores": compact(f32v),
                "stage_ms": {k: round(v, 3) for k, v in stage_ms.items()},
                "stage_roofline": {k: short_roof(v) for k, v in rl.items()},
                "split_stage_roofline": None if split is None else {k: short_roof(v) for k, v in
                                                                    split["stage_roofline"].items()}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_split_beside(args, wl, ns, f_dev, terms64, ms64, barrier, world, precision, pinned=None):
    """Time the split-BF16 (or FP32) path on the FP64 run's inputs and compare its terms.

    Error per term: max |split - f64| / max |f64| over all pairs and
    separations, against the FP64 GPU path (itself within 1e-12 of the
    oracle)."""
    import torch
    import paper_1910_06409_gb300._native as N
    stream = torch.cuda.current_stream()
    prec = {"bf16x3": N.GKE_PREC_BF16X3, "f32": N.GKE_PREC_F32}[precision]
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), ns, prec,
                      stream=stream.cuda_stream)
    npair = N.gke_npair(plan)
    t32 = torch.empty_like(terms64, dtype=torch.float32)
    for _ in range(args.warmup):
        N.gke_compute(plan, f_dev, ns, t32)
    torch.cuda.synchronize()
    N.gke_set_timing(plan, True)
    N.gke_stage_times(plan)
    l0 = N.gke_launch_count(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        N.gke_compute(plan, f_dev, ns, t32)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = N.gke_launch_count(plan) - l0
    stage_ms = {k: v / args.steps for k, v in N.gke_stage_times(plan).items()}
    N.gke_set_timing(plan, False)
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # end to end through the public call with pinned host buffers: the
    # snapshots in and the terms out inside the timed region
    e2e = None
    if not args.no_e2e and precision == "bf16x3":
        if pinned is not None:
            f_host = pinned[0]
            out_host = pinned[1][:t32.numel() * 4].view(torch.float32).view(t32.shape)
        else:
            f_host = f_dev.cpu().pin_memory()
            out_host = torch.empty(t32.shape, dtype=torch.float32).pin_memory()
        N.gke_compute(plan, f_host, ns, out_host)
        torch.cuda.synchronize()
        ke = max(1, min(args.steps, 3))
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ke):
            N.gke_compute(plan, f_host, ns, out_host)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_e2e = e0.elapsed_time(e1) / ke
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms_e2e], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e = float(t.item())
        e2e = {"value": world * npair * ns / (ms_e2e / 1e3), "unit": UNIT, "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": int(f_host.numel() * f_host.element_size()),
               "d2h_bytes_per_step": int(out_host.numel() * out_host.element_size())}
        del f_host, out_host
    N.gke_destroy(plan)
    err = {}
    for t, name in enumerate(TERM_NAMES):
        ref = terms64[t]
        scale = float(ref.abs().max())
        diff = float((t32[t].double() - ref).abs().max())
        err[name] = diff / scale if scale > 0 else diff
    del t32
    pk, pk_kind = peaks()
    rl = stage_rooflines(wl, ns, precision, stage_ms, pk, pk_kind)
    return {"value": world * npair * ns / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "e2e": e2e,
            "speedup_vs_f64": ms64 / ms, "max_rel_err": err, "tolerance": 1e-6,
            "within_tolerance": all(e <= 1e-6 for e in err.values()),
            "stage_ms": stage_ms, "gpu_launches": launches, "roofline": rl.get("correlate"),
            "stage_roofline": rl}


TERM_NAMES = ("A", "Phi_x", "Phi_y", "Phi_z", "phi", "xi", "residual")


def short_roof(r):
    """A stage roofline with rounded figures."""
    if r is None:
        return None
    keep = ("bound", "achieved", "peak", "unit", "frac", "launch_ms", "traffic")
    return {k: (round(r[k], 4) if isinstance(r.get(k), float) else r.get(k)) for k in keep if k in r}


def compact(run):
    """The split-path summary printed early in the JSON line."""
    if run is None:
        return None
    return {"value": run["value"], "unit": run["unit"], "ms_per_step": round(run["ms_per_step"], 3),
            "speedup_vs_f64": round(run["speedup_vs_f64"], 2),
            "max_rel_err": {k: float("%.3g" % v) for k, v in run["max_rel_err"].items()},
            "tolerance": run["tolerance"], "within_tolerance": run["within_tolerance"],
            "roofline": short_roof(run["roofline"]), "e2e": run.get("e2e"),
            "stage_ms": {k: round(v, 3) for k, v in run["stage_ms"].items()}, "gpu_launches": run["gpu_launches"]}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("f64", "bf16x3", "f32"), default="f64")
    ap.add_argument("--workload", default=S.RETAU200.name,
                    choices=sorted(S.WORKLOADS) + sorted(S.DUCT_WORKLOADS) + ["group"],
                    help="a channel workload, 'group', or a duct (one homogeneous direction)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-split", action="store_true",
                    help="with --precision f64: skip the split-BF16 run beside it")
    ap.add_argument("--cpu-points", type=int, default=2048)
    ap.add_argument("--ref-points", type=int, default=1024)
    ap.add_argument("--pair-domain", choices=("triangle", "wedge"), default="triangle",
                    help="wedge: y-inversion mirror sampling on the half-channel wedge (streaming mode)")
    ap.add_argument("--stride", type=int, default=1, help="uniform undersampling of r_x, r_z (streaming mode)")
    ap.add_argument("--batch", type=int, default=0, help="snapshots per accumulate call (streaming mode)")
    ap.add_argument("--nsnap", type=int, default=0, help="first n snapshots of the workload only (streaming mode)")
    ap.add_argument("--no-f64-check", action="store_true",
                    help="streaming mode: skip the untimed FP64 run that measures the per-term error")
    ap.add_argument("--step1", action="store_true",
                    help="time Step 1 for velocity-vorticity databases on the workload's snapshots")
    ap.add_argument("--passes", type=int, default=0,
                    help="profiling target: run this many untimed passes, print launches per pass, exit")
    args = ap.parse_args()
    duct = args.workload in S.DUCT_WORKLOADS
    if args.passes > 0:
        (run_passes_1h if duct else run_passes)(args)
        return
    world, rank, local = dist_setup()
    if duct:
        (run_reference_1h(args, world, rank) if args.impl == "reference" else run_one_homog(args, world, rank, local))
    elif args.impl == "reference":
        run_reference(args, world, rank)
    elif args.step1:
        run_step1(args, world, rank, local)
    elif args.workload == "group":
        run_group(args, world, rank, local)
    elif args.pair_domain != "triangle" or args.stride > 1 or args.batch:
        run_stream(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
