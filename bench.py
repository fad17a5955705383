"""Benchmark of the PML-BIE hot path on GB300.

Workload (one step = one full solve of one problem instance): two layers with
omega_1 = 4 pi above and omega_2 = 6 pi below, Gaussian bump of height 0.2
(r <= 1), cylindrical PML a1 = 2.5, T = 1, S = 3, N = 512 curve nodes,
M = 256 azimuthal samples (128 distinct modes, 1024 x 1024 complex system per
mode), plane wave from polar angle 30 degrees.  The step computes every modal
kernel (far pairs by FFT, close pairs by the kernel split), assembles the
Alpert-corrected block systems, builds the right-hand side, factors every
mode's system and solves it.  Synthetic, deterministic inputs (no dataset).

Metric: modal kernel entries per second of whole solve, entries = 4 N^2 M/2
per problem (S and K of both media on every node pair and distinct mode), for
the mixed path (FP64 kernels, FP32 LU, FP64 refinement to 1e-13 residual);
the plain FP64 GPU path is timed on the same problem for comparison.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run: every rank solves its own problem
instance (independent problems, no data-path collective; weak scaling).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(k1=4 * np.pi, k2=6 * np.pi, N=512, M=256, a1=2.5, T=1.0, S=3.0, bump_h=0.2, polar=np.pi / 6)
# smaller case of the same physics for profiler captures (matrices ~270 MB, above L2)
WORKLOADS = {"default": WORKLOAD, "small": dict(WORKLOAD, N=256, M=128),
             # large single instance and the smallest high-frequency instance
             "n1024_m512": dict(WORKLOAD, k1=10 * np.pi, k2=15 * np.pi, N=1024, M=512),
             "n1536_m512": dict(WORKLOAD, k1=12 * np.pi, k2=18 * np.pi, N=1536, M=512),
             # the high-frequency sweep's largest instance: its per-mode blocks
             # (412 GB for the mixed path) exceed HBM, so the solve runs in mode chunks
             "n4096_m512": dict(WORKLOAD, k1=20 * np.pi, k2=30 * np.pi, N=4096, M=512)}
METRIC = "modal kernel entries/s and solve s/problem, mixed vs FP64 GPU at 1e-6 rel err"
UNIT = "entries/s"


# ----------------------------------------------------------------------------
# multi-rank host logic (one process per GPU, independent problems: no
# data-path collective; the timing takes the slowest rank)
# ----------------------------------------------------------------------------
def init_dist(world, backend="nccl", device=None):
    """The process group for world > 1 (None for one rank)."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if device is not None:
        dist.init_process_group(backend, device_id=device)
    else:
        dist.init_process_group(backend)
    return dist


def max_over_ranks(ms, dist, device="cuda"):
    """The largest per-rank time (the job's time); ms itself for one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_value(world, units_per_rank, ms):
    """Whole-job throughput: every rank processes units_per_rank in ms."""
    return world * units_per_rank / (ms / 1e3)


def emit_line(line, rank, out=None):
    """Rank 0 prints the one JSON line; the other ranks print nothing."""
    if rank == 0:
        print(json.dumps(line), file=out or sys.stdout)
        return True
    return False


def entries_per_problem(w):
    return 4 * w["N"] ** 2 * (w["M"] // 2)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling every 50 ms in a child process; summary() keeps the
    samples whose timestamps fall inside the marked window (mark_start /
    mark_end around the timed region)."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None
        self.rows = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.5)   # first samples arrive before the timed region starts
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.1)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        import datetime
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) != 8:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            if self.t0 is not None and self.t1 is not None and not (self.t0 <= ts <= self.t1):
                continue
            self.rows.append(f[1:])

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------
# oracle (CPU baseline / reference arm): bounded sample of the same workload
# ----------------------------------------------------------------------------
def oracle_sample(w, rows=6):
    """Modal kernels (4 kernels, all distinct modes) of `rows` target nodes
    against every source node and their Alpert correction points, by the FP64
    CPU oracle.  Returns (entries computed, seconds)."""
    from oracle import kernels as KR
    from oracle.assemble import Quadrature
    from oracle.problem import Geometry, Params
    P = Params(k1=w["k1"], k2=w["k2"], N=w["N"], M=w["M"], a1=w["a1"], T=w["T"], S=w["S"], bump_h=w["bump_h"])
    G = Geometry(P)
    Q = Quadrature(G)
    sel = np.linspace(0, P.N - 1, rows).round().astype(int)
    t0 = time.perf_counter()
    for l in sel:
        src_m = np.nonzero(Q.grid_mask[l])[0]
        cidx = np.nonzero(Q.corr_target == l)[0]
        tg = {k: np.repeat(G.nodes[k][l], len(src_m) + len(cidx)) for k in ("rho", "z", "z_t", "rho_t", "bk", "ox", "oz")}
        sc = {k: np.concatenate([G.nodes[k][src_m], Q.corr_pts[k][cidx]])
              for k in ("rho", "z", "z_t", "rho_t", "nuc_r", "nuc_z", "bk", "ox", "oz")}
        pg = KR.pair_geometry(tg, sc, P)
        near = KR.near_mask(pg, P)
        lap = KR.laplace_modes({k: v[near] for k, v in pg.items()}, P.M - 2)
        for omega, sign in ((P.k1, 1.0), (P.k2, -1.0)):
            pgr = dict(pg)
            pgr["nuc_r"] = sign * pg["nuc_r"]
            pgr["nuc_z"] = sign * pg["nuc_z"]
            full = (np.zeros((len(near), P.M - 1), complex), np.zeros((len(near), P.M - 1), complex))
            full[0][near] = lap[0]
            full[1][near] = sign * lap[1]
            KR.modal_kernels(pgr, omega, P, lap=full, near=near)
    dt = time.perf_counter() - t0
    return rows * 4 * P.N * (P.M // 2), dt


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    w = WORKLOAD
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(w, rows=4)
    tot_e, tot_t = 0, 0.0
    for _ in range(args.steps):
        e, t = oracle_sample(w, rows=8)
        tot_e += e
        tot_t += t
    v = tot_e / tot_t
    cores = cpu_cores()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "two-layer bump, N=512 M=256 (128 modes), k1=4pi k2=6pi, PML a1=2.5 T=1 S=3, "
                                   "1 plane wave", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "modal kernels of 8 target rows x all sources + Alpert points, all "
                                       "128 modes, 4 kernels, per step (FP64 numpy oracle)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300 import binding as B
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = init_dist(world, "nccl", torch.device("cuda", dev))
    w = WORKLOAD
    kw = dict(a1=w["a1"], T=w["T"], S=w["S"], bump_h=w["bump_h"])
    pipes = measure_pipes(B)
    P = Problem(w["k1"], w["k2"], w["N"], w["M"], **kw)
    shape = (w["M"] // 2, w["N"], 1)
    outs = {k: torch.empty(shape, dtype=torch.complex128, device="cuda") for k in ("u1", "phi1", "u2", "phi2")}
    stream = torch.cuda.current_stream()
    polar = [w["polar"]]

    def step(prec):
        return P.solve(polar, precision=prec, stream=stream, outputs=outs)[1]

    for _ in range(max(args.warmup, 3)):
        rep = step(B.PMLBIE_MIXED)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    reps = []
    with ClockSampler(dev) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        clk.mark_start()
        e0.record(stream)
        for _ in range(args.steps):
            reps.append(step(B.PMLBIE_MIXED))
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist)
    mixed_out = {k: v.clone() for k, v in outs.items()}

    # plain FP64 GPU path on the same problem (1 warm + 2 timed); for N >= 1024
    # on modes 0-15 only (0-1 for N >= 3072), the time scaled to all modes
    # (modes cost alike)
    nm = w["M"] // 2
    sub = (0, nm) if w["N"] < 1024 else ((0, 16) if w["N"] < 3072 else (0, 2))
    sub_outs = {k: torch.empty((sub[1] - sub[0],) + shape[1:], dtype=torch.complex128, device="cuda")
                for k in outs}

    def step64():
        if sub == (0, nm):
            return P.solve(polar, precision=B.PMLBIE_FP64, stream=stream, outputs=sub_outs)[1]
        return P.solve(polar, precision=B.PMLBIE_FP64, stream=stream, outputs=sub_outs, modes=sub)[1]

    step64()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    fp64_reps = [step64() for _ in range(2)]
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1) / 2 * nm / (sub[1] - sub[0])
    rel = {k: (torch.linalg.vector_norm(mixed_out[k][sub[0]:sub[1]] - sub_outs[k]) /
               torch.linalg.vector_norm(sub_outs[k])).item() for k in outs}
    # scattered field at 32 fixed points (16 at z = +1 above, 16 at z = -1 below,
    # rho in [0, 2]) from the mixed and the FP64 densities, same modes
    fr = np.tile(np.linspace(0.0, 2.0, 16), 2)
    fz = np.repeat([1.0, -1.0], 16)
    fg = np.repeat([0, 1], 16)
    f64 = P.field(fr, fz, fg, sub_outs, modes=sub, stream=stream)
    f32 = P.field(fr, fz, fg, {k: v[sub[0]:sub[1]].contiguous() for k, v in mixed_out.items()}, modes=sub,
                  stream=stream)
    rel["field_32_points"] = (torch.linalg.vector_norm(f32 - f64) / torch.linalg.vector_norm(f64)).item()
    oracle_err = oracle_errors(w, sub, {"mixed": (mixed_out, f32), "fp64": (sub_outs, f64)})

    ng, nc = P.near_count()
    ncounts = near_counts(P)
    h2d = h2d_bytes(P, w)
    chunks = reps[-1].chunks
    # the device workspace of P goes before the end-to-end runs create their own
    P.close()
    torch.cuda.empty_cache()

    # end to end through the public API with host buffers: create (host tables,
    # first-call upload) + solve + copy of the outputs to pinned host memory
    pinned = [torch.empty(shape, dtype=torch.complex128, pin_memory=True).numpy() for _ in range(4)]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    create_s = 0.0
    for _ in range(e2e_steps):
        tc = time.perf_counter()
        Q = Problem(w["k1"], w["k2"], w["N"], w["M"], **kw)
        create_s += time.perf_counter() - tc
        B.pmlbie_solve_host(Q.handle, B.PMLBIE_MIXED, polar, *pinned, stream=stream)
        Q.close()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / e2e_steps, dist)
    create_ms = 1e3 * create_s / e2e_steps
    d2h = 4 * int(np.prod(shape)) * 16

    last = reps[-1]
    epp = entries_per_problem(w)
    value = job_value(world, epp, ms)
    pk = peaks()
    stages = {"far_kernel_ff": last.ms_far, "near_laplace_kernel": last.ms_near_laplace,
              "near_modes_kernel_ff": last.ms_near_ff,
              "near_modes_kernel_fp64_pml": last.ms_near - last.ms_near_laplace - last.ms_near_ff,
              "assemble": last.ms_assemble, "lu_fp32": last.ms_lu, "solve_refine": last.ms_solve}
    clocks = clk.summary()
    roof = near_roofline(w, last, pk, clocks, ncounts, pipes)
    roof_far = roofline(w, last, pk, clocks, pipes)
    roof_lu = lu_update_roofline(w, last, pk)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "float-float (FP32 pairs) sampling/FFT, FP64 PML close pairs and Laplace modes, c64 LU, c128 refinement",
        "data": "synthetic",
        "config": {"workload": "two-layer bump, N=%d M=%d (%d modes), k1=%gpi k2=%gpi, PML a1=2.5 T=1 S=3, "
                               "1 plane wave at 30 deg, mixed precision" % (w["N"], w["M"], w["M"] // 2,
                                                                           w["k1"] / np.pi, w["k2"] / np.pi),
                   "parallelism": "independent problems per GPU" if world > 1 else "1 GPU",
                   "l2": "working set > L2 (129 MB): %d MB of per-mode matrices rebuilt every step" %
                         int(((w["M"] // 2) * (2 * w["N"]) ** 2 * 24) / 1e6)},
        "solve_s_per_problem": ms / 1e3,
        "kernel_entries_per_s": epp / ((max(last.ms_far, last.ms_near) + last.ms_assemble) / 1e3),
        "far_pairs": last.far_pairs, "far_pairs_sampled": last.far_pairs_sampled,
        "far_pairs_per_cta": last.far_pairs_per_cta,
        "stages_ms": {k: round(v, 4) for k, v in stages.items()},
        "stages_note": ("far_kernel_ff runs beside the close-pair kernels (near_*, on a high-priority stream): "
                        "their times overlap; the others are sequential"),
        "mode_chunks": chunks,
        "refine_iters": last.refine_iters, "refine_residual": last.residual,
        "refine_backward_error": last.backward_error, "gmres_modes": last.gmres_modes,
        "gmres_iters": last.gmres_iters,
        "fp64_gpu": {"ms_per_step": ms64, "value": world * epp / (ms64 / 1e3),
                     "modes_timed": list(sub), "stages_ms": {
            "far_kernel": fp64_reps[-1].ms_far, "near_kernels": fp64_reps[-1].ms_near,
            "assemble": fp64_reps[-1].ms_assemble, "lu_fp64": fp64_reps[-1].ms_lu,
            "solve": fp64_reps[-1].ms_solve}},
        "speedup_mixed_vs_fp64": ms64 / ms,
        "mixed_vs_fp64_rel_err": rel,
        "oracle_rel_err": oracle_err,
        "near_pairs": {"grid": ng, "alpert": nc},
        "gpu_launches": int(sum(r.launches for r in reps)),
        "measured_pipe_peaks": pipes,
        "roofline": roof, "roofline_lu_update": roof_lu,
        "roofline_far": roof_far,
        "stage_rooflines": stage_rooflines(w, last, pk, pipes),
        "clocks": clocks,
        "e2e": {"value": world * epp / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "create_ms": create_ms,
                "note": "per step: create (host setup, create_ms of it) + solve_host to pinned buffers + destroy"},
    }
    if world == 1 and WORKLOAD is WORKLOADS["default"] and not args.no_extra:
        line["extra_workloads"] = extra_workloads(stream, pipes)
    if rank == 0 and not args.no_cpu_baseline:
        rows = max(12, int(160 * (512 * 256) / (w["N"] * w["M"])))
        e, t = oracle_sample(w, rows=rows)
        line["cpu_baseline"] = {"value": e / t, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                "sample": "modal kernels of %d target rows x all %d sources + their Alpert "
                                          "points, %d modes, 4 kernels (FP64 numpy oracle), %.1f s" %
                                          (rows, w["N"], w["M"] // 2, t)}
    emit_line(line, rank)
    if dist:
        dist.destroy_process_group()


def extra_workloads(stream, pipes=None):
    """Secondary measurements of the default run (one GPU; not the headline
    value): the large single instance n1024_m512 (one warm-up and two timed
    mixed solves) and the batched eight-instance workload (one warm-up and one
    timed batch call), CUDA events on the launching stream, inputs resident.
    Each reports its own entries/s and time per problem."""
    import torch
    from paper_2412_11162_gb300 import Problem, solve_batch
    from paper_2412_11162_gb300 import binding as B
    out = {}
    w = WORKLOADS["n1024_m512"]
    P = Problem(w["k1"], w["k2"], w["N"], w["M"], a1=w["a1"], T=w["T"], S=w["S"], bump_h=w["bump_h"])
    rep = P.solve([w["polar"]], precision=B.PMLBIE_MIXED, stream=stream)[1]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = [P.solve([w["polar"]], precision=B.PMLBIE_MIXED, stream=stream)[1] for _ in range(2)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 2
    r = reps[-1]
    n2, modes = 2 * w["N"], w["M"] // 2
    lu_flops = 8.0 / 3.0 * n2 ** 3 * modes
    wbytes = 4.0 * w["N"] ** 2 * modes * 16
    tf32 = pipes.get("tf32_tcgen05_tflops") if pipes else None
    hbm = peaks().get("hbm_gbs", 6794.1)
    # the far kernel alone (autotuning launch, per chunk); r.ms_far is its span beside the close pairs
    far_alone = float(getattr(r, "ms_far_alone", 0.0))
    far_ms = far_alone * max(1, r.chunks) if far_alone > 0 else r.ms_far
    out["n1024_m512"] = {"workload": "two-layer bump, N=1024 M=512 (256 modes), k1=10pi k2=15pi, mixed",
                         "ms_per_problem": ms, "entries_per_s": entries_per_problem(w) / (ms / 1e3),
                         "lu_tflops": lu_flops / (r.ms_lu / 1e3) / 1e12,
                         "lu_frac_tf32": (lu_flops / (r.ms_lu / 1e3) / 1e12 / tf32) if tf32 else None,
                         "far_block_writes_gbs": wbytes / (far_ms / 1e3) / 1e9,
                         "far_block_writes_frac_hbm": wbytes / (far_ms / 1e3) / 1e9 / hbm,
                         "note": "LU flops (8/3) (2N)^3 per mode against the measured TF32 tcgen05 rate; the far "
                                 "kernel's 4 N^2 (M/2) x 16 B block writes against the measured HBM copy bandwidth",
                         "stages_ms": {"far": r.ms_far, "near": r.ms_near, "assemble": r.ms_assemble,
                                       "lu": r.ms_lu, "solve_refine": r.ms_solve},
                         "refine_iters": r.refine_iters, "gmres_modes": r.gmres_modes,
                         "backward_error": r.backward_error}
    P.close()
    torch.cuda.empty_cache()
    inst, polar, azimuth = batched_instances()
    probs = [Problem(v["k1"], v["k2"], v["N"], v["M"], a1=v["a1"], T=v["T"], S=v["S"], bump_h=v["bump_h"])
             for v in inst]
    solve_batch(probs, polar, azimuth, precision=B.PMLBIE_MIXED, n_streams=2, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    _, reps = solve_batch(probs, polar, azimuth, precision=B.PMLBIE_MIXED, n_streams=2, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["batched8"] = {"workload": "8 instances (seed 2412): k1=linspace(2pi,8pi,8), k2=1.5 k1, N=%s, M=N/2, "
                                   "64 plane waves each, mixed, one batch call on 2 worker streams" %
                                   [v["N"] for v in inst],
                       "ms_per_batch": ms, "s_per_problem": ms / 1e3 / 8,
                       "entries_per_s": sum(entries_per_problem(v) for v in inst) / (ms / 1e3),
                       "gmres_modes": int(sum(x.gmres_modes for x in reps))}
    for q in probs:
        q.close()
    torch.cuda.empty_cache()
    return out


def measure_pipes(B):
    """TFLOP/s of the FP64 FMA, FP32 FMA and TF32 tensor-core pipes measured on
    this GPU by the library's probe (pmlbie_selftest_peak), before the timed
    region."""
    out = {}
    for kind, name in ((0, "fp64_fma_tflops"), (1, "fp32_fma_tflops"), (2, "tf32_tcgen05_tflops")):
        try:
            out[name] = B.pmlbie_selftest_peak(kind)
        except Exception as e:       # reported, not fatal: the roofline falls back to derived peaks
            out[name] = None
            out[name + "_error"] = str(e)[:200]
    return out


def oracle_errors(w, sub, runs):
    """Relative 2-norm errors of the solves against the FP64 oracle on the
    modes stored in tests/golden/bump_n512_m256_oracle.npz (written by the
    committed script beside it, which calls only oracle/): densities u1, phi1,
    u2, phi2 and the scattered field at the same 32 points.  runs: precision
    -> (outputs [mode][node][rhs] of the modes `sub`, field [mode][point][rhs]).
    None when the workload is not the stored one.  Computed after the timed
    region."""
    path = os.path.join(ROOT, "tests", "golden", "bump_n512_m256_oracle.npz")
    try:
        g = np.load(path)
    except OSError:
        return None
    if (int(g["N"]), int(g["M"])) != (w["N"], w["M"]) or abs(float(g["k1"]) - w["k1"]) > 1e-12 or \
            abs(float(g["k2"]) - w["k2"]) > 1e-12 or abs(float(g["polar"]) - w["polar"]) > 1e-15:
        return None
    modes = [int(n) for n in g["modes"] if sub[0] <= n < sub[1]]
    if not modes:
        return None
    idx = [n - sub[0] for n in modes]
    gi = [list(g["modes"]).index(n) for n in modes]
    out = {"modes": modes, "source": "tests/golden/bump_n512_m256_oracle.npz"}
    for prec, (dens, fld) in runs.items():
        e = {}
        for k in ("u1", "phi1", "u2", "phi2"):
            got = dens[k].cpu().numpy()[idx, :, 0]
            ref = g[k][gi]
            e[k] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        got = fld.cpu().numpy()[idx, :, 0]
        e["field_32_points"] = float(np.linalg.norm(got - g["field"][gi]) / np.linalg.norm(g["field"][gi]))
        out[prec] = e
    return out


def h2d_bytes(P, w):
    """Bytes the first device call uploads: node tables, pair classes,
    close-pair table, Alpert stencils, angle and twiddle tables."""
    ng, nc = P.near_count()
    return (w["N"] * (5 * 8 + 3 * 16 + 3 * 8 + 4 + 16) + w["N"] ** 2 + (ng + nc) * 144 + nc * 4 * (1 + 2 * 10)
            + (w["M"] // 2 + 1 + w["M"] + 2 * w["M"]) * 16 + 8)


def batched_instances():
    """Eight instances (seeded): omega_1 = linspace(2 pi, 8 pi, 8), omega_2 =
    1.5 omega_1, bump heights U[0.1, 0.4], N drawn from {256, 384, 512, 768,
    1024} (after the heights), M = N/2; 64 plane waves: polar (i + 1/2)(pi/2)/8,
    azimuth 2 pi j/8, i, j = 0..7."""
    rng = np.random.default_rng(2412)
    h = rng.uniform(0.1, 0.4, 8)
    Ns = rng.choice([256, 384, 512, 768, 1024], 8)
    k1 = np.linspace(2 * np.pi, 8 * np.pi, 8)
    inst = [dict(WORKLOAD, k1=float(k1[i]), k2=float(1.5 * k1[i]), N=int(Ns[i]), M=int(Ns[i]) // 2,
                 bump_h=float(h[i])) for i in range(8)]
    polar = [(i + 0.5) * (np.pi / 2) / 8 for i in range(8) for _ in range(8)]
    azimuth = [2 * np.pi * j / 8 for _ in range(8) for j in range(8)]
    return inst, polar, azimuth


def run_batched(args, rank, world):
    """One step = one batch call solving the eight instances (mixed precision,
    64 right-hand sides each) on two worker streams."""
    import torch
    from paper_2412_11162_gb300 import Problem, solve_batch
    from paper_2412_11162_gb300 import binding as B
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = init_dist(world, "nccl", torch.device("cuda", dev))
    inst, polar, azimuth = batched_instances()

    def make():
        return [Problem(w["k1"], w["k2"], w["N"], w["M"], a1=w["a1"], T=w["T"], S=w["S"], bump_h=w["bump_h"])
                for w in inst]

    pipes = measure_pipes(B)
    probs = make()
    stream = torch.cuda.current_stream()

    def step():
        return solve_batch(probs, polar, azimuth, precision=B.PMLBIE_MIXED, n_streams=2, stream=stream)

    for _ in range(max(args.warmup, 3)):
        outs, reps = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    steps = max(1, args.steps // 3)
    with ClockSampler(dev) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        clk.mark_start()
        e0.record(stream)
        for _ in range(steps):
            outs, reps = step()
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist)
    ent = sum(entries_per_problem(w) for w in inst)
    # FP64 check on the first instance, all 64 waves
    o64, _ = probs[0].solve(polar, precision=B.PMLBIE_FP64, azimuth=azimuth)
    rel = {k: (torch.linalg.vector_norm(outs[0][k] - o64[k]) / torch.linalg.vector_norm(o64[k])).item()
           for k in o64}
    # end to end: create the 8 problems, batch solve, copy all outputs to pinned host memory
    pinned = [[torch.empty(o["u1"].shape, dtype=torch.complex128, pin_memory=True) for _ in range(4)]
              for o in outs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Q = make()
    qo, _ = solve_batch(Q, polar, azimuth, precision=B.PMLBIE_MIXED, n_streams=2, stream=stream)
    for o, pin in zip(qo, pinned):
        for t, key in zip(pin, ("u1", "phi1", "u2", "phi2")):
            t.copy_(o[key], non_blocking=True)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), dist)
    for q in Q:
        q.close()
    d2h = sum(4 * o["u1"].numel() * 16 for o in outs)
    big = max(range(8), key=lambda i: reps[i].ms_far)
    clocks = clk.summary()
    roof = near_roofline(inst[big], reps[big], peaks(), clocks, near_counts(probs[big]), pipes)
    roof["kernel"] += " of the N=%d instance" % inst[big]["N"]
    roof_far = roofline(inst[big], reps[big], peaks(), clocks, pipes)
    roof_far["kernel"] += " of the N=%d instance" % inst[big]["N"]
    line = {
        "metric": METRIC, "value": job_value(world, ent, ms), "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128 kernels / c64 LU / c128 refinement", "data": "synthetic",
        "config": {"workload": "8 instances (seed 2412): k1=linspace(2pi,8pi,8), k2=1.5 k1, h~U[0.1,0.4], "
                               "N=%s, M=N/2; 64 plane waves (8 polar x 8 azimuth); mixed; 2 worker streams" %
                               [w["N"] for w in inst],
                   "parallelism": "the same batch on every GPU" if world > 1 else "1 GPU",
                   "l2": "working set > L2: every step rebuilds %.1f GB of per-mode matrices" %
                         (sum((w["M"] // 2) * (2 * w["N"]) ** 2 * 24 for w in inst) / 1e9)},
        "solve_s_per_problem": ms / 1e3 / 8,
        "per_instance": [{"N": w["N"], "M": w["M"], "k1_over_pi": w["k1"] / np.pi, "ms_far": r.ms_far,
                          "ms_near": r.ms_near, "ms_lu": r.ms_lu, "ms_solve": r.ms_solve,
                          "refine_iters": r.refine_iters, "gmres_modes": r.gmres_modes,
                          "backward_error": r.backward_error} for w, r in zip(inst, reps)],
        "mixed_vs_fp64_rel_err_instance0": rel,
        "gpu_launches": int(sum(r.launches for r in reps)),
        "roofline": roof, "roofline_far": roof_far, "clocks": clocks,
        "e2e": {"value": job_value(world, ent, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(sum(h2d_bytes(q, w) for q, w in zip(probs, inst))),
                "d2h_bytes_per_step": int(d2h),
                "note": "create the 8 problems (host tables) + batch solve + copy of all outputs to pinned host"},
    }
    emit_line(line, rank)
    if dist:
        dist.destroy_process_group()


def far_flops_per_launch(M, chunk_modes, sampled, sampled_physical, ordered):
    """Algorithmic FP64 flops of one far-kernel launch (fused multiply-add = 2
    flops).  The kernel samples each unordered pair {l, m} once for both
    orientations: (M/2 + 1) angle samples of S~ and of the geometric factor g
    of K~ (both media), four even-sequence DFTs of length M at 5 K log2 K +
    15 K flops each (K = M/2: a K-point complex FFT plus pre- and
    post-processing).  A sample costs 265 flops for a pair with a node in the
    PML (complex distance, square root and reciprocal by Newton-refined
    reciprocal square roots, 1/R^3, two e^{iq} by range reduction + series,
    complex products) and 126 for a pair of physical nodes (real distance and
    reciprocal square root, two sin/cos pairs, real products).  Each ordered
    far pair then costs 60 flops per mode of the launch's chunk: K^ of both
    media from g^ and the pair's normal factor (22 each), and the scaling and
    quadrature weights of the four entries (4 each)."""
    K = M // 2
    dft = 4 * (5.0 * K * np.log2(K) + 15.0 * K)
    pml = sampled - sampled_physical
    return (sampled_physical * ((K + 1) * 126.0 + dft) + pml * ((K + 1) * 265.0 + dft) +
            ordered * chunk_modes * 60.0)


def near_counts(P):
    """Close pairs of a problem by the path they take in the close-pair modes
    kernel: (packed: two physical nodes, both media in one transform; PML: a
    node in the PML, Taylor substitution, one pass per medium; plain: Alpert
    correction pairs that are far by the criterion; PML couples: PML grid
    pairs whose mirror is a PML pair too, computed together by one CTA)."""
    _, _, f, mirror = P.near_pairs()
    plain = (f & 2) != 0
    pml = ((f & 4) != 0) & ~plain
    idx = np.arange(len(f))
    has = pml & (mirror >= 0)
    mir = np.where(has, mirror, 0)
    couples = int((has & pml[mir] & (mir > idx)).sum())
    return int((~plain & ~pml).sum()), int(pml.sum()), int(plain.sum()), couples


def near_flops_per_launch(M, chunk_modes, packed, pml, plain, couples=0):
    """Algorithmic FP64 flops of one close-pair modes launch (fused
    multiply-add = 2 flops; Taylor degree L = 5).  Per pair, (M/2 + 1) split
    samples: 169 flops for a packed pair (distance, complex square root and
    reciprocal 51, per medium sin/cos, sinc-type factors and the four split
    values 59), 473 for a PML pair (51, per medium e^{iq} 79 and the four
    products with the Taylor polynomials of cH1 / cH3: Horner of their tails
    40 + 24, the full sums from the tails 8 + 24, with their products), 295
    for a plain pair (51, per medium e^{iq} and S~, K~ 122).  Transforms: E1 = 5 K log2 K + 15 K for a length-M even DFT
    (K = M/2), E2 = 5 M log2 M + 15 M for a length-2M one.  Packed: 4 E1 + 6 E2
    (Laplace spectra, one convolution pass), PML: 8 E1 + 10 E2 (two passes),
    plain: 4 E1.  Products 14 (M + 1) and fills 4 K per pass; per output mode
    8 (packed, plain) or 24 (PML) flops.  A PML couple (a grid pair and its
    mirror, one CTA) adds to one pair's work only the mirror's double-layer
    remainder samples (30 flops per angle, both media), their 2 E1, the
    mirror's D^ spectrum and one inverse transform per pass (3 E2), one
    product per pass 8 (M + 1), and 12 flops per output mode."""
    K = M // 2
    E1 = 5.0 * K * np.log2(K) + 15.0 * K
    E2 = 5.0 * M * np.log2(M) + 15.0 * M
    S1 = K + 1
    f_packed = S1 * 169.0 + 4 * E1 + 6 * E2 + 14.0 * (M + 1) + 4.0 * K + 8.0 * chunk_modes
    f_pml = S1 * 473.0 + 8 * E1 + 10 * E2 + 2 * (14.0 * (M + 1) + 4.0 * K) + 24.0 * chunk_modes
    f_mirror = S1 * 30.0 + 2 * E1 + 3 * E2 + 2 * 8.0 * (M + 1) + 12.0 * chunk_modes
    f_plain = S1 * 295.0 + 4 * E1 + 8.0 * chunk_modes
    return packed * f_packed + (pml - couples) * f_pml + couples * f_mirror + plain * f_plain


def source_sha(name):
    import hashlib
    try:
        return hashlib.sha256(open(os.path.join(ROOT, "paper_2412_11162_gb300", "csrc", name), "rb").read()).hexdigest()
    except OSError:
        return None


def profile_traffic(path, src_name, units):
    """DRAM bytes (read + write) of one launch scaled to `units` from a
    committed ncu summary (profiles/): its 'dram_bytes_per_unit' line, valid
    while 'source_sha256' matches the kernel's source file; else None."""
    try:
        text = open(os.path.join(ROOT, "profiles", path)).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.split(":")[0].strip() in ("source_sha256", "dram_bytes_per_unit"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256") != source_sha(src_name) or "dram_bytes_per_unit" not in vals:
        return None
    return float(vals["dram_bytes_per_unit"]) * units


def fp64_peak(pk, clk, pipes):
    """Measured FP64 FMA TFLOP/s (pmlbie_selftest_peak), else derived."""
    if pipes and pipes.get("fp64_fma_tflops"):
        return pipes["fp64_fma_tflops"], "measured: FP64 FMA probe on this GPU (pmlbie_selftest_peak)"
    mhz = clk.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    return 152 * 2 * 2 * mhz * 1e6 / 1e12, "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x %.0f MHz" % mhz


def near_roofline(w, rep, pk, clk, counts, pipes=None):
    """Roofline of the close-pair modes kernel for the pairs with a PML point
    (near_modes_kernel<0>, FP64 in both paths, the longest single kernel of
    the mixed step; one launch per mode chunk): FP64-ALU bound.  achieved =
    the algorithmic FP64 flops of those pairs (near_flops_per_launch) / the
    kernel's event time; peak = the measured FP64 FMA rate."""
    M = w["M"]
    peak, note = fp64_peak(pk, clk, pipes)
    launches = max(1, rep.chunks)
    npml = counts[1]
    couples = counts[3] if len(counts) > 3 else 0
    flops = near_flops_per_launch(M, rep.chunk_modes, 0, npml, 0, couples)
    ms1 = (rep.ms_near - rep.ms_near_laplace - rep.ms_near_ff) / launches
    ach = flops / (ms1 / 1e3) / 1e12
    traffic = profile_traffic("near_modes_kernel_pml_n256_m128.md", "kernels.cu", npml)
    return {"kernel": "near_modes_kernel<0> (close pairs with a PML point: Sec. 4.3 substitution split, even DFTs, "
                      "FFT convolution with the exact Laplace modes, FP64)",
            "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": traffic, "flops_per_launch": flops, "ms_per_launch": ms1, "launches_per_step": launches,
            "pairs": npml, "pml_couples": couples,
            "algorithmic_bytes": float(npml) * (2 * M + 4 * rep.chunk_modes) * 16,
            "peak_note": note,
            "traffic_note": ("ncu dram read+write per PML pair (profiles/near_modes_kernel_pml_n256_m128.md) x pairs"
                             if traffic else "null: no ncu capture of the current kernels.cu")}


def roofline(w, rep, pk, clk, pipes=None):
    """Roofline of the far-pair kernel of the mixed path (far_kernel_ff:
    float-float sampling, transforms and block scatter), the HBM view of
    SURVEY-style stage a3: algorithmic bytes = the 4 N^2 (M/2) complex128
    entries it writes per launch, against the measured HBM copy bandwidth.
    The kernel is bounded by instruction issue on its FP32 / integer pipes
    (ncu summary in profiles/), so this fraction is low by construction."""
    M = w["M"]
    launches = max(1, rep.chunks)
    # the kernel alone (its autotuning launch): in the solve it runs beside the
    # close-pair kernels, and rep.ms_far is its span there
    alone = float(getattr(rep, "ms_far_alone", 0.0))
    ms1 = alone if alone > 0 else rep.ms_far / launches
    wbytes = 4.0 * w["N"] ** 2 * rep.chunk_modes * 16
    hbm = pk.get("hbm_gbs", 6794.1)
    ach = wbytes / (ms1 / 1e3) / 1e9
    traffic = profile_traffic("far_kernel_ff_n256_m128.md", "kernels_ff.cu", 4.0 * w["N"] ** 2 * rep.chunk_modes)
    return {"kernel": "far_kernel_ff (S~, K~ sampling of both media per unordered pair + 4 even DFTs + block scatter "
                      "of both orientations, float-float)",
            "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
            "ms_per_launch": ms1, "launches_per_step": launches, "algorithmic_bytes": wbytes,
            "time_note": ("the kernel alone: its autotuning launch of the chosen CTA size (CUDA events); in the "
                          "step it runs beside the close-pair kernels" if alone > 0 else
                          "span of the launch in the step (runs beside the close-pair kernels)"),
            "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json)",
            "traffic_note": ("ncu dram read+write per entry written (profiles/far_kernel_ff_n256_m128.md) x "
                             "4 N^2 (M/2) entries"
                             if traffic else "null: no ncu capture of the current kernels_ff.cu")}


def lu_update_roofline(w, rep, pk):
    """Roofline of the FP32 LU's tensor-core trailing update (tcu::update_kernel,
    the largest total time per step: 31 updates at N=512): HBM-bound by
    construction (a rank-32 update does 16 flops per byte of the trailing
    matrix).  Algorithmic bytes = one read and one write of the complex64
    trailing matrix per update, sum_k 2 x 8 B x (n - 32 (k + 1))^2 per mode
    (the operand images are not counted); time = the device time of the update
    launches, from event pairs recorded around them inside the captured LU
    graph (report ms_lu_update; the A' image kernel runs beside the row-swap
    kernel on a side stream, outside these pairs)."""
    N, M = w["N"], w["M"]
    n, modes = 2 * N, M // 2
    launches = int(getattr(rep, "lu_update_launches", 0))
    ms = float(getattr(rep, "ms_lu_update", 0.0))
    wbytes = modes * sum(2 * 8.0 * (n - 32 * (k + 1)) ** 2 for k in range((n + 31) // 32 - 1))
    hbm = pk.get("hbm_gbs", 6794.1)
    ach = wbytes / (ms / 1e3) / 1e9 if ms > 0 else None
    traffic = profile_traffic("tc_update_kernel_n512_64modes.md", "tc_update.cuh", wbytes)
    return {"kernel": ("tcu::update_kernel (rank-32 trailing update of the complex64 LU on tcgen05, TF32 split "
                       "operands formed once per step; persistent warp-specialised update streaming the tiles by TMA)"),
            "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm if ach else None, "traffic": traffic, "ms_per_step": ms,
            "launches_per_step": launches, "algorithmic_bytes": wbytes,
            "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json)",
            "traffic_note": ("ncu dram read+write per algorithmic byte (profiles/tc_update_kernel_n512_64modes.md)"
                             if traffic else "null: no ncu capture of the current tc_update.cuh")}


def stage_rooflines(w, rep, pk, pipes=None):
    """Per-stage rooflines of the mixed step besides the far kernel's.

    * LU (FP32, tensor-core trailing updates): algorithmic flops (8/3) n^3 per
      mode (n = 2N, complex LU), against the TF32 dense peak taken as the
      measured sustained bf16 peak x the nominal TF32/bf16 ratio 1.1/2.25; and
      its algorithmic bytes: the complex128 -> complex64 conversion (16 + 8 B
      per entry) plus one read and one write of the complex64 trailing matrix
      per 32-column panel, sum_k 2 x 8 B x (n - 32 (k + 1))^2, against the
      measured HBM copy bandwidth.  The LU time includes the conversion, the
      Frobenius norms and the diagonal-block inverses, and (mixed path) runs
      beside the right-hand sides.
    * Block writes (fused into the far kernel): 4 N^2 (M/2) complex128
      entries per step against HBM.
    """
    N, M = w["N"], w["M"]
    n, modes = 2 * N, M // 2
    lu_flops = 8.0 / 3.0 * n ** 3 * modes
    upd = sum(2 * 8.0 * (n - 32 * (k + 1)) ** 2 for k in range(n // 32))
    lu_bytes = modes * (24.0 * n * n + upd)
    tf32 = (pipes or {}).get("tf32_tcgen05_tflops") or pk.get("bf16_tflops_sustained", 1692.2) * 1.1 / 2.25
    hbm = pk.get("hbm_gbs", 6794.1)
    s_lu = rep.ms_lu / 1e3
    wr = 4.0 * N * N * modes * 16
    # the far kernel alone (its autotuning launch); rep.ms_far is its span beside the close pairs
    alone = float(getattr(rep, "ms_far_alone", 0.0))
    far_ms = alone * max(1, getattr(rep, "chunks", 1)) if alone > 0 else rep.ms_far
    s_far = far_ms / 1e3
    return {
        "lu_fp32": {"bound": "hbm", "ms": rep.ms_lu, "flops": lu_flops, "tflops": lu_flops / s_lu / 1e12,
                    "tf32_peak_tflops": tf32, "frac_tf32": lu_flops / s_lu / 1e12 / tf32,
                    "bytes": lu_bytes, "gbs": lu_bytes / s_lu / 1e9, "frac_hbm": lu_bytes / s_lu / 1e9 / hbm,
                    "note": "rank-32 trailing updates: 16 flop per byte, below the TF32 ridge; "
                            "TF32 peak measured by the tcgen05 probe (pmlbie_selftest_peak), HBM measured copy"},
        "block_writes": {"bytes": wr, "ms": far_ms, "gbs": wr / s_far / 1e9,
                         "frac_hbm": wr / s_far / 1e9 / hbm,
                         "note": "fused into the far kernel, bounded by its FP32 / integer instruction issue"},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary n1024_m512 and batched8 measurements of the default run")
    ap.add_argument("--workload", default="default", choices=sorted(WORKLOADS) + ["batched8"],
                    help="default: N=512, M=256 (the headline); 'small' (N=256, M=128) is for profiler "
                         "captures; n1024_m512 / n1536_m512 / n4096_m512: the large single and "
                         "high-frequency instances (n4096_m512 runs in mode chunks); "
                         "batched8: eight seeded instances with 64 plane waves each, one batch call per step")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = WORKLOADS.get(args.workload, WORKLOADS["default"])
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched8":
        run_batched(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
