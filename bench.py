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
WORKLOADS = {"default": WORKLOAD, "small": dict(WORKLOAD, N=256, M=128)}
METRIC = "modal kernel entries/s and solve s/problem, mixed vs FP64 GPU at 1e-6 rel err"
UNIT = "entries/s"


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
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.stop = threading.Event()

    def _run(self):
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
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
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    w = WORKLOAD
    kw = dict(a1=w["a1"], T=w["T"], S=w["S"], bump_h=w["bump_h"])
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
        e0.record(stream)
        for _ in range(args.steps):
            reps.append(step(B.PMLBIE_MIXED))
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()
    mixed_out = {k: v.clone() for k, v in outs.items()}

    # plain FP64 GPU path on the same problem (1 warm + 2 timed)
    step(B.PMLBIE_FP64)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    fp64_reps = [step(B.PMLBIE_FP64) for _ in range(2)]
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1) / 2
    rel = {k: (torch.linalg.vector_norm(mixed_out[k] - outs[k]) / torch.linalg.vector_norm(outs[k])).item()
           for k in outs}

    # end to end through the public API with host buffers: create (host tables,
    # first-call upload) + solve + copy of the outputs to pinned host memory
    pinned = [torch.empty(shape, dtype=torch.complex128, pin_memory=True).numpy() for _ in range(4)]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Q = Problem(w["k1"], w["k2"], w["N"], w["M"], **kw)
        B.pmlbie_solve_host(Q.handle, B.PMLBIE_MIXED, polar, *pinned, stream=stream)
        Q.close()
    torch.cuda.synchronize()
    e2e_ms = 1e3 * (time.perf_counter() - t0) / e2e_steps
    H = P.nodes()
    ng, nc = P.near_count()
    # bytes uploaded by the first device call: node tables, pair classes, close-pair table, stencils
    h2d = (w["N"] * (5 * 8 + 3 * 16 + 3 * 8 + 4 + 16) + w["N"] ** 2 + (ng + nc) * 144 + nc * 4 * (1 + 2 * 10)
           + (w["M"] // 2 + 1 + w["M"]) * 16 + 8)
    d2h = 4 * int(np.prod(shape)) * 16

    last = reps[-1]
    epp = entries_per_problem(w)
    value = world * epp / (ms / 1e3)
    pk = peaks()
    # dominant kernel: the largest stage of the mixed step by device time
    stages = {"far_kernel": last.ms_far, "near_kernels": last.ms_near, "assemble": last.ms_assemble,
              "lu_fp32": last.ms_lu, "solve_refine": last.ms_solve}
    dom = max(stages, key=stages.get)
    roof = roofline(dom, stages[dom], w, last, pk)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128 kernels / c64 LU / c128 refinement", "data": "synthetic",
        "config": {"workload": "two-layer bump, N=%d M=%d (%d modes), k1=4pi k2=6pi, PML a1=2.5 T=1 S=3, "
                               "1 plane wave at 30 deg, mixed precision" % (w["N"], w["M"], w["M"] // 2),
                   "parallelism": "independent problems per GPU" if world > 1 else "1 GPU",
                   "l2": "working set > L2 (129 MB): %d MB of per-mode matrices rebuilt every step" %
                         int(((w["M"] // 2) * (2 * w["N"]) ** 2 * 24) / 1e6)},
        "solve_s_per_problem": ms / 1e3,
        "kernel_entries_per_s": epp / ((last.ms_far + last.ms_near + last.ms_assemble) / 1e3),
        "stages_ms": {k: round(v, 4) for k, v in stages.items()},
        "refine_iters": last.refine_iters, "refine_residual": last.residual,
        "fp64_gpu": {"ms_per_step": ms64, "value": world * epp / (ms64 / 1e3), "stages_ms": {
            "far_kernel": fp64_reps[-1].ms_far, "near_kernels": fp64_reps[-1].ms_near,
            "assemble": fp64_reps[-1].ms_assemble, "lu_fp64": fp64_reps[-1].ms_lu,
            "solve": fp64_reps[-1].ms_solve}},
        "speedup_mixed_vs_fp64": ms64 / ms,
        "mixed_vs_fp64_rel_err": rel,
        "near_pairs": {"grid": ng, "alpert": nc},
        "gpu_launches": int(sum(r.launches for r in reps)),
        "roofline": roof,
        "clocks": clk.summary(),
        "e2e": {"value": world * epp / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "note": "per step: create (host setup) + solve_host to pinned buffers + destroy"},
    }
    if rank == 0 and not args.no_cpu_baseline:
        e, t = oracle_sample(w, rows=48)
        line["cpu_baseline"] = {"value": e / t, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                "sample": "modal kernels of 48 target rows x all 512 sources + their Alpert "
                                          "points, 128 modes, 4 kernels (FP64 numpy oracle), %.1f s" % t}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def roofline(name, ms, w, rep, pk):
    """Roofline entry of the dominant stage; algorithmic work per launch as
    stated in the design notes."""
    N, M = w["N"], w["M"]
    nm, n2 = M // 2, 2 * N
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    if name == "lu_fp32":
        flops = nm * (8.0 / 3.0) * n2 ** 3          # complex LU: 8/3 n^3 real flops per mode
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # FP32 FMA pipe, derived (TFLOP/s)
        ach = flops / (ms / 1e3) / 1e12
        return {"kernel": "batched LU (FP32, CUDA cores)", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_note": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock (derived, not measured)"}
    if name in ("far_kernel", "near_kernels", "assemble"):
        # FP64 pipe: 152 SMs x 2 FP64 FMA/clk (GB300) x 2 flop x clock
        peak = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12
        if name == "far_kernel":
            samples = N * N * (M // 2 + 1)
            flops = samples * FAR_FLOPS_PER_SAMPLE
            ach = flops / (ms / 1e3) / 1e12
            return {"kernel": "far_kernel (sample + FFT + scatter, FP64)", "bound": "alu", "achieved": ach,
                    "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                    "peak_note": "FP64 pipe 2 FMA/clk/SM (1.25 TF/s nominal), derived"}
        return {"kernel": name, "bound": "alu", "achieved": None, "peak": peak, "unit": "TFLOP/s",
                "frac": None, "traffic": None}
    byts = nm * n2 * n2 * 16.0
    ach = byts / (ms / 1e3) / 1e9
    peak = pk.get("hbm_gbs", 6800.0)
    return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": None}


# FP64 flops the far kernel spends per (pair, angle) sample, counted from the
# formula with transcendental functions at their operation counts (see the
# design notes): distance and reciprocals ~40, two complex exponentials with
# range reduction ~2 x 45, kernels ~30, FFT share 4 x 5 log2(M) ~ 160 at M=256.
FAR_FLOPS_PER_SAMPLE = 320.0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="default", choices=sorted(WORKLOADS),
                    help="'small' (N=256, M=128) is for profiler captures only")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
