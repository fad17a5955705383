"""Multi-rank host logic of bench.py on CPU (gloo, world size 2, 127.0.0.1):
every rank times its own independent problem, the job's time is the slowest
rank's, the throughput counts the units of all ranks, and only rank 0 prints
the JSON line.  (No GPU: the data path has no collective to test.)"""
import io
import json
import os
import socket

import pytest


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist = bench.init_dist(world, "gloo")
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, device="cpu")     # rank 1 is the slow one
    value = bench.job_value(world, 1000, ms)
    buf = io.StringIO()
    printed = bench.emit_line({"value": value, "ms_per_step": ms, "n_gpus": world}, rank, out=buf)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, "rank%d.json" % rank), "w") as f:
        json.dump({"ms": ms, "value": value, "printed": printed, "text": buf.getvalue()}, f)


def test_two_ranks_gloo(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["ms"] == r1["ms"] == 15.0                      # max over ranks
    assert abs(r0["value"] - 2 * 1000 / 0.015) < 1e-6         # both ranks' units / the job time
    assert r0["printed"] and not r1["printed"] and r1["text"] == ""
    line = json.loads(r0["text"])
    assert line["n_gpus"] == 2 and line["ms_per_step"] == 15.0


def test_single_rank_needs_no_group():
    import bench
    assert bench.init_dist(1) is None
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.job_value(1, 10, 1000.0) == 10.0


def test_stage_rooflines_arithmetic():
    """The LU stage's algorithmic counts against a direct sum: (8/3) n^3 flops
    per mode, and per mode the conversion (24 B per entry) plus one read and
    one write of the complex64 trailing matrix after each 32-column panel."""
    import types
    import bench
    w = {"N": 64, "M": 8}
    n, modes = 128, 4
    rep = types.SimpleNamespace(ms_lu=2.0, ms_far=1.0)
    r = bench.stage_rooflines(w, rep, {"hbm_gbs": 1000.0, "bf16_tflops_sustained": 2250.0})
    lu = r["lu_fp32"]
    assert abs(lu["flops"] - 8.0 / 3.0 * n ** 3 * modes) < 1.0
    trailing = 0
    for k0 in range(0, n, 32):
        m = n - k0 - 32          # order of the trailing matrix after this panel
        trailing += 2 * 8 * m * m
    assert lu["bytes"] == modes * (24 * n * n + trailing)
    assert abs(lu["tf32_peak_tflops"] - 1100.0) < 1e-9
    assert abs(lu["frac_hbm"] - lu["bytes"] / 2e-3 / 1e9 / 1000.0) < 1e-12
    assert r["block_writes"]["bytes"] == 4 * 64 * 64 * 4 * 16
