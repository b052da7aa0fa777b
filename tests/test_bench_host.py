"""Host-side logic of bench.py on the CPU: the max-over-ranks timing with two
gloo ranks (the multi-rank path uses it on NCCL), and the parsing of the
clock/throttle samples that decide whether a run is kept."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.reduce_max(dist, 10.0 * (rank + 1))
        out[rank] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 20.0


def test_reduce_max_without_process_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(None, 3.5) == 3.5


def test_clock_samples_are_summarised():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1400, 2070, 700, 0x8, Active, Not Active, Not Active, Not Active"]
    assert "hw_slowdown" in c.summary()["reasons"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]


def _json_lines(text):
    import json
    out = []
    for ln in text.splitlines():
        ln = ln.strip()
        if ln.startswith("{"):
            out.append(json.loads(ln))
    return out


def _check_reference_line(d, n_gpus):
    assert d["impl"] == "reference" and d["metric"] == "agent-steps/s"
    assert d["unit"] == "agent-steps/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["n_gpus"] == n_gpus and d["steps"] == 1 and d["warmup"] == 0
    assert d["vs_baseline"] is None and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["ms_per_step"] > 0 and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference: the oracle timed on the host cores, one JSON
    line with the keys the benchmark contract asks for."""
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 1)


def test_reference_arm_under_torchrun_two_ranks():
    """Launched like the multi-GPU runs (torchrun, two ranks, gloo on the host):
    rank 0 alone times the oracle and prints the line; the other rank exits 0
    without work."""
    import subprocess
    port = 30500 + os.getpid() % 1000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 2)


def test_issue_roofline(monkeypatch):
    """The issue view needs a capture of the sweep's current source: without one
    (or once the source changed) it is null, with one it divides the captured
    instruction count by the live launch time."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "SWEEP_CAPTURE", {"src": None, "dram_bytes": None, "warp_inst": None})
    assert bench.issue_roofline(0.1) is None and bench.sweep_capture() is None
    cap = {"src": bench.sweep_source_hash(), "dram_bytes": 1.0e8, "warp_inst": 2.0e8}
    monkeypatch.setattr(bench, "SWEEP_CAPTURE", cap)
    r = bench.issue_roofline(0.1)                      # 100 us per launch
    assert abs(r["achieved_ginst_s"] - 2.0e8 / 1e-4 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved_ginst_s"] / (152 * 4 * 2.07)) < 1e-12
    monkeypatch.setattr(bench, "SWEEP_CAPTURE", dict(cap, src="0" * 16))
    assert bench.issue_roofline(0.1) is None


def test_parity_leg_compares_every_cell():
    """The CPU baseline leg's parity block: the oracle's own forces rounded to
    float32 stand in for the GPU's (error at float32 rounding), one planted
    contact-count mismatch is counted, and every cell is compared."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    from paper_2105_00039_gb300 import populations as P
    n, nbar, seed = 1500, 8.0, 8
    st = P.density_cube(n, nbar, seed=seed)
    ref = O.step_sampled(st, np.arange(n), O.Params(max_disp=0.0))
    fake = np.concatenate([ref["F"].astype(np.float32),
                           ref["npairs"][:, None].astype(np.float32)], axis=1)
    fake[7, 3] += 1.0
    pool = bench.OraclePool(2)
    try:
        cells, secs, cmp = pool.step(n, nbar, seed, gpu=fake)
    finally:
        pool.close()
    err, count_bad = cmp
    assert cells == n and err.size == n and secs > 0
    assert count_bad == 1
    assert 0.0 < float(err.max()) < 1e-6
