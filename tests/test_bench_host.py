"""Host-side logic of bench.py: rank aggregation over gloo (world size 2),
clock parsing, and the reference arm's JSON line on a small workload."""
import json
import math
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    got = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    dist.destroy_process_group()
    q.put((rank, got))


def test_max_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 15.0, 1: 15.0}


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_parse_clock_csv():
    sys.path.insert(0, ROOT)
    import bench
    text = ("0, 1965, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
            "0, 1875, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
            "0, 1920, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
    c = bench.parse_clock_csv(text)
    assert c["sm_mhz"] == 1920 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3
    assert bench.parse_clock_csv("") is None


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "mix10k_d32", "--steps", "2", "--warmup", "1",
                          "--cpu-sample", "4"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "impl", "cpu_baseline", "e2e", "config"):
        assert key in line
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_cost_sweep_fit_recovers_a_planted_model():
    """The %C_I(n, d) fit of the cost sweep: fastest windowed permilles made
    from a known log-linear model come back as its coefficients."""
    import bench
    rows = [{"n": n, "d": d, "best_windowed_permille": 100 + 30 * math.log2(n / 250000)
             - 40 * math.log2(d / 32)}
            for n in (250000, 500000, 1000000, 2000000) for d in (32, 128, 512)]
    fit = bench.fit_split_model(rows)
    c0, c1, c2 = fit["c"]
    assert abs(c1 - 30) < 1e-6 and abs(c2 + 40) < 1e-6
    assert abs(c0 - (100 - 30 * math.log2(250000) + 40 * math.log2(32))) < 1e-3
    assert fit["rms_permille"] < 1e-6


def test_cost_sweep_arguments():
    import bench
    a = bench.parse_args(["--cost-sweep", "--cost-grid", "1000,2000:16,32"])
    assert a.cost_sweep and a.cost_grid == "1000,2000:16,32"
