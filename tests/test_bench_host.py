"""Host-side logic of bench.py, on the CPU: the max-over-ranks timing of a
multi-process (replicas) run over a world of two gloo ranks, the autotuner
report parsing behind the roofline's kernel name, the convolution FLOP
count, and the JSON line of the reference (oracle) arm."""
import importlib.util
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = load_bench()
    # each rank timed a different duration; the job's time is the slowest
    got = bench.reduce_max(10.0 + 5.0 * rank, dist, "cpu")
    q.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res == {0: 15.0, 1: 15.0}


def test_reduce_max_single_process():
    bench = load_bench()
    assert bench.reduce_max(3.5, None, "cpu") == 3.5


def test_chosen_config_parses_autotune_report():
    bench = load_bench()
    rep = ("policy 0 T=1 R=8 WY=4 S=4 minb=3: 0.7849 ms/sweep\n"
           "policy 0 T=1 R=4 WY=8 S=5 minb=2: 0.7020 ms/sweep\n"
           "policy 0 T=1 R=8 WY=8 S=4 minb=1: 0.6938 ms/sweep\n"
           "policy 0 T=2 R=2 WY=4 S=6 minb=3: 0.6268 ms/sweep\n"
           "chosen: T=2\n")
    assert bench.chosen_config(rep, 1, "PolResident") == "jacobi_tb<PolResident,T=1,R=8,WY=8,S=4>"
    assert bench.chosen_config(rep, 2, "PolResident") == "jacobi_tb<PolResident,T=2,R=2,WY=4,S=6>"
    # the index is the position among that pass length's lines (registry order)
    assert bench.chosen_config(rep, 1, "PolResident", with_index=True)[1] == 2
    assert bench.chosen_config(rep, 2, "PolResident", with_index=True)[1] == 0
    assert bench.chosen_config("", 1, "PolResident", with_index=True)[1] == 0
    # the measured-traffic table covers exactly the compiled one-sweep shapes
    # of the resident fixed-point policy
    import re
    src = open(os.path.join(ROOT, "paper_2310_01882_b300", "csrc", "sweep_f64.cu")).read()
    block = src[src.index("res1[] = {"):src.index("};", src.index("res1[] = {"))]
    shapes = {f"jacobi_tb<PolResident,T=1,R={r},WY={wy},S={st}>"
              for r, wy, st in re.findall(r"TbCfg<PolResident, 1, (\d+), (\d+), (\d+), \d+>", block)}
    assert len(shapes) >= 2
    assert set(bench.MEASURED_TRAFFIC) == shapes


def test_wsnet_flops_matches_layer_count():
    """2 * 27 * voxels * cin * cout summed over the U-Net's 3x3x3 layers,
    counted from the oracle's own layer list."""
    from oracle import net as onet
    bench = load_bench()
    ch = [16, 32, 64, 64]
    p = onet.init_params(ch, seed=0)
    n = 32
    total = 0
    for name in onet.layer_names(len(ch)):
        w = p[name + ".w"]
        level = int(name[3])
        total += 2 * 27 * (n >> level) ** 3 * w.shape[3] * w.shape[4]
    assert bench.wsnet_flops(n, ch) == total


def test_reference_arm_line():
    """--impl reference prints one JSON line with the same metric and config
    as the GPU arm, the oracle as its CPU baseline, and host-only e2e."""
    bench = load_bench()
    bench.N = 24
    args = type("A", (), {"gpus": 1, "steps": 2, "warmup": 1})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(args, 0)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.HEADLINE_METRIC
    assert line["config"] == bench.headline_config(1)
    assert line["unit"] == "GLUP/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # other ranks print nothing
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(args, 1)
    assert buf.getvalue() == ""
