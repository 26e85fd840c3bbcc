"""Multi-rank host logic of the independent-domain runs, on CPU gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2606_00641_gb300 import dist as vdist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0, 25.0][rank]
    cells = [1000, 3000][rank]
    rate, ms_max, total = vdist.weak_scaling_rate(ms, cells, 7)
    out[rank] = (rate, ms_max, total)
    dist.destroy_process_group()


def test_weak_scaling_rate_over_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    expect = (1000 + 3000) * 7 / (25.0e-3) / 1e9
    for r in range(world):
        rate, ms_max, total = out[r]
        assert ms_max == 25.0 and total == 4000
        assert abs(rate - expect) < 1e-12 * expect


def test_weak_scaling_rate_without_a_group_is_local():
    rate, ms, cells = vdist.weak_scaling_rate(5.0, 100, 3)
    assert (ms, cells) == (5.0, 100) and abs(rate - 100 * 3 / 5e-3 / 1e9) < 1e-18


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_domains_covers_every_domain_once_and_balances(world):
    from paper_2606_00641_gb300 import fields
    sizes = [sp["side"] ** 2 for sp in fields.batch_specs(64, 4004)]
    owned = [vdist.shard_domains(sizes, world, r) for r in range(world)]
    flat = sorted(d for o in owned for d in o)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[d] for d in o) for o in owned]
    # greedy largest-first: no rank exceeds the mean by more than the largest domain
    assert max(loads) - sum(loads) / world <= max(sizes)


def test_reference_arm_under_torchrun_prints_one_line():
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--cpu-seconds", "0.3"]
    res = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
