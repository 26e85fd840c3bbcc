"""Multi-rank host logic on CPU gloo ranks: the independent-domain runs, and the
halo exchange of a domain decomposed into slabs."""
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
           "--gpus", "2", "--steps", "2", "--warmup", "1"]
    res = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


# ---------------------------------------------------------------------------
# Slab decomposition of one domain (the multi-GPU design): each rank advances a
# z-slab with the oracle's step, wrapping periodically inside the slab, and the
# one exchange per step swaps what wrapped: the +z populations that left the top
# layer (they landed in the local bottom layer) go to the upper neighbour, the
# -z ones that left the bottom layer go to the lower neighbour -- one population
# per lattice per face cell each way.  The result must equal the single-domain
# oracle bit for bit.
# ---------------------------------------------------------------------------

def _slab_main(rank, world, port, out, nz, steps):
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2606_00641_gb300 import fields
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shape = (nz, 6, 10)
    f0 = fields.ideal_fields(shape, 91, mach=1.0, cfl=0.2)
    tau = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]
    full = oracle.ideal_init(f0.Q, f0.gamma)
    zl = nz // world
    z0 = rank * zl
    f = np.ascontiguousarray(full[:, :, z0:z0 + zl])
    up, down = (rank + 1) % world, (rank - 1) % world
    sent = 0
    for _ in range(steps):
        f = oracle.ideal_step(f, f0.gamma, tau)
        send_up = torch.from_numpy(np.ascontiguousarray(f[:, 5, 0]))        # +z out of my top layer
        send_down = torch.from_numpy(np.ascontiguousarray(f[:, 6, zl - 1]))  # -z out of my bottom layer
        recv_low, recv_high = torch.empty_like(send_up), torch.empty_like(send_down)
        reqs = [dist.isend(send_up, up, tag=5), dist.isend(send_down, down, tag=6),
                dist.irecv(recv_low, down, tag=5), dist.irecv(recv_high, up, tag=6)]
        for r in reqs:
            r.wait()
        f[:, 5, 0] = recv_low.numpy()
        f[:, 6, zl - 1] = recv_high.numpy()
        sent += send_up.numel() + send_down.numel()
    ref = full
    for _ in range(steps):
        ref = oracle.ideal_step(ref, f0.gamma, tau)
    out[rank] = (bool(np.array_equal(f, ref[:, :, z0:z0 + zl])), sent)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,nz", [(2, 8), (3, 12)])
def test_slab_halo_exchange_reproduces_the_single_domain_bit_for_bit(world, nz):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    steps = 6
    mp.start_processes(_slab_main, args=(world, _free_port(), out, nz, steps), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        same, sent = out[r]
        assert same, r
        assert sent == steps * 2 * 8 * 6 * 10  # one population per lattice per face cell, each way


# ---------------------------------------------------------------------------
# The library's slab exchange (paper_2606_00641_gb300.slabs.SlabExchange) on
# gloo ranks: every rank holds its slab in the AA in-place layout of the GPU
# kernels, steps it with the kernels' addressing (emulated with the oracle's own
# single-cell collision, periodic inside the slab), and after every step packs
# the face planes the library packs (lo: first layer, +z slot; hi: last layer,
# -z slot), routes them with SlabExchange and unpacks what it receives.  Each
# slab's logical populations, read with the periodic addressing inside the slab
# as the moments kernels read them, must equal the single-domain oracle bit for
# bit at both parities.
# ---------------------------------------------------------------------------

_C7 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]  # (x, y, z)
_OPP7 = [0, 2, 1, 4, 3, 6, 5]
_TAU = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]


def _shift(a, c):
    """result[x] = a[x - c] over the last three axes (z, y, x), periodic."""
    import numpy as np
    return np.roll(a, shift=(c[2], c[1], c[0]), axis=(-3, -2, -1))


def _aa_step(A, parity, gamma):
    """One step of the kernels' AA addressing on A[lattice, slot, z, y, x]."""
    import numpy as np

    import oracle

    def collide(F):
        out = F.copy()
        for z in range(F.shape[2]):
            for y in range(F.shape[3]):
                for x in range(F.shape[4]):
                    out[:, :, z, y, x] = oracle.ideal_collide_cell(3, gamma, _TAU, F[:, :, z, y, x])
        return out
    if parity == 0:
        return collide(A)[:, _OPP7]
    F = np.stack([_shift(A[:, _OPP7[i]], _C7[i]) for i in range(7)], axis=1)
    P = collide(F)
    return np.stack([_shift(P[:, i], _C7[i]) for i in range(7)], axis=1)


def _logical(A, parity):
    import numpy as np
    if parity == 0:
        return A
    return np.stack([_shift(A[:, _OPP7[i]], _C7[i]) for i in range(7)], axis=1)


def _exchange_main(rank, world, port, out, shape, steps):
    import numpy as np
    import torch.distributed as dist

    import oracle
    from paper_2606_00641_gb300 import fields, slabs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    f0 = fields.ideal_fields(shape, 93, mach=1.0, cfl=0.2)
    full = oracle.ideal_init(f0.Q, f0.gamma)
    z0, z1 = slabs.split_layers(shape[0], world)[rank]
    state = {"A": np.ascontiguousarray(full[:, :, z0:z1])}
    plane = shape[1] * shape[2]

    def pack(lo, hi):
        lo.numpy().view(np.float64)[:] = state["A"][:, 5, 0].ravel()
        hi.numpy().view(np.float64)[:] = state["A"][:, 6, -1].ravel()

    def unpack(lo, hi):
        state["A"][:, 5, 0] = lo.numpy().view(np.float64).reshape(8, shape[1], shape[2])
        state["A"][:, 6, -1] = hi.numpy().view(np.float64).reshape(8, shape[1], shape[2])

    ex = slabs.SlabExchange(pack, unpack, 8 * plane * 8)
    assert (ex.world, ex.rank) == (world, rank)
    ref = full
    results = []
    for s in range(steps):
        state["A"] = _aa_step(state["A"], s & 1, f0.gamma)
        ex.exchange(s + 1)
        ref = oracle.ideal_step(ref, f0.gamma, _TAU)
        got = _logical(state["A"], (s + 1) & 1)
        results.append(bool(np.array_equal(got, ref[:, :, z0:z1])))
    sums = ex.allreduce_sums(oracle.ideal_moments(_logical(state["A"], steps & 1)).reshape(8, -1).sum(1))
    ref_sums = oracle.ideal_moments(ref).reshape(8, -1).sum(1)
    out[rank] = (results, ex.bytes_sent, float(np.abs(sums - ref_sums).max() / np.abs(ref_sums).max()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,shape", [(2, (8, 4, 5)), (3, (10, 4, 5)), (2, (2, 3, 4))])
def test_slab_exchange_routes_the_aa_halo_bit_for_bit(world, shape):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    steps = 5
    mp.start_processes(_exchange_main, args=(world, _free_port(), out, shape, steps), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        results, sent, sums_err = out[r]
        assert all(results), (r, results)  # every step, both parities
        assert sent == steps * 2 * 8 * shape[1] * shape[2] * 8  # two face messages per step
        assert sums_err < 1e-14


def test_route_pairs_every_send_with_the_receiving_slab():
    from paper_2606_00641_gb300 import slabs
    for world in (2, 3, 5):
        for count in (1, 2):
            for r in range(world):
                hi_to, lo_to, hi_from, lo_from = slabs.route(r, world, count)
                # the slab a message goes to expects it from this one
                assert slabs.route(hi_to, world, count)[2] == r
                assert slabs.route(lo_to, world, count)[3] == r
            # after an even step hi goes up; after an odd step it comes back down
            assert slabs.route(0, world, 1)[0] == 1 % world and slabs.route(0, world, 2)[0] == world - 1


def test_split_layers_covers_the_axis():
    from paper_2606_00641_gb300 import slabs
    assert slabs.split_layers(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert slabs.split_layers(4, 4) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    with pytest.raises(ValueError):
        slabs.split_layers(3, 4)


def _avg_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_2606_00641_gb300 import closure
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = torch.arange(6, dtype=torch.float32) * (rank + 1) + rank
    loss = closure.average_gradients(g, 0.5 + rank, None)
    out[rank] = (g.tolist(), loss)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_data_parallel_gradients_are_averaged_over_the_ranks(world):
    # every rank ends with the mean gradient and the mean loss (closure.dp_train_step
    # then applies one and the same Adam step on every rank)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_avg_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    want = [sum(i * (r + 1) + r for r in range(world)) / world for i in range(6)]
    want_loss = sum(0.5 + r for r in range(world)) / world
    for r in range(world):
        g, loss = out[r]
        assert max(abs(a - b) for a, b in zip(g, want)) < 1e-6
        assert abs(loss - want_loss) < 1e-12


def test_data_parallel_average_without_a_group_is_the_identity():
    import torch
    from paper_2606_00641_gb300 import closure
    g = torch.tensor([1.0, -2.0, 3.5])
    assert closure.average_gradients(g, 0.25) == 0.25
    assert g.tolist() == [1.0, -2.0, 3.5]
