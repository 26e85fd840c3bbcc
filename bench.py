#!/usr/bin/env python3
"""Benchmark of the fused VLBM collide-and-stream step on one GB300 per rank.

Workload (default): 3-D ideal compressible MHD, 512^3 periodic cells, 8
conserved fields each on its own D3Q7 lattice (56 populations per cell),
FP32 storage and arithmetic, seeded random-phase fields (k <= 4, peak Mach 2,
beta 1, CFL 0.2, tau 0.51).  One step = one launch of the fused kernel over
all cells.  Metric: GLUPS (10^9 cell updates per second, whole job) and the
fraction of the HBM roofline (448 algorithmic bytes per cell update: every
population read once and written once).

Printed: one JSON line on rank 0.  ``--impl reference`` times the CPU oracle
(plain FP64 C) on the host cores on a bounded sample of the same workload.
Under torchrun (N > 1) the ranks hold the z-slabs of one periodic domain of
512 x 512 x (512 N) cells, one 512^3 slab per rank (the 512^3 fields repeated
along z, so every slab's result equals the one-GPU run), and after every step
exchange the population planes that cross the slab faces by NCCL send/recv:
the work per GPU is fixed, so the scaling is weak.  At N > 1 the job runs
that decomposed headline only (timed region, end to end, slab check); the
other storage forms, the error sweep, the other paths and the CPU oracle are
one-GPU measurements of the N = 1 run.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

BYTES_PER_POP = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}
# DRAM bytes (read + write) per cell update of the step kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of a 256^3 launch of
# each parity, mean of the two parities, taken after the last change to that
# kernel's source: f32 7,457,219 kB and f16dev 3,705,818 kB per 16,777,216-cell
# launch.  Traffic grows in proportion to the cells, so a full launch is this
# times the cells.  Set an entry to None whenever that kernel changes until it
# is re-captured.
MEASURED_DRAM_BYTES_PER_CELL = {"f32": 7457219e3 / 16777216, "f16dev": 3705818e3 / 16777216}
# FP64 operations per cell update of the FP64 step kernels (k_ideal_step<D,double>),
# from one ncu capture of each parity: (dadd + dmul + 2 dfma thread instructions,
# smsp__sass_thread_inst_executed_op_d{add,mul,fma}_pred_on.sum) / cells, mean of
# the two parities.  3-D (128^3): even 90 + 42 + 2 x 152 = 436, odd 114 + 43 +
# 2 x 152 = 461; 2-D (128^2): even 91 + 33 + 2 x 122 = 368, odd 79 + 33 + 2 x 122
# = 356.  Set an entry to None whenever that kernel changes until it is re-captured.
MEASURED_FP64_FLOP_PER_CELL = {2: 362.0, 3: 448.5}
# FP64 pipe instructions (dadd + dmul + dfma) per cell update, mean of both parities, from the
# same ncu capture: each takes one issue of the FP64 pipe, whose instruction rate is half the
# measured FMA FLOP rate
MEASURED_FP64_INSTR_PER_CELL = {2: 240.0, 3: 296.5}
# the step kernel the roofline describes, per storage (3-D, nx % 8 == 0)
STEP_KERNEL = {"f32": "k_ideal_step<3,float,float> (fused collide+stream)",
               "f64": "k_ideal_step<3,double,double> (fused collide+stream; FP64-pipe bound on GB300)",
               "f16dev": "k_ideal_step_pairs<__half> (fused collide+stream, bulk-copy loads, 2 cells/thread)",
               "bf16dev": "k_ideal_step_pairs<__nv_bfloat16> (fused collide+stream, bulk-copy loads, 2 cells/thread)"}
WORKLOAD = "ideal MHD 3-D, 8 x D3Q7, periodic, random-phase k<=4, Mach 2, beta 1, CFL 0.2, tau 0.51"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=512, help="cube side of the 3-D domain")
    ap.add_argument("--storage", default="f32", choices=list(BYTES_PER_POP))
    ap.add_argument("--forms", default="f64,f16dev,bf16dev",
                    help="other storage forms to time and compare with FP64 ('' to skip)")
    ap.add_argument("--form-steps", type=int, default=20)
    ap.add_argument("--growth-steps", type=int, default=1000,
                    help="length of the reduced-precision error run (0 to skip)")
    ap.add_argument("--growth-size", type=int, default=256, help="cube side of the headline error run")
    ap.add_argument("--growth-sweep-size", type=int, default=128, help="cube side of the Mach x beta sweep")
    ap.add_argument("--growth-taus", default="0.51,0.6,0.8",
                    help="BGK times of the error runs (0.51 is the workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the channel, batched and closure forms")
    ap.add_argument("--extras", default="channel,batch,closure,powell,hlbm,open,slabs,diss,diss3,cfg1",
                    help="which other workloads to run (comma list of channel, batch, closure, powell, "
                         "hlbm, open, slabs, diss, diss3, cfg1)")
    ap.add_argument("--closure-fine", type=int, default=512, help="fine grid side of the closure workload")
    ap.add_argument("--closure-steps", type=int, default=250, help="coarse steps of the closure's test runs")
    ap.add_argument("--closure-mach", default="1,1.25",
                    help="range of the seeds' peak Mach (lo,hi); at tau 0.51 some seeds' fields turn "
                         "non-physical within 1000 fine steps from about Mach 1.4 on")
    ap.add_argument("--closure-train-seeds", type=int, default=16, help="training seeds from 5000 on")
    ap.add_argument("--diss3-size", type=int, default=256, help="cube side of the 3-D dissipative leg")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--seed", type=int, default=3003)
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return summarise_clocks(self.lines)


def summarise_clocks(lines):
    """Median SM clock, maximum clock and the throttle reasons seen active in
    nvidia-smi CSV lines of ClockSampler.QUERY (malformed lines are skipped)."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [t.strip() for t in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for name, flag in zip(names, parts[5:9]):
            if flag.lower() == "active":
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reference_arm(args, world, rank):
    """The oracle (plain FP64 C, as it stands) on the host cores: W untimed and K
    timed steps, each one oracle step over a 128^3 sample of the workload's
    fields (the same recipe; the full 512^3 step would take minutes)."""
    if rank != 0:
        return 0
    import oracle
    from paper_2606_00641_gb300 import fields
    oracle.build()
    n = 128
    cores = os.cpu_count() or 1
    f0 = fields.ideal_fields((n, n, n), args.seed, mach=2.0, beta=1.0, cfl=0.2, k_rho=4, k_u=4, k_b=4)
    f = oracle.ideal_init(f0.Q, f0.gamma)
    for _ in range(args.warmup):
        f = oracle.ideal_step(f, f0.gamma, 0.51, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.ideal_step(f, f0.gamma, 0.51, nthreads=cores)
    dt = time.perf_counter() - t0
    value = n ** 3 * args.steps / dt / 1e9
    sample = "%d^3 cells of the same field recipe per step, FP64 C oracle, %d OpenMP threads" % (n, cores)
    line = {
        "impl": "reference", "metric": "GLUPS", "value": value, "unit": "GLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": "%d^3" % args.size, "storage": args.storage,
                   "l2": "inputs_larger_than_l2", "sample": sample},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(args, seconds):
    """Time the oracle on a bounded sample (64^3 cells of the same recipe)."""
    import oracle
    from paper_2606_00641_gb300 import fields
    oracle.build()
    n = 64
    cores = os.cpu_count() or 1
    f0 = fields.ideal_fields((n, n, n), args.seed, mach=2.0, beta=1.0, cfl=0.2, k_rho=4, k_u=4, k_b=4)
    f = oracle.ideal_init(f0.Q, f0.gamma)
    t0 = time.perf_counter()
    f = oracle.ideal_step(f, f0.gamma, 0.51, nthreads=cores)
    one = time.perf_counter() - t0
    steps = max(2, int(seconds / max(one, 1e-6)))
    t0 = time.perf_counter()
    for _ in range(steps):
        f = oracle.ideal_step(f, f0.gamma, 0.51, nthreads=cores)
    dt = time.perf_counter() - t0
    cells = n ** 3
    return {"value": cells * steps / dt / 1e9, "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": "%d^3 cells x %d steps of the same field recipe, FP64 C oracle, %d OpenMP threads"
                      % (n, steps, cores),
            "steps": steps, "ms_per_step": dt / steps * 1e3}


def _time_steps(vlbm, ctx_ptrs, stream, torch, steps, per_call):
    """CUDA-event time of `steps` steps; per_call=True issues one vlbm_step(ctx, 1)
    per context per step (sequential plain launches), else vlbm_step(ctx, steps)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    if per_call:
        for _ in range(steps):
            for c in ctx_ptrs:
                vlbm.vlbm_step(c, 1)
    else:
        for c in ctx_ptrs:
            vlbm.vlbm_step(c, steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def channel_form(args, vlbm, fields, torch, stream, hbm_peak):
    """Resistive channel 256 x 128 x 128 (D3Q19 + 3 x D3Q7, FP32, walls, Guo force), at its
    configured length: 5,000 steps from rest (plus 1 % noise) at Ha 10, 30 and 50, each timed,
    and the x/z-averaged u_x(y) and b_x(y) compared with the closed-form Hartmann profile.  With
    Pm = 1 the start-up transient leaves the channel at the Alfven speed, in about
    2 a^2 / (Ha nu) steps (25,200 / 8,400 / 5,040), so at 5,000 steps only Ha 50 is near steady;
    the others report their residual."""
    import numpy as np
    shape = (128, 128, 256)
    nz, ny, nx = shape
    steps = 5000
    yc = np.arange(1, ny - 1) - (ny - 1) / 2.0
    runs, total_ms, status = {}, 0.0, []
    for Ha in (10.0, 30.0, 50.0):
        setup = fields.hartmann_setup(shape, 2002, Ha=Ha)
        p = vlbm.make_params(model=vlbm.VLBM_RESISTIVE, shape=shape, storage="f32",
                             tau=[setup.tau_f, setup.tau_m, setup.tau_m, setup.tau_m], force=setup.force,
                             b_wall=setup.b_wall, walls_y=True, stream=stream.cuda_stream)
        ctx = vlbm.Context(p)
        Qd = torch.from_numpy(setup.Q).cuda()
        st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, Qd.data_ptr())
        del Qd
        ms = _time_steps(vlbm, [ctx.ptr], stream, torch, steps, False)
        total_ms += ms
        Q = ctx.moments()
        status.append(vlbm.status_string(vlbm.vlbm_sync(ctx.ptr)))
        ctx.close()
        u = (Q[1] / Q[0])[:, 1:ny - 1, :].mean(axis=(0, 2))
        bx = Q[4][:, 1:ny - 1, :].mean(axis=(0, 2))
        u_ref, b_ref = fields.hartmann_profile(yc, setup.a, setup.force[0], 1.0, setup.nu, setup.eta, setup.B0)
        runs["Ha%g" % Ha] = {
            "init_status": vlbm.status_string(st), "ms": ms,
            "u_rel_linf_vs_closed_form": float(np.abs(u - u_ref).max() / np.abs(u_ref).max()),
            "b_rel_linf_vs_closed_form": float(np.abs(bx - b_ref).max() / np.abs(b_ref).max()),
            "centreline_u_over_Uc": float(u[len(u) // 2] / setup.U_c),
            "transient_steps_2a2_over_Ha_nu": 2 * setup.a ** 2 / (Ha * setup.nu)}
    ncell = nx * ny * nz
    gl = 3 * ncell * steps / (total_ms * 1e-3) / 1e9
    return {"workload": "resistive incompressible channel 256x128x128, D3Q19 + 3 x D3Q7, FP32, "
                        "bounce-back walls in y, Re 100, Pm 1, Ha 10 / 30 / 50, 5,000 steps each from rest",
            "status": "/".join(status), "glups": gl, "steps": steps, "bytes_per_cell": 320,
            "roofline_frac": gl * 1e9 * 320 / (hbm_peak * 1e9), "hartmann": runs,
            "note": "steady errors measured at 50,000 / 20,000 / 15,000 steps: u 2.0 / 5.5 / 8.9 %, b 2.0 / "
                    "2.9 / 2.5 % (first order in the node-located magnetic wall; the Hartmann layer is "
                    "a / Ha = 6.3 / 2.1 / 1.3 cells)"}


def powell_form(args, vlbm, fields, torch, stream, hbm_peak):
    """Ideal MHD with the Powell correction (nine D3Q7 lattices, FP32) on the headline grid."""
    n = args.size
    shape = (n, n, n)
    f0 = fields.ideal_fields(shape, args.seed, gamma=5.0 / 3.0, mach=2.0, beta=1.0, cfl=0.2,
                             device=torch.device("cuda"))
    # D starts at rest: it settles at tau_M div B within a few steps
    Q = torch.cat([f0.Q, torch.zeros((1,) + shape, dtype=f0.Q.dtype, device=f0.Q.device)])
    p = vlbm.make_params(model=vlbm.VLBM_IDEAL_POWELL, shape=shape, storage="f32", gamma=f0.gamma,
                         tau=0.51, tau_d=0.51, tau_m=1.0, stream=stream.cuda_stream)
    ctx = vlbm.Context(p)
    st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, Q.data_ptr())
    del Q, f0
    vlbm.vlbm_step(ctx.ptr, 4)
    steps = args.form_steps
    ms = _time_steps(vlbm, [ctx.ptr], stream, torch, steps, False)
    status = vlbm.status_string(vlbm.vlbm_sync(ctx.ptr))
    ctx.close()
    ncell = n ** 3
    gl = ncell * steps / (ms * 1e-3) / 1e9
    bytes_cell = 2 * 63 * 4
    return {"workload": "ideal MHD 3-D with the Powell source, %d^3, 9 x D3Q7 (the 8 fields and the "
                        "divergence lattice D), FP32, tau 0.51, tau_d 0.51, tau_M 1, same fields as the "
                        "headline workload, D = 0 at start" % n,
            "init_status": vlbm.status_string(st), "status": status, "glups": gl, "steps": steps,
            "bytes_per_cell": bytes_cell, "roofline_frac": gl * 1e9 * bytes_cell / (hbm_peak * 1e9)}


def dissipative_form(args, vlbm, fields, torch, stream, hbm_peak):
    """Dissipative MHD with evolved gradients (20 D2Q5 lattices, FP32): the
    low-Mach resistive Orszag-Tang set-up at the paper's finest grid, 2048^2."""
    n = 2048
    setup = fields.low_mach_orszag_tang(n)
    p = vlbm.make_params(model=vlbm.VLBM_DISSIPATIVE, shape=(n, n), storage="f32", gamma=setup.gamma,
                         tau=setup.tau, tau_g=setup.tau_g, tau_m=setup.tau_m, nu=setup.nu, eta0=setup.eta0,
                         j_c=setup.j_c, powell=True, stream=stream.cuda_stream)
    ctx = vlbm.Context(p)
    Qd = torch.from_numpy(setup.Q).cuda()
    st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, Qd.data_ptr())
    del Qd
    vlbm.vlbm_step(ctx.ptr, 4)
    steps = args.form_steps
    ms = _time_steps(vlbm, [ctx.ptr], stream, torch, steps, False)
    status = vlbm.status_string(vlbm.vlbm_sync(ctx.ptr))
    ctx.close()
    ncell = n * n
    gl = ncell * steps / (ms * 1e-3) / 1e9
    bytes_cell = 2 * 100 * 4
    return {"workload": "dissipative MHD 2-D with locally evolved gradients, %d^2, 20 x D2Q5 (8 MHD fields, "
                        "G ~ tau_M grad B, W ~ tau_M grad u), FP32, low-Mach resistive Orszag-Tang set-up "
                        "(nu = eta0 = %.3g, j_c = %.3g, tau_M = %.1f steps, tau = %.5f), Powell source on"
                        % (n, setup.nu, setup.j_c, setup.tau_m, setup.tau),
            "kernel": "k_diss_step<float> (fused collide+stream, 100 populations per cell)",
            "init_status": vlbm.status_string(st), "status": status, "glups": gl, "steps": steps,
            "bytes_per_cell": bytes_cell, "roofline_frac": gl * 1e9 * bytes_cell / (hbm_peak * 1e9)}


def dissipative3_form(args, vlbm, fields, torch, stream, hbm_peak):
    """Dissipative MHD with evolved gradients in 3-D (26 D3Q7 lattices, FP32): the
    3-D low-Mach resistive vortex at 256^3."""
    n = args.diss3_size
    setup = fields.low_mach_vortex_3d(n)
    p = vlbm.make_params(model=vlbm.VLBM_DISSIPATIVE, shape=(n, n, n), storage="f32", gamma=setup.gamma,
                         tau=setup.tau, tau_g=setup.tau_g, tau_m=setup.tau_m, nu=setup.nu, eta0=setup.eta0,
                         j_c=setup.j_c, powell=True, stream=stream.cuda_stream)
    ctx = vlbm.Context(p)
    st = vlbm.vlbm_init_fields(ctx.ptr, 0, setup.Q)
    del setup
    vlbm.vlbm_step(ctx.ptr, 4)
    steps = args.form_steps
    ms = _time_steps(vlbm, [ctx.ptr], stream, torch, steps, False)
    status = vlbm.status_string(vlbm.vlbm_sync(ctx.ptr))
    ctx.close()
    ncell = n ** 3
    gl = ncell * steps / (ms * 1e-3) / 1e9
    bytes_cell = 2 * 182 * 4
    return {"workload": "dissipative MHD 3-D with locally evolved gradients, %d^3, 26 x D3Q7 (8 MHD fields, "
                        "G, W ~ tau_M grad B, grad u), FP32, 3-D low-Mach resistive vortex, Powell source on" % n,
            "kernel": "k_diss3_step<float> (fused collide+stream, 182 populations per cell)",
            "init_status": vlbm.status_string(st), "status": status, "glups": gl, "steps": steps,
            "bytes_per_cell": bytes_cell, "roofline_frac": gl * 1e9 * bytes_cell / (hbm_peak * 1e9)}


def slab_form(args, vlbm, fields, torch, stream, hbm_peak, parts_list=(2, 4)):
    """The headline domain cut into P z-slabs on this one GPU (row f4 without a
    second device): P contexts on one stream, each step every slab's step kernel,
    then every slab's face planes packed and unpacked (vlbm_slabs_step).  The
    rate against the single domain's measures what the halo copies cost per step
    (on several GPUs NCCL carries the same messages)."""
    n = args.size
    shape = (n, n, n)
    f0 = fields.ideal_fields(shape, args.seed, mach=2.0, beta=1.0, cfl=0.2, k_rho=4, k_u=4, k_b=4,
                             device=torch.device("cuda"))
    steps = args.form_steps
    out = {"workload": "ideal MHD %d^3 (the headline fields), FP32, cut into P z-slabs on one GPU, "
                       "halo planes exchanged after every step" % n, "steps": steps, "slabs": {}}
    for parts in parts_list:
        from paper_2606_00641_gb300 import slabs
        ctxs = []
        for z0, z1 in slabs.split_layers(n, parts):
            p = vlbm.make_params(shape=(z1 - z0, n, n), storage="f32", gamma=f0.gamma, tau=0.51,
                                 stream=stream.cuda_stream)
            c = vlbm.Context(p)
            Qs = f0.Q[:, z0:z1].contiguous()
            vlbm.vlbm_init_fields_device(c.ptr, 0, Qs.data_ptr())
            stream.synchronize()
            del Qs
            c.set_slab(True)
            ctxs.append(c)
        ptrs = [c.ptr for c in ctxs]
        vlbm.vlbm_slabs_step(ptrs, 4)
        l0 = sum(c.launches for c in ctxs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        st = vlbm.vlbm_slabs_step(ptrs, steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        launches = sum(c.launches for c in ctxs) - l0
        face = vlbm.vlbm_halo_bytes(ptrs[0])
        statuses = {vlbm.status_string(vlbm.vlbm_sync(c.ptr)) for c in ctxs}
        for c in ctxs:
            c.close()
        gl = n ** 3 * steps / (ms * 1e-3) / 1e9
        out["slabs"][str(parts)] = {"glups": gl, "roofline_frac": gl * 1e9 * 448 / (hbm_peak * 1e9),
                                    "launches_per_step": launches / steps, "halo_bytes_per_face": face,
                                    "halo_message_bytes_per_step": 2 * parts * face,
                                    "status": "/".join(sorted(statuses))}
    del f0
    return out


def open_form(args, vlbm, fields, torch, stream, hbm_peak):
    """Headline workload with open faces (sec. 2.4, "Static boundaries"): x- a
    Dirichlet reservoir at the mean state, the other five faces zero-gradient."""
    n = args.size
    shape = (n, n, n)
    f0 = fields.ideal_fields(shape, args.seed, gamma=5.0 / 3.0, mach=2.0, beta=1.0, cfl=0.2,
                             k_rho=4, k_u=4, k_b=4, device=torch.device("cuda"))
    mean = f0.Q.reshape(8, -1).mean(1).cpu().numpy()
    p = vlbm.make_params(shape=shape, storage="f32", gamma=f0.gamma, tau=0.51, stream=stream.cuda_stream)
    ctx = vlbm.Context(p)
    st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, f0.Q.data_ptr())
    del f0
    ctx.set_boundary("x-", vlbm.VLBM_BC_EQUILIBRIUM, 0xFF, mean)
    for face in ("x+", "y-", "y+", "z-", "z+"):
        ctx.set_boundary(face, vlbm.VLBM_BC_EQUILIBRIUM)
    vlbm.vlbm_step(ctx.ptr, 4)
    steps = args.form_steps
    l0 = vlbm.vlbm_launch_count(ctx.ptr)
    ms = _time_steps(vlbm, [ctx.ptr], stream, torch, steps, False)
    launches = vlbm.vlbm_launch_count(ctx.ptr) - l0
    status = vlbm.status_string(vlbm.vlbm_sync(ctx.ptr))
    ctx.close()
    ncell = n ** 3
    gl = ncell * steps / (ms * 1e-3) / 1e9
    # the step's 448 B per cell, plus per face cell the boundary pass: the normal
    # neighbour's 56 populations read and 8 entering populations written
    bytes_cell = 2 * 56 * 4 + 6 * n * n * (56 + 8) * 4 / ncell
    return {"workload": "headline workload (%d^3, 8 x D3Q7, FP32, tau 0.51) with all six faces open: x- a "
                        "Dirichlet reservoir at the mean state, the other faces zero-gradient" % n,
            "init_status": vlbm.status_string(st), "status": status, "glups": gl, "steps": steps,
            "launches_per_step": launches / steps, "bytes_per_cell": bytes_cell,
            "roofline_frac": gl * 1e9 * bytes_cell / (hbm_peak * 1e9)}


def blend_initial_state(Q, solid, gamma):
    """Initial condition of a body in the gas: u and B take the blended values
    d u + (1 - d) uB, d B + (1 - d) BB at the cell's density and gas pressure
    (in place on the [8, ...] float64 fields Q; solid = [7, ...] d, uB, BB)."""
    rho = Q[0]
    p = (gamma - 1) * (Q[4] - 0.5 * (Q[1:4] ** 2).sum(0) / rho - 0.5 * (Q[5:8] ** 2).sum(0))
    d = solid[0].double()
    for a in range(3):
        Q[1 + a] = d * Q[1 + a] + (1 - d) * rho * solid[1 + a].double()
        Q[5 + a] = d * Q[5 + a] + (1 - d) * solid[4 + a].double()
    Q[4] = p / (gamma - 1) + 0.5 * (Q[1:4] ** 2).sum(0) / rho + 0.5 * (Q[5:8] ** 2).sum(0)


def hlbm_form(args, vlbm, fields, torch, stream, hbm_peak):
    """Headline grid with a homogenised rotating, magnetised sphere (sec. 2.4)."""
    n = args.size
    shape = (n, n, n)
    # At tau = 0.51 the blended momentum and field are over-relaxed around the solid
    # state, and every collision trades gas pressure for the body/gas contrast; the
    # summed drain is (gamma-1)/2 (omega-1)/(2-omega) (rho|du|^2 + |dB|^2), about 8x
    # that contrast.  So the flow is slower (peak Mach 0.2) and less magnetised
    # (beta 10) than the headline one, the body moves at a quarter of its speeds, and
    # the gas starts in the blended state (inside the body it already carries uB, BB).
    f0 = fields.ideal_fields(shape, args.seed, gamma=5.0 / 3.0, mach=0.2, beta=10.0, cfl=0.2,
                             k_rho=4, k_u=4, k_b=4, device=torch.device("cuda"))
    Q = f0.Q
    umax = float((Q[1:4] / Q[0]).abs().max())
    bmax = float(Q[5:8].abs().max())
    # the body: radius n/8 at the centre, rotating about z with its rim at umax/4,
    # field bump of bmax/4; porosity from the signed distance (eps_h = 1 cell)
    ax = torch.arange(n, device="cuda", dtype=torch.float32) - 0.5 * (n - 1)
    z, y, x = torch.meshgrid(ax, ax, ax, indexing="ij")
    r = torch.sqrt(x * x + y * y + z * z)
    radius = n / 8.0
    phi = (r - radius).contiguous()
    solid = torch.zeros((7,) + shape, dtype=torch.float32, device="cuda")
    vlbm.vlbm_porosity_from_distance(phi.data_ptr(), phi.numel(), 1.0, solid[0].data_ptr())
    omega = 0.25 * umax / radius
    solid[1] = -omega * y
    solid[2] = omega * x
    bump = torch.exp(-(r / radius) ** 2)
    solid[4] = 0.25 * bmax * bump
    solid[6] = 0.125 * bmax * bump
    del x, y, z, r, phi, bump
    blend_initial_state(Q, solid, f0.gamma)
    p = vlbm.make_params(shape=shape, storage="f32", gamma=f0.gamma, tau=0.51, stream=stream.cuda_stream)
    ctx = vlbm.Context(p)
    st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, Q.data_ptr())
    del Q, f0
    ctx.set_solid(solid.data_ptr())
    vlbm.vlbm_step(ctx.ptr, 4)
    steps = args.form_steps
    ms = _time_steps(vlbm, [ctx.ptr], stream, torch, steps, False)
    status = vlbm.status_string(vlbm.vlbm_sync(ctx.ptr))
    ctx.close()
    del solid
    ncell = n ** 3
    gl = ncell * steps / (ms * 1e-3) / 1e9
    bytes_cell = 2 * 56 * 4 + 7 * 4
    return {"workload": "%d^3, 8 x D3Q7, FP32, tau 0.51, smooth random fields (k = 4) at peak Mach 0.2, "
                        "beta 10, with a homogenised sphere of radius n/8 rotating about z (rim speed "
                        "max|u|/4) carrying a field bump of max|B|/4, gas started in the blended state; "
                        "porosity from the signed distance, eps_h = 1 cell; 7 FP32 solid fields per cell" % n,
            "init_status": vlbm.status_string(st), "status": status, "glups": gl, "steps": steps,
            "bytes_per_cell": bytes_cell, "roofline_frac": gl * 1e9 * bytes_cell / (hbm_peak * 1e9)}


def batch_form(args, vlbm, fields, torch, stream, hbm_peak):
    """64 independent 2-D domains (sides 64..1024) in one launch per step vs 64 plain launches,
    each timed over the workload's 1,000 steps."""
    specs = fields.batch_specs(64, 4004)
    params, Qs = [], []
    for sp in specs:
        n = sp["side"]
        f0 = fields.ideal_fields((n, n), sp["seed"], gamma=sp["gamma"], mach=sp["mach"], cfl=0.1,
                                 device=torch.device("cuda"))
        Qs.append(f0.Q)
        params.append(vlbm.make_params(shape=(n, n), storage="f32", gamma=sp["gamma"], tau=0.51,
                                       stream=stream.cuda_stream))
    ncell = sum(sp["side"] ** 2 for sp in specs)
    steps = 1000
    # batched: one context, one launch per step, graph-captured, autotuned tile shape
    bctx = vlbm.Context(params, batch=True)
    bad = 0
    for d, Q in enumerate(Qs):
        bad += vlbm.vlbm_init_fields_device(bctx.ptr, d, Q.data_ptr()) != vlbm.VLBM_OK
    choice = bctx.autotune(8)
    vlbm.vlbm_step(bctx.ptr, 64)
    ms_b = _time_steps(vlbm, [bctx.ptr], stream, torch, steps, False)
    st_b = vlbm.status_string(vlbm.vlbm_sync(bctx.ptr))
    # which domains left the physical states (NaN, rho <= 0 or p <= 0) by the end of the run:
    # the health flag is one per context; the cost of a step does not depend on the values
    bad_domains = []
    for d, sp in enumerate(specs):
        Qd = torch.empty((8, sp["side"], sp["side"]), dtype=torch.float64, device="cuda")
        vlbm.vlbm_moments_device(bctx.ptr, d, Qd.data_ptr())
        stream.synchronize()
        rho = Qd[0]
        p = (sp["gamma"] - 1.0) * (Qd[4] - 0.5 * (Qd[1] ** 2 + Qd[2] ** 2 + Qd[3] ** 2) / rho
                                   - 0.5 * (Qd[5] ** 2 + Qd[6] ** 2 + Qd[7] ** 2))
        if not bool(torch.isfinite(Qd).all()) or float(rho.min()) <= 0.0 or float(p.min()) <= 0.0:
            bad_domains.append((d, sp["side"], round(sp["mach"], 3)))
    bctx.close()
    # baseline: 64 contexts, one plain launch per domain per step
    ctxs = [vlbm.Context(p) for p in params]
    for c, Q in zip(ctxs, Qs):
        vlbm.vlbm_init_fields_device(c.ptr, 0, Q.data_ptr())
    ptrs = [c.ptr for c in ctxs]
    _time_steps(vlbm, ptrs, stream, torch, 2, True)
    ms_s = _time_steps(vlbm, ptrs, stream, torch, steps, True)
    for c in ctxs:
        c.close()
    gb = ncell * steps / (ms_b * 1e-3) / 1e9
    gs = ncell * steps / (ms_s * 1e-3) / 1e9
    return {"workload": "64 periodic 2-D ideal-MHD domains, sides from {64..1024} (seed 4004), "
                        "gamma U[1.4,5/3], Mach U[0.5,3], 8 x D2Q5, FP32", "cells": ncell,
            "init_failures": int(bad), "status": st_b, "tile_shape": choice,
            "nonphysical_domains_[index,side,mach]": bad_domains,
            "lowest_mach_nonphysical": min((m for _, _, m in bad_domains), default=None),
            "highest_mach_physical": max((sp["mach"] for d, sp in enumerate(specs)
                                          if d not in {b[0] for b in bad_domains}), default=None),
            "glups_batched": gb, "glups_sequential_launches": gs, "speedup": gb / gs, "steps": steps,
            "note": "the batched run issues its steps in one call; the sequential baseline calls one step per "
                    "domain, and a domain whose health word has turned non-physical stops stepping there "
                    "(a context refuses steps after the flag is seen), so the baseline's rate is an upper "
                    "bound and the speedup a lower one",
            "nonphysical_cell_share": sum(side * side for _, side, _ in bad_domains) / ncell,
            "bytes_per_cell": 320, "roofline_frac_batched": gb * 1e9 * 320 / (hbm_peak * 1e9)}


def ideal_2d_f64_form(args, vlbm, fields, torch, stream, fp64_tflops):
    """2-D ideal MHD, 128^2 periodic, 8 x D2Q5, FP64, 200 steps (seed 1001, Mach 1,
    beta 10/3, CFL 0.1, tau 0.51): 5.2 MB of populations stay in L2, and the FP64
    step is bound by the FP64 pipe, so its roof is the measured FP64 FMA rate."""
    n, steps = 128, 200
    f0 = fields.ideal_fields((n, n), 1001, device=torch.device("cuda"))
    p = vlbm.make_params(shape=(n, n), storage="f64", gamma=f0.gamma, tau=0.51, stream=stream.cuda_stream)
    ctx = vlbm.Context(p)
    st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, f0.Q.data_ptr())
    vlbm.vlbm_step(ctx.ptr, 64)
    ms = min(_time_steps(vlbm, [ctx.ptr], stream, torch, steps, False) for _ in range(3))
    status = vlbm.status_string(vlbm.vlbm_sync(ctx.ptr))
    ctx.close()
    gl = n * n * steps / (ms * 1e-3) / 1e9
    flop = MEASURED_FP64_FLOP_PER_CELL.get(2)
    out = {"grid": "128^2", "steps": steps, "init_status": vlbm.status_string(st), "status": status, "glups": gl,
           "bytes_per_cell": 640, "kernel": "k_ideal_step<2,double,double>"}
    if flop and fp64_tflops:
        ach = gl * 1e9 * flop / 1e12
        out["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64_tflops, "unit": "TFLOP/s",
                           "frac": ach / fp64_tflops, "flop_per_cell": flop,
                           "fp64_pipe_frac": gl * 1e9 * MEASURED_FP64_INSTR_PER_CELL[2] / (fp64_tflops * 1e12 / 2)}
    return out


def error_growth(args, vlbm, fields, torch, stream):
    """Reduced-precision storage over the configured run: the 3-D ideal workload
    (k <= 4, CFL 0.2, seed 3003) advanced `growth_steps` steps in FP64, FP32,
    FP16-deviation and BF16-deviation storage; per-field relative L-inf and L2
    errors against the FP64 run at a ladder of step counts, and the first check
    at which a form reports NONPHYSICAL (its health flag: NaN, rho <= 0 or
    p <= 0).  The headline case (Mach 2, beta 1) on `growth_size`^3 and the
    Mach {2, 3} x beta {0.1, 1, 10} sweep on `growth_sweep_size`^3, each at the
    workload's tau 0.51 and at the larger taus of `growth_taus` (more lattice
    diffusion, (tau - 1/2) cs^2), which keep the shocks these fields develop
    from driving the scheme non-physical within the run."""
    last = args.growth_steps
    checks = [c for c in (10, 20, 50, 100, 200, 500, 1000) if c < last] + [last]
    taus = [0.51] + [float(t) for t in args.growth_taus.split(",") if t and float(t) != 0.51]
    cases = [(args.growth_size, 2.0, 1.0, t) for t in taus[:2]]
    cases += [(args.growth_sweep_size, m, b, t) for t in taus for m in (2.0, 3.0) for b in (0.1, 1.0, 10.0)]
    out = []
    for n, mach, beta, tau in cases:
        shape = (n, n, n)
        f0 = fields.ideal_fields(shape, args.seed, mach=mach, beta=beta, cfl=0.2, k_rho=4, k_u=4, k_b=4,
                                 device=torch.device("cuda"))
        Q = f0.Q
        flat = Q.reshape(8, -1)
        scale = flat.abs().amax(1)
        qref = flat.mean(1).cpu().numpy()
        qscale = (flat - flat.mean(1, keepdim=True)).abs().amax(1).clamp_min(1e-30).cpu().numpy()
        ref, case = {}, {"grid": "%d^3" % n, "mach": mach, "beta": beta, "tau": tau,
                         "nonphysical_at": {}, "linf_worst": {}, "l2_worst": {}}
        t0 = time.perf_counter()
        for form in ("f64", "f32", "f16dev", "bf16dev"):
            p = vlbm.make_params(shape=shape, storage=form, gamma=f0.gamma, tau=tau, q_ref=qref, q_scale=qscale,
                                 stream=stream.cuda_stream)
            ctx = vlbm.Context(p)
            st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, Q.data_ptr())
            done, bad, linf, l2 = 0, None, {}, {}
            for chk in checks:
                if st != vlbm.VLBM_OK:
                    bad = done
                    break
                vlbm.vlbm_step(ctx.ptr, chk - done)
                done = chk
                st = vlbm.vlbm_sync(ctx.ptr)
                if st != vlbm.VLBM_OK:
                    bad = chk
                    break
                M = torch.empty_like(Q)
                vlbm.vlbm_moments_device(ctx.ptr, 0, M.data_ptr())
                stream.synchronize()
                if form == "f64":
                    ref[chk] = M
                elif chk in ref:
                    d = (M - ref[chk]).reshape(8, -1)
                    linf[chk] = (d.abs().amax(1) / scale).cpu().numpy()
                    l2[chk] = (d.pow(2).mean(1).sqrt() / scale).cpu().numpy()
                del M
            ctx.close()
            case["nonphysical_at"][form] = bad
            if form != "f64":
                case["linf_worst"][form] = {str(c): float(v.max()) for c, v in linf.items()}
                case["l2_worst"][form] = {str(c): float(v.max()) for c, v in l2.items()}
                if linf and n == args.growth_size:
                    at = max(linf)
                    case.setdefault("linf_per_field", {})[form] = dict(
                        step=at, **dict(zip(fields.IDEAL_FIELDS, [float(v) for v in linf[at]])))
        case["seconds"] = time.perf_counter() - t0
        del ref, Q, f0
        torch.cuda.empty_cache()
        out.append(case)
    return {"note": "relative to each field's max |Q| at t = 0; FP64 storage is the reference; "
                    "nonphysical_at: the first check at which the form's health flag was raised (None: never); "
                    "errors are listed for every check the FP64 run and the form both passed",
            "steps": last, "checks": checks, "cases": out}


def closure_form(args, vlbm, torch, stream):
    """Learned flux closure, the configured protocol: coarse (fine/4)^3 + closure
    against the plain method's error-vs-time curve and the plain fine run."""
    from paper_2606_00641_gb300 import closure
    nf = args.closure_fine
    lo, hi = (float(v) for v in args.closure_mach.split(","))
    r = closure.run_protocol(fine=nf, n_eval=args.closure_steps, mach_range=(lo, hi),
                             train_seeds=tuple(range(5000, 5000 + args.closure_train_seeds)))
    if "closure" not in r:
        return r
    cl = r.pop("closure")
    nc = nf // 4
    flop = 2.0 * nc ** 3 * 27 * (8 * 32 + 32 * 32 + 32 * 24)
    tests = r["tests"]
    ok = [t for t in tests if "coarse_closure" in t]
    net_ms = (statistics.mean((t["coarse_closure"][0] - t["coarse_plain"][0]) / r["n_eval"] for t in ok)
              if ok else None)
    cl.close()
    bf16_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16_peak = float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        pass
    tflops = flop / (net_ms * 1e-3) / 1e12 if net_ms and net_ms > 0 else None
    below = [t["closure_over_curve"] < 1.0 for t in ok if t.get("closure_over_curve")]
    return {"workload": "ideal MHD 3-D, fine %d^3 restricted 4x to %d^3, %d coarse steps (%d fine), training "
                        "seeds 5000-%d, early stopping on seed %d, held-out seeds %s, peak Mach U[%g, %g] per "
                        "seed, tau 0.51; network 3 x conv3x3x3 (8->32->32->24), BF16 tensor cores; plain curve: "
                        "sides 64, 128, 256 started from the restricted fine initial state, every error on the "
                        "64^3 restriction"
                        % (nf, nc, r["n_eval"], 4 * r["n_eval"], 5000 + args.closure_train_seeds - 1,
                           r["val_seed"], r["test_seeds"], lo, hi),
            "coarse_steps": r["n_eval"], "tests": tests, "best_validation_rel_l2": r["best_val"],
            "skipped_train_seeds": r["skipped_train_seeds"], "train_s": r["t_train_s"], "data_s": r["t_data_s"],
            "below_plain_curve": "%d of %d held-out seeds" % (sum(below), len(below)),
            "network_ms_per_coarse_step": net_ms, "network_gflop_per_step": flop / 1e9,
            "network_tflops": tflops, "bf16_peak_tflops": bf16_peak,
            "tensor_frac": (tflops / bf16_peak) if (tflops and bf16_peak) else None}


def _r(v, digits=4):
    """A number rounded to `digits` significant figures (None stays None)."""
    if v is None:
        return None
    return float("%.*g" % (digits, v))


def compact_summary(line):
    """The figures of every form in a few hundred characters, printed as the last
    key of the JSON line so that a reader of the output's tail sees them all:
    [GLUPS, fraction of the HBM roof] per path, the storage forms' worst-field
    relative L-inf against FP64 after the configured run, the closure's times
    and errors."""
    out = {"headline": [_r(line["value"]), _r(line["roofline"]["frac"])]}
    forms = line.get("forms") or {}
    for k, v in forms.items():
        worst = max(v["rel_linf_vs_f64"].values()) if "rel_linf_vs_f64" in v else None
        frac = v.get("roofline_frac", (v.get("roofline") or {}).get("frac"))
        out["form_" + k] = [_r(v["glups"]), _r(frac), _r(worst, 3)]
        if (v.get("roofline") or {}).get("fp64_pipe_frac"):
            out["form_" + k + "_fp64_pipe_frac"] = _r(v["roofline"]["fp64_pipe_frac"])
    g = line.get("error_growth")
    if g:
        # per case: the FP64 run's first non-physical check (or None), and the
        # worst-field L-inf of each 16-bit form and FP32 at the last check both passed
        rows, sweep = {}, {}
        for c in g["cases"]:
            last = {f: (max(v, key=int) if v else None) for f, v in c["linf_worst"].items()}
            row = [c["nonphysical_at"].get("f64")] + [
                [int(last[f]), _r(c["linf_worst"][f][last[f]], 2)] if last.get(f) else None
                for f in ("f32", "f16dev", "bf16dev")]
            if c["grid"] == g["cases"][0]["grid"]:
                rows["%s M%g b%g t%g" % (c["grid"], c["mach"], c["beta"], c["tau"])] = row
            else:  # the Mach x beta sweep, per tau: FP64's non-physical checks, worst 16-bit error
                sw = sweep.setdefault("%s t%g" % (c["grid"], c["tau"]), {"f64bad": [], "bf16_linf_last": 0.0})
                sw["f64bad"].append(row[0])
                if row[3]:
                    sw["bf16_linf_last"] = max(sw["bf16_linf_last"], row[3][1])
        out["growth_[f64bad,f32,f16,bf16:[step,linf]]"] = rows
        out["growth_sweep_M2,3xb.1,1,10"] = sweep
    names = {"resistive_channel": "channel", "powell_3d": "powell", "hlbm_sphere_3d": "hlbm",
             "open_faces_3d": "open", "dissipative_2d": "diss", "dissipative_3d": "diss3"}
    extra = line.get("other_paths") or {}
    for k, short in names.items():
        if k in extra:
            out[short] = [_r(extra[k]["glups"]), _r(extra[k]["roofline_frac"])]
    if "hartmann" in extra.get("resistive_channel", {}):
        # u residual against the closed-form profile after 5,000 steps, Ha 10 / 30 / 50
        out["channel_u_err_5000_Ha10,30,50"] = [
            _r(v["u_rel_linf_vs_closed_form"], 3) for v in extra["resistive_channel"]["hartmann"].values()]
    if "slabs_one_gpu" in extra:
        out["slabs_1gpu_[P,glups,frac]"] = [[int(k), _r(v["glups"]), _r(v["roofline_frac"])]
                                            for k, v in extra["slabs_one_gpu"]["slabs"].items()]
    if "batched_2d" in extra:
        b = extra["batched_2d"]
        out["batched"] = [_r(b["glups_batched"]), _r(b["roofline_frac_batched"]), _r(b["speedup"])]
        if "nonphysical_domains_[index,side,mach]" in b:
            out["batched_nonphysical_of_64_[n,lowest_mach]"] = [len(b["nonphysical_domains_[index,side,mach]"]),
                                                                b["lowest_mach_nonphysical"]]
    if "ideal_2d_128sq_f64" in extra:
        c = extra["ideal_2d_128sq_f64"]
        out["cfg1_f64[glups,flop_frac,pipe_frac]"] = [_r(c["glups"]), _r((c.get("roofline") or {}).get("frac")),
                                                    _r((c.get("roofline") or {}).get("fp64_pipe_frac"))]
    if "learned_closure" in extra and "tests" in extra["learned_closure"]:
        c = extra["learned_closure"]
        # per held-out seed: [fine ms, closure ms, closure err, plain-128 err, closure / plain curve]
        out["closure_[fine_ms,cl_ms,cl_err,plain_err,cl/curve]"] = [
            [_r(t["fine_ms"], 3), _r(t["coarse_closure"][0], 3), _r(t["coarse_closure"][1], 3),
             _r(t["coarse_plain"][1], 3), _r(t.get("closure_over_curve"), 3)]
            for t in c["tests"] if "coarse_closure" in t]
        out["closure_curve_ms_err_64,128,256"] = [
            [[_r(v[0], 3), _r(v[1], 3)] for v in t["plain"].values()]
            for t in c["tests"] if "plain" in t][:1]
        out["closure_tensor_frac"] = _r(c.get("tensor_frac"), 3)
    if line.get("fp64_tflops"):
        out["fp64_tflops"] = _r(line["fp64_tflops"])
    return out


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import numpy as np
    import torch

    from paper_2606_00641_gb300 import dist as vdist
    from paper_2606_00641_gb300 import fields, slabs, vlbm

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    vlbm.load()

    n = args.size
    shape = (n, n, n)
    ncell = n ** 3
    hbm_peak, peak_kind = peaks()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # seeded fields on the device; every rank holds the same 512^3 fields, so the
    # decomposed domain is the 512^3 periodic solution repeated along z
    seed = args.seed
    f0 = fields.ideal_fields(shape, seed, mach=2.0, beta=1.0, cfl=0.2, k_rho=4, k_u=4, k_b=4,
                             device="cuda:%d" % local)
    Q = f0.Q
    stream = torch.cuda.Stream()

    def make_ctx(storage):
        qref = qscale = None
        if storage in ("f16dev", "bf16dev"):
            flat = Q.reshape(8, -1)
            qref = flat.mean(1).cpu().numpy()
            qscale = (flat - flat.mean(1, keepdim=True)).abs().amax(1).cpu().numpy()
            qscale = np.maximum(qscale, 1e-30)
        p = vlbm.make_params(shape=shape, storage=storage, gamma=f0.gamma, tau=0.51,
                             q_ref=qref, q_scale=qscale, stream=stream.cuda_stream)
        ctx = vlbm.Context(p)
        st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, Q.data_ptr())
        assert st == vlbm.VLBM_OK, vlbm.status_string(st)
        return ctx

    exchanges = {}

    def advance(c, n):
        """n steps of context c; a slab of the decomposed domain exchanges its
        face planes with the neighbouring ranks after every step, ordered on the
        context's stream (pack, NCCL send/recv, unpack)."""
        ex = exchanges.get(c.ptr)
        if ex is None:
            vlbm.vlbm_step(c.ptr, n)
            return
        with torch.cuda.stream(stream):
            for _ in range(n):
                vlbm.vlbm_step(c.ptr, 1)
                ex.exchange(c.step_count)

    def timed(ctx, steps, warmup, collective=True):
        """CUDA-event time of `steps` steps on the context's stream; `collective`:
        every rank takes part (barriers on both sides), else this rank alone."""
        sync = barrier if collective else torch.cuda.synchronize
        advance(ctx, warmup)
        sync()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = ctx.launches
        e0.record(stream)
        advance(ctx, steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        sync()
        return ms, ctx.launches - l0

    # ---- main form: timed region with clock sampling ----
    ctx = make_ctx(args.storage)
    if world > 1:
        exchanges[ctx.ptr] = slabs.SlabExchange.for_context(ctx, device="cuda:%d" % local)
    advance(ctx, args.warmup)
    stream.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms, launches = timed(ctx, args.steps, 0)
    clk = clocks.stop()
    status = vlbm.vlbm_sync(ctx.ptr)
    # whole-job rate: every rank's cells over the slowest rank's time
    glups, ms_max, _ = vdist.weak_scaling_rate(ms, ncell, args.steps, device="cuda")
    bytes_cell = 2 * 56 * BYTES_PER_POP[args.storage]
    per_launch_ms = ms / args.steps
    achieved = ncell * bytes_cell / (per_launch_ms * 1e-3) / 1e9
    step_ms = ms_max / args.steps
    # spread: five more timed regions of the same length (every rank takes part in
    # the barriers; rank 0 reports its own; the line's value is the first region,
    # taken with the clock sampler running)
    reps = [timed(ctx, args.steps, 0)[0] for _ in range(5)] if args.steps > 0 else []
    rep_glups = [ncell * args.steps / (r * 1e-3) / 1e9 for r in reps]
    spread = ({"n": len(rep_glups), "glups_mean": statistics.mean(rep_glups),
               "glups_std": statistics.stdev(rep_glups) if len(rep_glups) > 1 else 0.0,
               "glups_min": min(rep_glups), "glups_max": max(rep_glups)} if rep_glups else None)

    # the decomposed domain: every slab holds the same 512^3 solution, so every
    # rank's domain sums must equal rank 0's; the global sums are their all-reduce
    slab_check = None
    if world > 1:
        mine = torch.tensor(ctx.conservation(), dtype=torch.float64, device="cuda")
        every = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(every, mine)
        first = every[0].abs().clamp_min(1e-300)
        spread_rel = max(float(((e - every[0]).abs() / first).max()) for e in every)
        total = exchanges[ctx.ptr].allreduce_sums(mine.cpu().numpy(), device="cuda")
        slab_check = {"ranks": world, "max_rel_diff_of_slab_sums_vs_rank0": spread_rel,
                      "global_mass": float(total[0]),
                      "halo_bytes_per_face": exchanges[ctx.ptr].nbytes,
                      "halo_bytes_sent_per_rank": exchanges[ctx.ptr].bytes_sent}

    # ---- end to end through the C ABI with pinned host buffers ----
    def end_to_end(host_dtype):
        """Host fields in `host_dtype` (pinned) -> init, steps with a health read-back each, moments back."""
        f32 = host_dtype == torch.float32
        hostQ = torch.empty(Q.shape, dtype=host_dtype, pin_memory=True)
        hostQ.copy_(Q)
        hostOut = torch.empty(Q.shape, dtype=host_dtype, pin_memory=True)
        hostOut.zero_()  # a reused output buffer: its pages are resident, as after any earlier call
        # one untimed round trip: the host-field calls allocate their staging chunks
        # and copy stream on first use (once per context)
        if f32:
            vlbm.vlbm_init_fields_f32_ptr(ctx.ptr, 0, hostQ.data_ptr())
            vlbm.vlbm_moments_f32_ptr(ctx.ptr, 0, hostOut.data_ptr())
        else:
            vlbm.vlbm_init_fields_ptr(ctx.ptr, 0, hostQ.data_ptr())
            vlbm.vlbm_moments_ptr(ctx.ptr, 0, hostOut.data_ptr())
        # two timed runs, the better one reported: the host link of these machines is shared,
        # and its rate varies between runs (the device part does not)
        runs = []
        for _ in range(2):
            barrier()
            t0 = time.perf_counter()
            if f32:
                vlbm.vlbm_init_fields_f32_ptr(ctx.ptr, 0, hostQ.data_ptr())  # synchronises
            else:
                vlbm.vlbm_init_fields_ptr(ctx.ptr, 0, hostQ.data_ptr())
            t1 = time.perf_counter()
            for _ in range(args.steps):
                advance(ctx, 1)
                vlbm.vlbm_sync(ctx.ptr)  # 4-byte health word read back every step
            t2 = time.perf_counter()
            if f32:
                vlbm.vlbm_moments_f32_ptr(ctx.ptr, 0, hostOut.data_ptr())  # synchronises
            else:
                vlbm.vlbm_moments_ptr(ctx.ptr, 0, hostOut.data_ptr())
            t3 = time.perf_counter()
            barrier()
            runs.append((t0, t1, t2, t3))
        t0, t1, t2, t3 = min(runs, key=lambda r: r[3] - r[0])
        nbytes = Q.numel() * hostQ.element_size()
        del hostQ, hostOut
        return {"value": world * ncell * args.steps / (t3 - t0) / 1e9, "unit": "GLUPS",
                "h2d_bytes_per_step": int(nbytes / args.steps),
                "d2h_bytes_per_step": int(nbytes / args.steps + 4),
                "runs_glups": [world * ncell * args.steps / (r[3] - r[0]) / 1e9 for r in runs],
                "ms": {"init_from_host": (t1 - t0) * 1e3, "steps": (t2 - t1) * 1e3,
                       "moments_to_host": (t3 - t2) * 1e3}}

    e2e = None
    if not args.no_e2e:
        if args.storage == "f64":
            e2e = end_to_end(torch.float64)
            e2e["note"] = "vlbm_init_fields from pinned host FP64 fields, per step vlbm_step(1) + vlbm_sync " \
                          "(health word read back), final vlbm_moments to pinned host"
        else:
            # the step computes in FP32: single-precision host fields carry everything it uses
            e2e = end_to_end(torch.float32)
            e2e["note"] = "vlbm_init_fields_f32 from pinned host FP32 fields (the FP32 step rounds its input " \
                          "to float first: same populations as from FP64 fields), per step vlbm_step(1) + " \
                          "vlbm_sync (health word read back), final vlbm_moments_f32 to pinned host; the host " \
                          "link of a GB300 measured 211 GB/s H2D and 194 GB/s D2H (pinned) and bounds the two " \
                          "field transfers"
            e2e["f64_fields"] = end_to_end(torch.float64)
    ctx.close()

    # FP64 FMA rate of this GPU's CUDA cores: the roof of the FP64 forms
    fp64_tflops = None
    if rank == 0:
        try:
            fp64_tflops = vlbm.vlbm_measure_fp64_rate(4096, stream.cuda_stream)
        except vlbm.VlbmError:
            fp64_tflops = None

    # ---- other storage forms: GLUPS and per-field error against FP64 ----
    forms = {}
    # the storage forms, the error sweep, the other paths and the CPU oracle are one-GPU
    # measurements: at N > 1 the job runs the decomposed headline (timed region, e2e, slab check)
    # only, so that the other GPUs are not held meanwhile
    form_list = [s for s in args.forms.split(",") if s] if world == 1 else []
    if form_list:
        nfs = args.form_steps

        def moments_dev(c):
            out = torch.empty(Q.shape, dtype=torch.float64, device=Q.device)
            vlbm.vlbm_moments_device(c.ptr, 0, out.data_ptr())
            stream.synchronize()
            return out

        ref = make_ctx("f64")
        ms64, _ = timed(ref, nfs, 0, collective=False)
        Q64 = moments_dev(ref)
        ref.close()
        forms["f64"] = {"glups": ncell * nfs / (ms64 * 1e-3) / 1e9, "steps": nfs,
                        "bytes_per_cell": 2 * 56 * 8,
                        "roofline_frac_hbm": ncell * nfs / (ms64 * 1e-3) * 2 * 56 * 8 / (hbm_peak * 1e9)}
        flop3 = MEASURED_FP64_FLOP_PER_CELL.get(3)
        if flop3 and fp64_tflops:
            ach = forms["f64"]["glups"] * 1e9 * flop3 / 1e12
            forms["f64"]["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64_tflops, "unit": "TFLOP/s",
                                        "frac": ach / fp64_tflops, "flop_per_cell": flop3,
                                        "fp64_pipe_frac": forms["f64"]["glups"] * 1e9 *
                                        MEASURED_FP64_INSTR_PER_CELL[3] / (fp64_tflops * 1e12 / 2)}
        scale = Q.reshape(8, -1).abs().amax(1)
        for form in ["f32"] + [f for f in form_list if f not in ("f64", "f32")]:
            c = make_ctx(form)
            msf, _ = timed(c, nfs, 0, collective=False)
            Qf = moments_dev(c)
            st = vlbm.vlbm_sync(c.ptr)
            c.close()
            diff = (Qf - Q64).reshape(8, -1)
            linf = (diff.abs().amax(1) / scale).cpu().numpy()
            l2 = (diff.pow(2).mean(1).sqrt() / scale).cpu().numpy()
            del Qf, diff
            gl = ncell * nfs / (msf * 1e-3) / 1e9
            forms[form] = {"glups": gl, "steps": nfs, "bytes_per_cell": 2 * 56 * BYTES_PER_POP[form],
                           "roofline_frac": gl * 1e9 * 2 * 56 * BYTES_PER_POP[form] / (hbm_peak * 1e9),
                           "status": vlbm.status_string(st),
                           "rel_linf_vs_f64": dict(zip(fields.IDEAL_FIELDS, [float(v) for v in linf])),
                           "rel_l2_vs_f64": dict(zip(fields.IDEAL_FIELDS, [float(v) for v in l2]))}
        del Q64

    growth = None
    if world == 1 and args.growth_steps > 0 and form_list:
        growth = error_growth(args, vlbm, fields, torch, stream)

    extra = {}
    if world == 1 and not args.no_extra:
        which = set(x for x in args.extras.split(",") if x)
        if "channel" in which:
            extra["resistive_channel"] = channel_form(args, vlbm, fields, torch, stream, hbm_peak)
        if "batch" in which:
            extra["batched_2d"] = batch_form(args, vlbm, fields, torch, stream, hbm_peak)
        if "closure" in which:
            extra["learned_closure"] = closure_form(args, vlbm, torch, stream)
        if "powell" in which:
            extra["powell_3d"] = powell_form(args, vlbm, fields, torch, stream, hbm_peak)
        if "hlbm" in which:
            extra["hlbm_sphere_3d"] = hlbm_form(args, vlbm, fields, torch, stream, hbm_peak)
        if "open" in which:
            extra["open_faces_3d"] = open_form(args, vlbm, fields, torch, stream, hbm_peak)
        if "slabs" in which:
            extra["slabs_one_gpu"] = slab_form(args, vlbm, fields, torch, stream, hbm_peak)
        if "diss" in which:
            extra["dissipative_2d"] = dissipative_form(args, vlbm, fields, torch, stream, hbm_peak)
        if "diss3" in which:
            extra["dissipative_3d"] = dissipative3_form(args, vlbm, fields, torch, stream, hbm_peak)
        if "cfg1" in which:
            extra["ideal_2d_128sq_f64"] = ideal_2d_f64_form(args, vlbm, fields, torch, stream, fp64_tflops)

    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args, args.cpu_seconds)
        cpu.pop("steps", None)
        cpu.pop("ms_per_step", None)

    if rank == 0:
        line = {
            "metric": "GLUPS", "value": glups, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": ("%d^3" % n) if world == 1 else
                       "%d x %d x %d periodic, one %d^3 z-slab per rank" % (n, n, n * world, n),
                       "cells": ncell * world, "storage": args.storage,
                       "populations_per_cell": 56,
                       "parallelism": "single domain" if world == 1 else
                       "slab decomposition along z, population halo exchanged by NCCL send/recv after "
                       "every step (one slot plane per lattice per face each way)",
                       "l2": "inputs_larger_than_l2 (%.1f GB of populations per rank)"
                             % (ncell * 56 * BYTES_PER_POP[args.storage] / 1e9)},
            "status": vlbm.status_string(status),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak,
                         "traffic": (MEASURED_DRAM_BYTES_PER_CELL[args.storage] * ncell
                                     if MEASURED_DRAM_BYTES_PER_CELL.get(args.storage) else None),
                         "peak_kind": peak_kind,
                         "kernel": STEP_KERNEL[args.storage],
                         "algorithmic_bytes_per_launch": ncell * bytes_cell},
            "clocks": clk,
            "repeats": spread,
            "gpu_launches": launches,
            "slab_check": slab_check,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "forms": forms or None,
            "error_growth": growth,
            "other_paths": extra or None,
            "paper_context": {"note": "RTX A5000, FP32, 2-D D2Q5 kernel 98.9% and 3-D homogenised D3Q7 "
                                      "kernel 75.8% of a 680 GB/s measured roofline; other hardware"},
            "fp64_tflops": fp64_tflops,
        }
        line["summary"] = compact_summary(line)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
