"""Training and evaluation of the learned flux closure (coarse 3-D ideal MHD).

Everything numerical runs in the library's kernels (fine and coarse steps,
restriction, network forward/backward, Adam); this module only orders the
calls and keeps device buffers (torch tensors) alive.

Set-up (acoustic scaling): a coarse cell is factor^3 fine cells and one coarse
step spans `factor` fine steps, so the lattice-unit fields of the restricted
fine run are valid coarse-lattice fields at the same tau.  Training pairs are
(R Q_fine(n factor), R Q_fine((n+1) factor)) with R the conservative block
average; the loss is the one-coarse-step error of the corrected coarse step.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import fields, vlbm


@dataclass
class ClosureRun:
    rel_l2_plain: float
    rel_l2_closure: float
    fine_ms: float
    coarse_plain_ms: float
    coarse_closure_ms: float
    steps_coarse: int


def _field_kwargs(mach):
    return dict(mach=mach, beta=1.0, cfl=0.2, k_rho=2, k_u=2, k_b=2)


def fine_trajectory(fine_shape, factor, seed, mach, n_pairs, tau, torch, stream, warm=0):
    """Restricted states R Q(n factor), n = 0..n_pairs, of one fine run (device tensors)."""
    f0 = fields.ideal_fields(fine_shape, seed, device="cuda", **_field_kwargs(mach))
    p = vlbm.make_params(shape=fine_shape, storage="f32", gamma=f0.gamma, tau=tau, stream=stream.cuda_stream)
    coarse_shape = tuple(n // factor for n in fine_shape)
    out = []
    with vlbm.Context(p) as ctx:
        st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, f0.Q.data_ptr())
        if st != vlbm.VLBM_OK:
            raise RuntimeError("fine init: " + vlbm.status_string(st))
        del f0
        if warm:
            ctx.step(warm)
        Qf = torch.empty((8,) + tuple(fine_shape), dtype=torch.float64, device="cuda")
        for n in range(n_pairs + 1):
            if n:
                ctx.step(factor)
            vlbm.vlbm_moments_device(ctx.ptr, 0, Qf.data_ptr())
            Qc = torch.empty((8,) + coarse_shape, dtype=torch.float64, device="cuda")
            vlbm.vlbm_restrict(Qf.data_ptr(), fine_shape, factor, Qc.data_ptr(), stream.cuda_stream)
            out.append(Qc)
        stream.synchronize()
        if ctx.sync() != vlbm.VLBM_OK:
            raise RuntimeError("fine run became nonphysical")
    return out


def normalisation(states):
    """Per-field mean, spread and output scale from training states."""
    import torch
    allq = torch.stack(states).transpose(0, 1).reshape(8, -1)
    mu = allq.mean(1).cpu().numpy()
    sigma = allq.std(1).cpu().numpy()
    amp = allq.abs().amax(1).cpu().numpy()
    sigma = np.maximum(sigma, 1e-3 * amp + 1e-30)
    return mu, sigma


def train(closure, trajectories, steps, rng, log_every=0):
    """Adam steps on random (state, next state) pairs drawn from the trajectories,
    each coarse step started from the equilibrium of the restricted state."""
    losses = []
    for it in range(steps):
        tr = trajectories[rng.integers(len(trajectories))]
        n = int(rng.integers(len(tr) - 1))
        losses.append(closure.train_step(tr[n].data_ptr(), tr[n + 1].data_ptr()))
        if log_every and it % log_every == 0:
            print("closure train step %d loss %.4e" % (it, losses[-1]), flush=True)
    return losses


def _world(group):
    import torch.distributed as dist
    return dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1


def average_gradients(grads, loss, group=None):
    """Data-parallel training: the mean of every process's gradient (a tensor,
    changed in place) and loss over `group` (torch.distributed all-reduce; the
    identity for one process).  Returns the mean loss."""
    import torch
    import torch.distributed as dist
    world = _world(group)
    if world == 1:
        return float(loss)
    lt = torch.tensor([float(loss)], dtype=torch.float64, device=grads.device)
    dist.all_reduce(grads, group=group)
    dist.all_reduce(lt, group=group)
    grads.div_(world)
    return float(lt.item()) / world


def dp_train_step(closure, ctx, Qt, grads, group=None):
    """One data-parallel training step: this process's loss and gradient for one
    corrected coarse step of `ctx` against Qt, the gradient averaged over the
    processes of `group`, one Adam step with the average (the same on every
    process, so the weights stay equal).  `grads`: a device float tensor of
    vlbm_closure_num_params entries.  Returns the mean loss."""
    loss = closure.grad_step_ctx(ctx.ptr, Qt.data_ptr(), grads.data_ptr())
    loss = average_gradients(grads, loss, group)
    closure.apply_grads(grads.data_ptr())
    return loss


def train_in_the_loop(closure, trajectories, episodes, gamma, tau, stream, rng, rollout=None, log_every=0,
                      group=None):
    """Solver-in-the-loop training: each episode restarts a coarse run from the
    restricted fine state at a random time and advances it with the current
    closure, one Adam step per coarse step against the restricted fine state
    of the same time (gradient through the last step only).  With a process
    group of more than one process, every process runs its own episodes (its
    own trajectories and rng) and the gradients are averaged at every step
    (`dp_train_step`); each process must run the same number of episodes and
    roll-out steps."""
    import torch
    losses = []
    shape = tuple(trajectories[0][0].shape[1:])
    p = vlbm.make_params(shape=shape, storage="f32", gamma=gamma, tau=tau, stream=stream.cuda_stream)
    dp = _world(group) > 1
    if dp and not rollout:
        raise ValueError("data-parallel training needs a fixed roll-out length on every process")
    grads = torch.empty(closure.nparam, dtype=torch.float32, device="cuda") if dp else None
    with vlbm.Context(p) as ctx:
        for ep in range(episodes):
            tr = trajectories[rng.integers(len(trajectories))]
            n_roll = rollout or (len(tr) - 1)
            start = int(rng.integers(len(tr) - n_roll)) if n_roll < len(tr) - 1 else 0
            st = vlbm.vlbm_init_fields_device(ctx.ptr, 0, tr[start].data_ptr())
            if st != vlbm.VLBM_OK:
                raise RuntimeError("coarse init: " + vlbm.status_string(st))
            for n in range(start + 1, start + n_roll + 1):
                if dp:
                    losses.append(dp_train_step(closure, ctx, tr[n], grads, group))
                else:
                    losses.append(closure.train_step_ctx(ctx.ptr, tr[n].data_ptr()))
            if ctx.sync() != vlbm.VLBM_OK:
                losses.append(float("nan"))
            if log_every and ep % log_every == 0:
                print("closure episode %d loss %.4e" % (ep, losses[-1]), flush=True)
    return losses


def train_with_validation(closure, trajectories, episodes, gamma, tau, stream, rng, validate, val_every=10,
                          rollout=4, log=None, group=None):
    """In-the-loop training with early stopping: every `val_every` episodes
    `validate()` returns the held-out error of the corrected coarse run; the
    weights with the lowest validation error (the zero-output start included)
    are restored at the end.  Returns (best error, history)."""
    best_w = closure.get_weights()
    best = validate()
    history = [(0, best)]
    done = 0
    while done < episodes:
        n = min(val_every, episodes - done)
        train_in_the_loop(closure, trajectories, n, gamma, tau, stream, rng, rollout=rollout, group=group)
        done += n
        err = validate()
        history.append((done, err))
        if log:
            log("episode %d validation error %.4e (best %.4e)" % (done, err, best))
        if np.isfinite(err) and err < best:
            best, best_w = err, closure.get_weights()
    closure.set_weights(best_w)
    return best, history


@dataclass
class FineReference:
    Qc0: object          # restricted initial state (device, 8 x coarse cells)
    Qref: object         # restricted fine state after n_coarse * factor fine steps
    fine_ms: float       # device time of the fine steps
    gamma: float
    n_coarse: int


def fine_reference(fine_shape, factor, seed, mach, n_coarse, tau, torch, stream):
    """Run the fine solver once and keep the restricted start and end states."""
    coarse_shape = tuple(n // factor for n in fine_shape)
    f0 = fields.ideal_fields(fine_shape, seed, device="cuda", **_field_kwargs(mach))
    gamma = f0.gamma
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p = vlbm.make_params(shape=fine_shape, storage="f32", gamma=gamma, tau=tau, stream=stream.cuda_stream)
    Qc0 = torch.empty((8,) + coarse_shape, dtype=torch.float64, device="cuda")
    Qref = torch.empty_like(Qc0)
    with vlbm.Context(p) as ctx:
        vlbm.vlbm_init_fields_device(ctx.ptr, 0, f0.Q.data_ptr())
        del f0
        Qf = torch.empty((8,) + tuple(fine_shape), dtype=torch.float64, device="cuda")
        vlbm.vlbm_moments_device(ctx.ptr, 0, Qf.data_ptr())
        vlbm.vlbm_restrict(Qf.data_ptr(), fine_shape, factor, Qc0.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        ev0.record(stream)
        ctx.step(n_coarse * factor)
        ev1.record(stream)
        ev1.synchronize()
        fine_ms = ev0.elapsed_time(ev1)
        vlbm.vlbm_moments_device(ctx.ptr, 0, Qf.data_ptr())
        vlbm.vlbm_restrict(Qf.data_ptr(), fine_shape, factor, Qref.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        if ctx.sync() != vlbm.VLBM_OK:
            raise RuntimeError("fine reference run became nonphysical")
    return FineReference(Qc0=Qc0, Qref=Qref, fine_ms=fine_ms, gamma=gamma, n_coarse=n_coarse)


def coarse_error(ref, closure, tau, torch, stream):
    """Relative L2 error (normalised per field by the reference spread) of the
    coarse run from ref.Qc0 after ref.n_coarse steps, with `closure` (or None),
    its device time and final status."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    shape = tuple(ref.Qc0.shape[1:])
    pc = vlbm.make_params(shape=shape, storage="f32", gamma=ref.gamma, tau=tau, stream=stream.cuda_stream)
    with vlbm.Context(pc) as c:
        vlbm.vlbm_init_fields_device(c.ptr, 0, ref.Qc0.data_ptr())
        if closure is not None:
            vlbm.vlbm_set_closure(c.ptr, closure)
        stream.synchronize()
        ev0.record(stream)
        c.step(ref.n_coarse)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        out = torch.empty_like(ref.Qc0)
        vlbm.vlbm_moments_device(c.ptr, 0, out.data_ptr())
        stream.synchronize()
        vlbm.vlbm_set_closure(c.ptr, None)
        st = c.sync()
    scale = ref.Qref.reshape(8, -1).std(1) + 1e-30
    d = (out - ref.Qref).reshape(8, -1) / scale[:, None]
    return float(d.pow(2).mean().sqrt()), ms, st


def evaluate(closure, fine_shape, factor, seed, mach, n_coarse, tau, torch, stream, ref=None):
    """Plain and closure-corrected coarse runs against the restricted fine run."""
    if ref is None:
        ref = fine_reference(fine_shape, factor, seed, mach, n_coarse, tau, torch, stream)
    e_p, ms_p, st_p = coarse_error(ref, None, tau, torch, stream)
    e_c, ms_c, st_c = coarse_error(ref, closure, tau, torch, stream)
    return ClosureRun(rel_l2_plain=e_p, rel_l2_closure=e_c, fine_ms=ref.fine_ms, coarse_plain_ms=ms_p,
                      coarse_closure_ms=ms_c, steps_coarse=n_coarse), (st_p, st_c)


def init_weights(rng, hidden=32, last_scale=0.1):
    """He-style random weights in the library's flat order (last layer scaled)."""
    parts = []
    for o, c, s in ((hidden, 8, 1.0), (hidden, hidden, 1.0), (24, hidden, last_scale)):
        parts.append(rng.normal(0.0, s * np.sqrt(2.0 / (27 * c)), size=o * c * 27))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def run_experiment(fine_shape=(512, 512, 512), factor=4, train_seeds=tuple(range(5000, 5008)), val_seed=5100,
                   test_seeds=(5101, 5102, 5103), mach=1.5, tau=0.51, n_pairs=32, n_eval=32, episodes=150,
                   val_every=10, rollout=4, lr=1e-5, out_scale_rel=0.005, seed=0, log=None):
    """Train in the loop on restricted fine runs of `train_seeds` with early
    stopping on `val_seed`; report plain and corrected coarse errors and
    times on the held-out `test_seeds`."""
    import torch
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    trajs = [fine_trajectory(fine_shape, factor, s, mach, n_pairs, tau, torch, stream) for s in train_seeds]
    t_data = time.perf_counter() - t0
    mu, sigma = normalisation([q for tr in trajs for q in tr])
    coarse_shape = tuple(n // factor for n in fine_shape)
    gamma = 5.0 / 3.0
    cl = vlbm.Closure(coarse_shape, gamma, tau, mu, sigma, out_scale_rel * sigma, lr=lr,
                      stream=stream.cuda_stream)
    rng = np.random.default_rng(seed)
    cl.set_weights(init_weights(rng, last_scale=0.0))
    vref = fine_reference(fine_shape, factor, val_seed, mach, n_eval, tau, torch, stream)
    t0 = time.perf_counter()
    best, hist = train_with_validation(cl, trajs, episodes, gamma, tau, stream, rng,
                                       lambda: coarse_error(vref, cl, tau, torch, stream)[0],
                                       val_every=val_every, rollout=rollout, log=log)
    t_train = time.perf_counter() - t0
    del trajs
    tests = []
    for s in test_seeds:
        res, st = evaluate(cl, fine_shape, factor, s, mach, n_eval, tau, torch, stream)
        tests.append({"seed": s, "rel_l2_plain_coarse": res.rel_l2_plain, "rel_l2_closure_coarse": res.rel_l2_closure,
                      "fine_ms": res.fine_ms, "coarse_plain_ms": res.coarse_plain_ms,
                      "coarse_closure_ms": res.coarse_closure_ms, "status": [int(v) for v in st]})
    return {"closure": cl, "best_val": best, "history": hist, "tests": tests, "t_data_s": t_data,
            "t_train_s": t_train, "fine_shape": fine_shape, "coarse_shape": coarse_shape, "n_eval": n_eval}


# ---------------------------------------------------------------------------
# Time to solution against the plain method's error-vs-time curve
# ---------------------------------------------------------------------------

def _run_plain(Q0, gamma, tau, steps, torch, stream):
    """A plain FP32 run from device fields Q0: final fields, device ms of the steps, status."""
    shape = tuple(Q0.shape[1:])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p = vlbm.make_params(shape=shape, storage="f32", gamma=gamma, tau=tau, stream=stream.cuda_stream)
    with vlbm.Context(p) as c:
        st = vlbm.vlbm_init_fields_device(c.ptr, 0, Q0.data_ptr())
        if st != vlbm.VLBM_OK:
            return None, 0.0, st
        stream.synchronize()
        ev0.record(stream)
        c.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        out = torch.empty_like(Q0)
        vlbm.vlbm_moments_device(c.ptr, 0, out.data_ptr())
        stream.synchronize()
        return out, ev0.elapsed_time(ev1), c.sync()


def _restricted(Q, factor, torch, stream):
    shape = tuple(Q.shape[1:])
    out = torch.empty((8,) + tuple(n // factor for n in shape), dtype=torch.float64, device="cuda")
    vlbm.vlbm_restrict(Q.data_ptr(), shape, factor, out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return out


def _rel_l2(Q, ref):
    scale = ref.reshape(8, -1).std(1) + 1e-30
    d = (Q - ref).reshape(8, -1) / scale[:, None]
    return float(d.pow(2).mean().sqrt())


def _curve_error_at(points, t):
    """Plain error at device time t on the log-log line through the two curve
    points around t (the last segment beyond the ends); points = [(ms, err)]."""
    pts = sorted((float(a), float(b)) for a, b in points if a > 0 and b > 0)
    if len(pts) < 2:
        return None
    i = 0
    while i < len(pts) - 2 and pts[i + 1][0] < t:
        i += 1
    (t0, e0), (t1, e1) = pts[i], pts[i + 1]
    if t1 == t0:
        return e0
    w = (np.log(t) - np.log(t0)) / (np.log(t1) - np.log(t0))
    return float(np.exp(np.log(e0) + w * (np.log(e1) - np.log(e0))))


def resolution_curve(closure, seed, mach, n_coarse, tau, torch, stream, fine=512, coarse=128,
                     sides=(64, 128, 256), measure=64):
    """One held-out seed: the fine run (fine^3, n_coarse fine / coarse steps in
    acoustic scaling) and plain runs at every side in `sides`, each started from
    the conservative restriction of the fine initial state (so every run solves
    the same physical problem: the seeded recipe normalises its amplitudes and
    its lattice scale on the grid it is sampled on), for n_coarse side / coarse
    steps; the coarse run (side `coarse`) with and without `closure`.  Every
    final state is restricted to `measure`^3 and compared there with the
    restricted fine state (relative L2, per field over the reference spread).
    Returns device times, errors and where the closure sits against the plain
    error-vs-time curve (log-log interpolation between the plain points)."""
    f0 = fields.ideal_fields((fine,) * 3, seed, device="cuda", **_field_kwargs(mach))
    gamma = f0.gamma
    Qf = f0.Q
    del f0
    starts = {n: _restricted(Qf, fine // n, torch, stream) for n in sorted(set(sides) | {coarse})}
    Qf_end, fine_ms, st = _run_plain(Qf, gamma, tau, n_coarse * fine // coarse, torch, stream)
    del Qf
    row = {"seed": seed, "mach": mach, "fine_status": int(st), "fine_ms": fine_ms}
    if st != vlbm.VLBM_OK:
        return row
    ref = _restricted(Qf_end, fine // measure, torch, stream)
    ref_c = _restricted(Qf_end, fine // coarse, torch, stream)
    del Qf_end
    torch.cuda.empty_cache()

    def at_measure(Q, n):
        return Q if n == measure else _restricted(Q, n // measure, torch, stream)

    curve = {}
    for n in sides:
        out, ms, stn = _run_plain(starts[n], gamma, tau, n_coarse * n // coarse, torch, stream)
        curve[str(n)] = [ms, _rel_l2(at_measure(out, n), ref) if stn == vlbm.VLBM_OK else None, int(stn)]
        del out
    row["plain"] = curve
    for name, cl in (("coarse_plain", None), ("coarse_closure", closure)):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p = vlbm.make_params(shape=(coarse,) * 3, storage="f32", gamma=gamma, tau=tau, stream=stream.cuda_stream)
        with vlbm.Context(p) as c:
            vlbm.vlbm_init_fields_device(c.ptr, 0, starts[coarse].data_ptr())
            if cl is not None:
                vlbm.vlbm_set_closure(c.ptr, cl)
            stream.synchronize()
            ev0.record(stream)
            c.step(n_coarse)
            ev1.record(stream)
            ev1.synchronize()
            out = torch.empty_like(starts[coarse])
            vlbm.vlbm_moments_device(c.ptr, 0, out.data_ptr())
            stream.synchronize()
            vlbm.vlbm_set_closure(c.ptr, None)
            stc = c.sync()
        # [device ms, error on the measure grid, error on the coarse grid, status]
        row[name] = [ev0.elapsed_time(ev1), _rel_l2(at_measure(out, coarse), ref), _rel_l2(out, ref_c), int(stc)]
    pts = [(v[0], v[1]) for v in curve.values() if v[1] is not None]
    t_c, e_c = row["coarse_closure"][0], row["coarse_closure"][1]
    e_curve = _curve_error_at(pts, t_c)
    row["plain_curve_error_at_closure_time"] = e_curve
    row["closure_over_curve"] = (e_c / e_curve) if e_curve else None
    return row


def cfg5_mach(seed: int, lo: float = 1.0, hi: float = 3.0) -> float:
    """Peak Mach of a seed's fields in the learned-closure workload: drawn
    uniformly in [lo, hi] from the seed (a seeded draw, no arithmetic of the method)."""
    return float(np.random.default_rng(seed).uniform(lo, hi))


def run_protocol(fine=512, factor=4, train_seeds=tuple(range(5000, 5016)), val_seed=5016,
                 test_seeds=(5100, 5101, 5102, 5103), mach_range=(1.0, 3.0), tau=0.51, n_pairs=16,
                 warm_steps=(0, 100, 200, 300), n_eval=250, episodes=160, val_every=20, rollout=4, lr=1e-5,
                 out_scale_rel=0.005, seed=0, sides=(64, 128, 256), measure=64, log=None, group=None):
    """The learned-closure workload end to end: restricted fine trajectories of
    `train_seeds` (each starting `warm_steps[i % 4]` fine steps into its run, so
    early and developed states are both seen), in-the-loop training with early
    stopping on `val_seed` over an `n_eval`-coarse-step run, then on each held-out
    seed the fine run, the plain error-vs-time curve and the coarse runs with and
    without the closure (resolution_curve).  Seeds whose fine run turns
    non-physical are reported and left out of the training data.

    With a process group of P > 1 processes (one GPU each), process r takes the
    training seeds r, r + P, ...; the feature normalisation is the mean of the
    processes' (they see equal shares), the weights start equal, every process
    draws its own episodes, gradients are averaged at every step, and every
    process validates (so that all keep the same weights); the held-out seeds
    run on process 0 only."""
    import torch
    stream = torch.cuda.Stream()
    shape = (fine,) * 3
    coarse = fine // factor
    world = _world(group)
    rank = 0
    if world > 1:
        import torch.distributed as dist
        rank = dist.get_rank(group)
        train_seeds = tuple(train_seeds)[rank::world]
    t0 = time.perf_counter()
    trajs, skipped = [], []
    for i, s in enumerate(train_seeds):
        try:
            trajs.append(fine_trajectory(shape, factor, s, cfg5_mach(s, *mach_range), n_pairs, tau, torch, stream,
                                         warm=warm_steps[i % len(warm_steps)]))
        except RuntimeError:
            skipped.append(s)
    t_data = time.perf_counter() - t0
    if not trajs:
        return {"skipped_train_seeds": skipped, "error": "every training run became non-physical"}
    mu, sigma = normalisation([q for tr in trajs for q in tr])
    if world > 1:  # the same normalisation on every process: mean of the processes' mean and variance
        stats = torch.tensor(np.concatenate([mu, sigma ** 2 + mu ** 2]), dtype=torch.float64,
                             device="cuda" if dist.get_backend(group) == "nccl" else "cpu")
        dist.all_reduce(stats, group=group)
        stats = stats.cpu().numpy() / world
        mu = stats[:8]
        sigma = np.sqrt(np.maximum(stats[8:] - mu ** 2, 0.0))
    gamma = 5.0 / 3.0
    cl = vlbm.Closure((coarse,) * 3, gamma, tau, mu, sigma, out_scale_rel * sigma, lr=lr, stream=stream.cuda_stream)
    rng = np.random.default_rng(seed)
    cl.set_weights(init_weights(rng, last_scale=0.0))  # equal on every process
    if world > 1:
        rng = np.random.default_rng([seed, rank])  # each process its own episodes
    vref = fine_reference(shape, factor, val_seed, cfg5_mach(val_seed, *mach_range), n_eval, tau, torch, stream)
    t0 = time.perf_counter()
    best, hist = train_with_validation(cl, trajs, episodes, gamma, tau, stream, rng,
                                       lambda: coarse_error(vref, cl, tau, torch, stream)[0],
                                       val_every=val_every, rollout=rollout, log=log, group=group)
    t_train = time.perf_counter() - t0
    del trajs, vref
    torch.cuda.empty_cache()
    rows = [resolution_curve(cl, s, cfg5_mach(s, *mach_range), n_eval, tau, torch, stream, fine=fine, coarse=coarse,
                             sides=sides, measure=measure) for s in test_seeds] if rank == 0 else []
    return {"closure": cl, "best_val": best, "history": hist, "tests": rows, "t_data_s": t_data,
            "t_train_s": t_train, "skipped_train_seeds": skipped, "n_eval": n_eval, "coarse": coarse,
            "fine": fine, "train_seeds": list(train_seeds), "val_seed": val_seed, "test_seeds": list(test_seeds)}
