"""Slab decomposition of one periodic domain over several contexts.

The domain is cut along its last axis (z in 3-D, y in 2-D) into slabs of
whole layers; every slab is a library context marked with ``vlbm_set_slab``.
After each step the population planes that wrapped inside a slab move to the
neighbouring slabs (``vlbm_halo_pack`` / ``vlbm_halo_unpack``, routing in
``route``), which completes the streaming of Eq. 2 across the slab faces:
the decomposed run equals the single domain bit for bit.

Two drivers of the same exchange:

* ``LocalSlabs`` -- all slabs in this process on one device, one stream:
  ``vlbm_slabs_step`` does the steps and the exchange inside the library.
* ``SlabExchange`` -- one slab per process (one process per GPU): the host
  routes the packed face messages with ``torch.distributed`` point-to-point
  operations (NCCL on GPUs, gloo in the CPU tests) and one all-reduce adds
  the conservation sums.

Only argument marshalling and message routing live here; the steps, packing
and unpacking run in the library's kernels.
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np


def route(rank: int, world: int, step_count: int) -> Tuple[int, int, int, int]:
    """(hi_to, lo_to, hi_from, lo_from) of slab `rank` after a step that left
    its step count at `step_count`.

    After an even step (odd count) the odd step that follows reads, across the
    faces, the neighbours' planes: a slab's hi plane goes up (to rank + 1) and
    its lo plane down.  After an odd step (even count) the planes the boundary
    cells wrote for the neighbours go back: hi down, lo up."""
    up, down = (rank + 1) % world, (rank - 1) % world
    if step_count & 1:
        return up, down, down, up
    return down, up, up, down


def split_layers(n: int, parts: int) -> List[Tuple[int, int]]:
    """[first, last) layer ranges of `parts` slabs of an axis of n layers (the
    first n % parts slabs one layer thicker)."""
    if parts < 1 or parts > n:
        raise ValueError("need 1 <= parts <= %d layers" % n)
    base, extra = divmod(n, parts)
    out, z = [], 0
    for r in range(parts):
        w = base + (1 if r < extra else 0)
        out.append((z, z + w))
        z += w
    return out


class LocalSlabs:
    """P slabs of one domain in this process, on one device, sharing one stream.

    ``make_params(shape)`` returns the parameters of a slab of grid shape
    `shape` ((nz, ny, nx) or (ny, nx)); every slab is given the stream of the
    first slab's parameters, or one new torch stream when that is NULL."""

    def __init__(self, make_params: Callable, shape: Sequence[int], parts: int):
        from . import vlbm
        self._v = vlbm
        self.shape = tuple(int(n) for n in shape)
        self.parts = int(parts)
        self.ranges = split_layers(self.shape[0], self.parts)
        self._stream = None
        stream = None
        self.ctxs = []
        for z0, z1 in self.ranges:
            p = make_params((z1 - z0,) + self.shape[1:])
            if stream is None:
                stream = p.stream
                if not stream:
                    import torch
                    self._stream = torch.cuda.Stream()
                    stream = self._stream.cuda_stream
            p.stream = stream
            self.ctxs.append(vlbm.Context(p))
        self.ptrs = [c.ptr for c in self.ctxs]

    def init_fields(self, Q: np.ndarray) -> int:
        """Each slab from its layers of the global fields Q [nvar, (nz,) ny, nx]; marks the slabs."""
        worst = self._v.VLBM_OK
        for c, (z0, z1) in zip(self.ctxs, self.ranges):
            st = c.init_fields(np.ascontiguousarray(Q[:, z0:z1]))
            worst = worst if st == self._v.VLBM_OK else st
            c.set_slab(True)
        return worst

    def step(self, n: int) -> int:
        return self._v.vlbm_slabs_step(self.ptrs, n)

    def sync(self) -> int:
        out = self._v.VLBM_OK
        for c in self.ctxs:
            st = c.sync()
            out = out if st == self._v.VLBM_OK else st
        return out

    def moments(self) -> np.ndarray:
        return np.concatenate([c.moments() for c in self.ctxs], axis=1)

    def conservation(self) -> np.ndarray:
        """Sums of the decomposed domain: the slabs' FP64 sums added in slab order."""
        total = None
        for c in self.ctxs:
            s = c.conservation()
            total = s if total is None else total + s
        return total

    @property
    def launches(self) -> int:
        return sum(c.launches for c in self.ctxs)

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SlabExchange:
    """The halo exchange of this process's slab with the slabs of the other ranks.

    `pack(lo, hi)` fills the two send messages, `unpack(lo, hi)` consumes the two
    received ones (tensors of `nbytes` bytes on `device`); for a library context
    they are ``vlbm_halo_pack`` / ``vlbm_halo_unpack`` on the tensors' data
    pointers (``for_context``).  With NCCL the point-to-point operations are
    ordered on the current torch stream: run ``exchange`` under
    ``torch.cuda.stream(s)`` where s is the context's stream, and the pack, the
    transfers and the unpack follow the step in stream order with no host
    synchronisation.  A group of one rank exchanges nothing."""

    def __init__(self, pack: Callable, unpack: Callable, nbytes: int, device=None, group=None):
        import torch
        import torch.distributed as dist
        self._dist = dist
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.pack, self.unpack = pack, unpack
        self.nbytes = int(nbytes)
        mk = lambda: torch.empty(self.nbytes, dtype=torch.uint8, device=device)  # noqa: E731
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()
        self.bytes_sent = 0

    @classmethod
    def for_context(cls, ctx, device=None, group=None) -> "SlabExchange":
        """The exchange of a library slab context (``ctx.set_slab`` when the group has > 1 rank)."""
        import torch.distributed as dist
        world = dist.get_world_size(group) if dist.is_initialized() else 1
        if world > 1:
            ctx.set_slab(True)
        return cls(lambda lo, hi: ctx.halo_pack(lo.data_ptr(), hi.data_ptr()),
                   lambda lo, hi: ctx.halo_unpack(lo.data_ptr(), hi.data_ptr()),
                   ctx.halo_bytes, device=device, group=group)

    def _global(self, r: int) -> int:
        return self._dist.get_global_rank(self.group, r) if self.group is not None else r

    def exchange(self, step_count: int) -> None:
        """Move the face messages after the step that left the count at `step_count`."""
        if self.world == 1:
            return
        dist = self._dist
        hi_to, lo_to, hi_from, lo_from = route(self.rank, self.world, step_count)
        self.pack(self.send_lo, self.send_hi)
        # one order on every rank: with two ranks both messages go to the same peer,
        # and NCCL pairs the sends and receives of a peer in issue order
        ops = [dist.P2POp(dist.isend, self.send_hi, self._global(hi_to), self.group, tag=1),
               dist.P2POp(dist.isend, self.send_lo, self._global(lo_to), self.group, tag=2),
               dist.P2POp(dist.irecv, self.recv_hi, self._global(hi_from), self.group, tag=1),
               dist.P2POp(dist.irecv, self.recv_lo, self._global(lo_from), self.group, tag=2)]
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        self.unpack(self.recv_lo, self.recv_hi)
        self.bytes_sent += 2 * self.nbytes

    def allreduce_sums(self, sums, device=None) -> np.ndarray:
        """Conservation sums of the decomposed domain: this slab's FP64 sums added over the ranks."""
        import torch
        t = torch.as_tensor(np.asarray(sums, dtype=np.float64), device=device)
        if self.world > 1:
            self._dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()
