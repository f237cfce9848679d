"""Particle shards of one configuration: the host side of ssh_shard_* (argument marshalling and exchanges only).

Both sums of a step are reductions over the particles (Simulations), so one configuration can be split over
several GPUs: each holds a shard context (ssh_opts.shard_first / shard_count) that sums n~ over its own particles
and forces only them.  The library does every step of the arithmetic; this module allocates each shard's two
exchange buffers and sums them element-wise over the shards -- first over the shards this process holds, then over
the processes through a Comm (torch.distributed: NCCL for CUDA buffers, gloo for host buffers).  The density buffer
holds exact int64 level groups, so its sum is exact in any order; each element of the dot-product buffer is
non-zero on one shard at most, so its binary64 sum is exact too.  Every shard therefore ends each step with the
whole configuration's Phi, S_max and n~ and the same FIRE decisions, bit for bit those of one unsharded context.

A ShardGroup drives any objects with the shard_* methods of ssh.Context; `pointer` turns a buffer into what those
methods take (a device address for the library).
"""
from __future__ import annotations

import math

ALIGN = 2048   # shard boundaries lie on multiples of the FIRE dot-product chunk (ssh.h, ssh_opts.shard_first)


def shard_ranges(N: int, G: int, align: int = ALIGN) -> list[tuple[int, int]]:
    """G contiguous shards (first, count) of N particles, boundaries on multiples of `align`, as even as that
    allows (a shard ends at N or holds a multiple of `align`)."""
    blocks = math.ceil(N / align)
    if G < 1 or G > blocks:
        raise ValueError(f"{G} shards of N = {N} need at least {G} chunks of {align} particles")
    out, b0 = [], 0
    for r in range(G):
        b1 = blocks * (r + 1) // G
        first, end = b0 * align, min(N, b1 * align)
        out.append((first, end - first))
        b0 = b1
    return out


class Comm:
    """Element-wise sums over the processes that hold the other shards (none by default: one process)."""
    rank, world = 0, 1

    def allreduce_sum_(self, t):
        return t


class TorchComm(Comm):
    """torch.distributed in-place SUM all-reduce (NCCL for CUDA tensors, gloo for CPU tensors) of a process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self._dist = dist
        self._group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def allreduce_sum_(self, t):
        self._dist.all_reduce(t, op=self._dist.ReduceOp.SUM, group=self._group)
        return t


class ShardGroup:
    """The shards of one configuration held by this process (usually one per process), and the Comm to the
    processes that hold the rest.

    shards  objects with shard_words / shard_density / shard_finish / shard_fire_begin / shard_step_dots /
            shard_step_move / shard_step_finish / fire_state (ssh.Context built with shard=...)
    alloc   alloc(n, kind) -> a zeroed buffer of n int64 ("i64") or binary64 ("f64") words
    pointer pointer(buffer) -> the argument the shard methods take (default: buffer.data_ptr())
    sync    called before a buffer is summed and after the sum, when the shards and the sums do not share one
            stream (e.g. ssh.Context.sync and torch.cuda.synchronize); None when they do
    """

    def __init__(self, shards, comm: Comm | None = None, alloc=None, pointer=None, sync=None):
        if not shards:
            raise ValueError("no shards")
        self.shards = list(shards)
        self.comm = comm or Comm()
        self._ptr = pointer or (lambda t: t.data_ptr())
        self._sync = sync
        dens_words, dots_words = self.shards[0].shard_words()
        for s in self.shards[1:]:
            if s.shard_words() != (dens_words, dots_words):
                raise ValueError("the shards belong to different configurations")
        self.dens = [alloc(dens_words, "i64") for _ in self.shards]
        self.dots = [alloc(dots_words, "f64") for _ in self.shards]
        self.dens_tot = alloc(dens_words, "i64")
        self.dots_tot = alloc(dots_words, "f64")

    def _sum(self, bufs, tot):
        if self._sync:
            self._sync("before")
        tot.copy_(bufs[0])
        for b in bufs[1:]:
            tot.add_(b)
        self.comm.allreduce_sum_(tot)
        if self._sync:
            self._sync("after")

    def eval(self, want_force: bool = True):
        """Phi, S_max, n~ of the whole configuration and F of each shard's particles, left in the shard contexts."""
        for s, b in zip(self.shards, self.dens):
            s.shard_density(self._ptr(b))
        self._sum(self.dens, self.dens_tot)
        for s in self.shards:
            s.shard_finish(self._ptr(self.dens_tot), want_force)

    def fire_begin(self, params=None, **kw):
        """A FIRE run (one fixed-point stage) from the current positions: one exchanged evaluation, then the start."""
        self.eval(True)
        for s in self.shards:
            s.shard_fire_begin(params, **kw)

    def step(self):
        """One FIRE step: dot products -> exchange -> controls, move, density -> exchange -> finish, acceptance."""
        for s, b in zip(self.shards, self.dots):
            s.shard_step_dots(self._ptr(b))
        self._sum(self.dots, self.dots_tot)
        for s, b in zip(self.shards, self.dens):
            s.shard_step_move(self._ptr(self.dots_tot), self._ptr(b))
        self._sum(self.dens, self.dens_tot)
        for s in self.shards:
            s.shard_step_finish(self._ptr(self.dens_tot))

    def steps(self, n: int):
        for _ in range(n):
            self.step()

    def state(self) -> dict:
        """The FIRE state (ssh_fire_state), which every shard holds identically; checked across this process's shards."""
        st = [s.fire_state() for s in self.shards]
        keys = ("steps", "rejected", "smax", "phi", "dt", "running")
        for other in st[1:]:
            if any(other[k] != st[0][k] for k in keys):
                raise RuntimeError(f"shards disagree on the FIRE state: {st[0]} vs {other}")
        return st[0]
