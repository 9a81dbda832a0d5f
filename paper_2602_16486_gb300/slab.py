"""One lattice over several processes, one slab per rank (the decomposition of
``flbm_create_slab``), with the halo messages sent over ``torch.distributed``.

Only data movement lives here: the step, the statistics and the region bookkeeping are
the library's (``flbm_step``, ``flbm_stats``, ``flbm_slab_halo``). A message is a list of
contiguous runs of the slab's population array, sent and received run by run as views of
the caller-owned device buffer, so no packing kernel and no copy sits in between.

Ordering. Around every step taken from an odd step count each rank exchanges one message
with the rank below and one with the rank above (periodic in z). A rank posts its sends
as (side 0, side 1) and its receives as (side 1, side 0): with two ranks both neighbours
are the same peer, and the lower rank's side-0 message is the upper rank's side-1
message, so this order pairs them whatever way the backend matches messages between one
pair of ranks (in posting order).
"""
from __future__ import annotations

import numpy as np

from . import flbm as _fl


def exchange(buf, elem_bytes, lattice, dims, z_count, phase, rank, world, group=None):
    """One phase (0: before the step, 1: after it) of this rank's halo exchange.

    buf   : 1-D uint8 tensor over the slab's whole local array (the dev_buf given to
            flbm_create_slab), on the device the process group's backend uses.
    dims  : the whole lattice; z_count: this rank's owned planes (each rank computes its
            own send and receive offsets; the regions of a message pair up in order).
    """
    import torch.distributed as dist

    lo, hi = (rank - 1) % world, (rank + 1) % world
    regions = {side: _fl.flbm_slab_halo(lattice, dims, z_count, phase, side) for side in (0, 1)}

    def view(off, n):
        return buf[off * elem_bytes:(off + n) * elem_bytes]

    if world == 1:  # the slab is its own neighbour on both sides
        for side in (0, 1):
            send, _, n = regions[side]
            _, recv, _ = regions[1 - side]
            for s, r in zip(send, recv):
                view(r, n).copy_(view(s, n))
        return
    ops = []
    for side, peer in ((0, lo), (1, hi)):
        send, _, n = regions[side]
        ops += [dist.P2POp(dist.isend, view(s, n), peer, group) for s in send]
    for side, peer in ((1, hi), (0, lo)):
        _, recv, n = regions[side]
        ops += [dist.P2POp(dist.irecv, view(r, n), peer, group) for r in recv]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def split_planes(nz, world):
    """(z_begin, z_count) of every rank: planes split as evenly as possible, the first
    nz mod world ranks one plane thicker (the split flbm_domain_create uses)."""
    out, z = [], 0
    for r in range(world):
        zc = nz // world + (1 if r < nz % world else 0)
        out.append((z, zc))
        z += zc
    return out


def combine_stats(st, world, group=None, device="cpu"):
    """Statistics of the whole lattice from every rank's slab statistics: the sums (mass,
    momentum, non-finite count) add and the means are weighted by the owned sites, in
    FP64 (an all-reduce of the same sums the slabs' records hold). `device`: where the
    process group's backend takes tensors ("cuda" for NCCL)."""
    import torch
    import torch.distributed as dist

    n = float(st["sites"])
    vec = np.concatenate([[n, st["mass"], float(st["nonfinite"])], st["mom"], np.asarray(st["u_mean"]) * n,
                          np.asarray(st["uu"]) * n, np.asarray(st["k_mean"]) * n, np.asarray(st["k_cov"]).ravel() * n])
    t = torch.tensor(vec, dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, group=group)
    v = t.cpu().numpy()
    q = len(st["k_mean"])
    total = v[0]
    out = dict(st)
    out["sites"] = int(round(total))
    out["mass"] = float(v[1])
    out["nonfinite"] = int(round(v[2]))
    out["mom"] = v[3:6].copy()
    out["u_mean"] = v[6:9] / total
    out["uu"] = v[9:15] / total
    out["k_mean"] = v[15:15 + q] / total
    out["k_cov"] = (v[15 + q:15 + q + q * q] / total).reshape(np.asarray(st["k_cov"]).shape)
    return out


class SlabLattice:
    """This rank's slab of one lattice; `step(n)` advances the whole lattice n steps
    together with the other ranks (collective: every rank calls it)."""

    def __init__(self, lattice, dims, lam, kBT, rho0, seed, rank, world, storage=_fl.FLBM_FP32,
                 cuda_stream=None, group=None, device=None):
        import torch

        self.lattice, self.dims = int(lattice), tuple(int(x) for x in dims)
        self.rank, self.world, self.group = rank, world, group
        self.z_begin, self.z_count = split_planes(self.dims[2], world)[rank]
        nbytes = _fl.flbm_slab_required_bytes(lattice, self.dims, self.z_count, storage)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
        self.elem_bytes = 4 if storage == _fl.FLBM_FP32 else 2
        self.stream = cuda_stream
        self.ctx = _fl.flbm_create_slab(lattice, self.dims, self.z_begin, self.z_count, lam, kBT, rho0, seed,
                                        storage, cuda_stream, self.buf.data_ptr(), nbytes)
        self._ghosts = False

    def _exchange(self, phase):
        # The library's work on the slab is ordered on its stream and the messages on the
        # process group's streams: synchronise the device on both sides of the exchange.
        import torch

        _fl.flbm_sync(self.ctx)
        exchange(self.buf, self.elem_bytes, self.lattice, self.dims, self.z_count, phase, self.rank, self.world,
                 self.group)
        if self.buf.is_cuda:
            torch.cuda.synchronize(self.buf.device)

    def init_uniform(self, u0=(0.0, 0.0, 0.0), amp=0.0, perturb_seed=0):
        _fl.flbm_init_uniform(self.ctx, u0, amp, perturb_seed)
        self._ghosts = False

    def step(self, n=1):
        for _ in range(int(n)):
            odd = _fl.flbm_get_step(self.ctx) & 1
            if odd and not self._ghosts:
                self._exchange(0)
            _fl.flbm_step(self.ctx, 1)
            if odd:
                self._exchange(1)
            self._ghosts = False

    def stats(self):
        """Statistics of the whole lattice (collective)."""
        if _fl.flbm_get_step(self.ctx) & 1 and not self._ghosts:
            self._exchange(0)
            self._ghosts = True
        return combine_stats(_fl.flbm_stats(self.ctx), self.world, self.group, self.buf.device)

    def close(self):
        if self.ctx:
            _fl.flbm_destroy(self.ctx)
            self.ctx = None
