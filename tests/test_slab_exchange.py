"""The halo logic of the slab decomposition on CPU, with two (and one) gloo ranks.

The library's region lists (flbm_slab_halo, host only) and the process-to-process
exchange (paper_2602_16486_gb300.slab.exchange) move the slots of an in-place AA-pattern
array between slabs; the per-site update is replaced here by the identity, so that after
k steps every population must have streamed exactly k c_i (Eq. streaming, periodic), bit
for bit. Ghost planes start as NaN, so any slot read before the exchange filled it shows.
The statistics of the slabs, combined over ranks (slab.combine_stats), must equal the
oracle's statistics of the whole lattice.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _emulate(rank, world, lattice, dims, steps, port, out):
    import sys

    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2602_16486_gb300 import slab

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c, w, _ = oracle.tables(lattice)
        Q = len(w)
        opp = [int(np.where((c == -c[i]).all(1))[0][0]) for i in range(Q)]
        nx, ny, nz = dims
        z0, zc = slab.split_planes(nz, world)[rank]
        rng = np.random.default_rng(5)
        f0 = rng.standard_normal((Q, nz, ny, nx)).astype(np.float32)  # logical, even state
        A = np.full((Q, zc + 2, ny, nx), np.nan, dtype=np.float32)
        A[:, 1:zc + 1] = f0[:, z0:z0 + zc]
        buf = torch.from_numpy(A.reshape(-1).view(np.uint8))  # shares memory with A
        zz, yy, xx = np.meshgrid(np.arange(1, zc + 1), np.arange(ny), np.arange(nx), indexing="ij")

        def at(i, dz, dy, dx):  # index arrays of slot i at owned sites shifted by (dx, dy, dz)
            return (i, zz + dz, (yy + dy) % ny, (xx + dx) % nx)

        for k in range(steps):
            if k % 2 == 0:  # reads and writes the site's own slots
                F = [A[at(i, 0, 0, 0)].copy() for i in range(Q)]
                for i in range(Q):
                    A[at(opp[i], 0, 0, 0)] = F[i]
            else:
                slab.exchange(buf, 4, lattice, dims, zc, 0, rank, world)
                F = [A[at(opp[i], -c[i, 2], -c[i, 1], -c[i, 0])].copy() for i in range(Q)]
                for i in range(Q):
                    A[at(i, c[i, 2], c[i, 1], c[i, 0])] = F[i]
                slab.exchange(buf, 4, lattice, dims, zc, 1, rank, world)
        if steps % 2:  # odd state: the arriving populations sit in the neighbours' slots
            slab.exchange(buf, 4, lattice, dims, zc, 0, rank, world)
            got = np.stack([A[at(opp[i], -c[i, 2], -c[i, 1], -c[i, 0])] for i in range(Q)])
        else:
            got = np.stack([A[at(i, 0, 0, 0)] for i in range(Q)])
        # streaming alone: f_i(x, k) = f_i(x - k c_i, 0)
        want = np.stack([np.roll(f0[i], shift=(steps * c[i, 2], steps * c[i, 1], steps * c[i, 0]),
                                 axis=(0, 1, 2))[z0:z0 + zc] for i in range(Q)])
        same = bool(np.array_equal(got, want))
        # statistics: each rank's owned sites, combined over ranks, against the whole lattice
        g = (np.abs(f0) * 0.01 + w.reshape(-1, 1, 1, 1)).astype(np.float64)
        mine = oracle.stats(lattice, (nx, ny, zc), g[:, z0:z0 + zc])
        comb = slab.combine_stats(mine, world)
        ref = oracle.stats(lattice, (nx, ny, nz), g)
        stats_ok = comb["sites"] == ref["sites"] and comb["mass"] == pytest.approx(ref["mass"], rel=1e-13)
        for key in ("mom", "u_mean", "uu", "k_mean", "k_cov"):
            stats_ok = stats_ok and np.allclose(comb[key], ref[key], rtol=1e-12, atol=1e-15)
        out.put((rank, same, bool(stats_ok), int(np.isnan(got).sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(world, lattice, dims, steps):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_emulate, args=(r, world, lattice, dims, steps, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world,lattice,dims,steps", [
    (2, 1, (5, 4, 7), 5),   # D3Q27, slabs of 4 and 3 planes, odd final state
    (2, 1, (4, 3, 2), 4),   # D3Q27, one plane per slab, even final state
    (2, 3, (3, 5, 6), 7),   # D3Q19
    (1, 1, (4, 4, 3), 3),   # one slab: its own neighbour on both sides
])
def test_slab_halo_exchange_streams_exactly(world, lattice, dims, steps):
    res = _run(world, lattice, dims, steps)
    for rank, same, stats_ok, nans in res:
        assert nans == 0, f"rank {rank} read an unfilled ghost slot"
        assert same, f"rank {rank}: populations did not stream by {steps} c_i"
        assert stats_ok, f"rank {rank}: combined statistics differ from the whole lattice's"


def test_slab_halo_regions_without_gpu():
    import paper_2602_16486_gb300 as fl

    dims = (6, 5, 8)
    for lattice, nreg in ((1, 9), (2, 9), (3, 5)):
        q = 27 if lattice != 3 else 19
        zc = 3
        n_local = 6 * 5 * (zc + 2)
        seen = set()
        for phase in (0, 1):
            for side in (0, 1):
                send, recv, ln = fl.flbm_slab_halo(lattice, dims, zc, phase, side)
                assert len(send) == len(recv) == nreg and ln == 30
                for o in send + recv:
                    assert 0 <= o and o + ln <= q * n_local and (o % n_local) % ln == 0
                seen.update((phase, side, o) for o in send)
        assert len(seen) == 4 * nreg
    with pytest.raises(fl.FlbmError):
        fl.flbm_slab_halo(0, (6, 5, 1), 1, 0, 0)  # D2Q9 is not decomposed
    with pytest.raises(fl.FlbmError):
        fl.flbm_slab_halo(1, dims, 9, 0, 0)  # more planes than the lattice
    with pytest.raises(fl.FlbmError):
        fl.flbm_slab_halo(1, dims, 3, 2, 0)  # no phase 2
    assert fl.flbm_slab_required_bytes(1, (8, 8, 16), 4, fl.FLBM_FP32) == 27 * 8 * 8 * 6 * 4
