"""EqualRegions partition (Sec. 4.2.4.2) and partition halos (Sec. 4.4):
host-side invariants, and a halo exchange between gloo ranks on the CPU
after which every rank's one-ring operator on its owned nodes equals the
global result (the oracle evaluates the stencil, reading only owned and
halo values)."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1908_06091_b300 import nabla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("P", [1, 2, 3, 4, 7, 8, 32, 100])
def test_equal_regions_balance_and_bands(P):
    N = 32
    g = nabla.Grid(N)
    part, zones = nabla.equal_regions(g, P)
    assert zones.sum() == P and np.array_equal(zones, zones[::-1])  # equal-area zones mirror
    counts = np.bincount(part, minlength=P)
    assert counts.min() >= g.size // P and counts.max() <= -(-g.size // P)
    # parts are numbered band by band from north to south: grid order is
    # north to south, so the first node of each part never precedes the
    # first node of a lower-numbered band
    lat = g.lonlat()[:, 1]
    zone_of = np.repeat(np.arange(zones.size), zones)[part]
    for z in range(zones.size - 1):
        assert lat[zone_of == z].min() >= lat[zone_of == z + 1].max() - 1e-12


@pytest.mark.parametrize("P", [2, 5, 16])
def test_halo_is_the_one_ring_of_the_owned_nodes(P):
    g = nabla.Grid(24)
    m = nabla.Mesh(g, 1)
    part = nabla.equal_regions(g, P)[0][m.permutation()]  # functionspace order
    rp, nbr = m.csr()
    seen = np.zeros(m.V, dtype=int)
    for p in range(P):
        owned, halo = nabla.partition_halo(m, part, p)
        assert np.array_equal(owned, np.flatnonzero(part == p))
        ring = set()
        for i in owned:
            ring.update(nbr[rp[i]:rp[i + 1]].tolist())
        assert set(halo.tolist()) == ring - set(owned.tolist())
        assert np.all(np.diff(halo) > 0)
        seen[owned] += 1
    assert np.all(seen == 1)


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N = 16
        g = nabla.Grid(N)
        m = nabla.Mesh(g, 1)
        perm = m.permutation()  # functionspace -> grid index
        part = nabla.equal_regions(g, world)[0]  # grid order
        part_fs = part[perm]
        owned, halo = nabla.partition_halo(m, part_fs, rank)
        owned_g, halo_g = perm[owned], perm[halo]  # grid ids
        om = oracle.build_mesh(N)
        rng = np.random.default_rng(7)
        f_global = rng.standard_normal(om.V)
        # this rank starts with its owned values only
        f = np.full(om.V, np.nan)
        f[owned_g] = f_global[owned_g]
        # halo exchange: every rank learns the others' halos, then sends the
        # values it owns that they need
        halos = [None] * world
        dist.all_gather_object(halos, halo_g.tolist())
        mine = set(owned_g.tolist())
        reqs = []
        for q_ in range(world):
            if q_ == rank:
                continue
            ids = np.array([i for i in halos[q_] if i in mine], dtype=np.int64)
            reqs.append(dist.isend(torch.as_tensor(f[ids]), dst=q_))
        for q_ in range(world):
            if q_ == rank:
                continue
            ids = np.array([i for i in halo_g.tolist() if part[i] == q_], dtype=np.int64)
            buf = torch.empty(ids.size, dtype=torch.float64)
            dist.recv(buf, src=q_)
            f[ids] = buf.numpy()
        for r in reqs:
            r.wait()
        got = oracle.grad(om, f)[owned_g, 0, :]
        ref = oracle.grad(om, f_global)[owned_g, 0, :]
        q.put((rank, bool(np.isfinite(got).all()), bool(np.array_equal(got, ref)), int(halo_g.size)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,port", [(2, 29521), (4, 29525)])
def test_gloo_halo_exchange_reproduces_the_global_gradient(world, port):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = [q.get(timeout=5) for _ in range(world)]
    assert all(finite and equal and nh > 0 for _, finite, equal, nh in got), got
