"""Multi-rank host path on CPU (gloo, world size 2): positions shard into contiguous
ranges with no collective on the data path; the ranks' packed outputs, gathered in
rank order, equal one single-process evaluation.  The per-rank compute here is the
FP64 oracle (no GPU in this test)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import obsgen
from paper_2009_07010_gb300 import shard


def test_shard_ranges_partition_and_balance():
    npix = np.array([32, 256, 64, 64, 128, 32, 256, 32], np.int32)
    for world in (1, 2, 3, 5, 8, 11):
        rs = shard.shard_ranges(npix, world)
        assert rs[0][0] == 0 and rs[-1][1] == len(npix)
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        assert all(a <= b for a, b in rs)
    rs = shard.shard_ranges(np.full(100, 64), 4)
    assert [b - a for a, b in rs] == [25, 25, 25, 25]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    obs = obsgen.tiny_obs(nant=4, ntime=12, nchan=4, tavg=3, favg=2)
    full = obsgen.random_batch(4, 7, sizes=(4, 6, 8))
    lm, npix, first = shard.shard(full.lm, full.npix, rank, world)
    out = oracle.psf(obs, oracle.EXACT, obsgen.Batch(lm, npix, full.cell_rad)) if len(npix) else np.zeros(0)
    parts = [None] * world
    dist.all_gather_object(parts, (first, out))
    if rank == 0:
        q.put(parts)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reassemble_single_process_result():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    import oracle
    obs = obsgen.tiny_obs(nant=4, ntime=12, nchan=4, tavg=3, favg=2)
    full = obsgen.random_batch(4, 7, sizes=(4, 6, 8))
    ref = oracle.psf(obs, oracle.EXACT, full)
    got = np.concatenate([p[1] for p in sorted(parts, key=lambda x: x[0])])
    assert got.shape == ref.shape
    np.testing.assert_array_equal(got, ref)


# ---- CLEAN by facets: each facet image is cleaned on its own, so facets shard like positions

def _facets():
    """Four 48 x 48 facets of a field centred on (0.01, 0.005), one source each, on the
    small array; the facet-centre PSF serves every component of a facet."""
    obs = obsgen.tiny_obs(weights=True)
    cell, N, nf = 3e-5, 16, 48
    centres = [(0.01 + dx * nf * cell, 0.005 + dy * nf * cell) for dy in (-0.5, 0.5) for dx in (-0.5, 0.5)]
    srcs = [(20, 22, 1.0), (27, 25, 0.8), (24, 19, 0.9), (22, 26, 0.7)]
    return obs, cell, N, nf, centres, srcs


def _clean_facet(f):
    import oracle
    obs, cell, N, nf, centres, srcs = _facets()
    x, y, c = srcs[f]
    l0, m0 = centres[f][0] + (x - nf // 2) * cell, centres[f][1] + (y - nf // 2) * cell
    b = obsgen.Batch(np.array([[l0, m0]]), np.array([N], np.int32), cell)
    P = oracle.psf(obs, oracle.UV, b).reshape(N, N)
    d = np.zeros((nf, nf))
    d[y - N // 2:y + N // 2, x - N // 2:x + N // 2] = c * P / P[N // 2, N // 2]
    res, model, comps = oracle.clean(obs, "uv", d, cell, N, 0.3, 0.1, 50, centre=centres[f], facet_psf=True)
    return res, comps


def _facet_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b = shard.shard_ranges(np.full(4, 48), world)[rank]
    mine = [(f, _clean_facet(f)) for f in range(a, b)]
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    if rank == 0:
        q.put(parts)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_clean_facets_like_one_process():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_facet_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(item for part in parts for item in part)
    assert sorted(got) == [0, 1, 2, 3]
    for f in range(4):
        res, comps = _clean_facet(f)
        np.testing.assert_array_equal(got[f][0], res)
        assert got[f][1] == comps and len(comps) > 1
