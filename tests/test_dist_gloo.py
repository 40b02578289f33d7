"""Shot sharding and the gradient all-reduce across ranks, run as two gloo
processes on the CPU with the FP64 oracle as the per-rank solver: the summed
gradient and misfit equal the oracle's over all shots at once, including a
rank that owns no shot."""
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2304_05592_gb300 import dist as wdist
from paper_2304_05592_gb300 import synth


def test_shard_ranges_cover_the_survey_once():
    for nshot in (0, 1, 5, 32, 33):
        for world in (1, 2, 3, 8):
            got = [list(wdist.shard(nshot, r, world)) for r in range(world)]
            assert sum(got, []) == list(range(nshot))
            sizes = [len(g) for g in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        wdist.shard(4, 2, 2)


def _problem(nshot):
    p = synth.small_2d(21, nt=120, nshot=nshot)
    g = oracle.Grid(p.ndim, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, vref=p.vref)
    q = np.repeat(oracle.ricker(p.f0, p.dt, p.nt)[None, :, None], p.nshot, axis=0)
    d_obs = synth.observed_noise((p.nshot, p.nt, p.rec.shape[1]), 1e-3, 5).astype(np.float64)
    return p, g, q, d_obs


def _rank(rank, world, port, nshot, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    p, g, q, d_obs = _problem(nshot)

    def grad_fn(shots):
        idx = list(shots)
        if not idx:
            return 0.0, torch.zeros((p.nz, p.nx), dtype=torch.float64)
        phi, gr = oracle.gradient(g, p.vel, p.src[idx], q[idx], p.rec[idx], d_obs[idx])
        return phi, torch.from_numpy(np.asarray(gr, np.float64))

    phi, gsum = wdist.sharded_gradient(grad_fn, nshot)
    if rank == 0:
        out.put((phi, gsum.numpy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("nshot", [3, 1])
def test_two_ranks_sum_to_the_all_shot_gradient(nshot):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, nshot, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    phi, gsum = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, g, qq, d_obs = _problem(nshot)
    phi_ref, g_ref = oracle.gradient(g, p.vel, p.src, qq, p.rec, d_obs)
    assert abs(phi - phi_ref) <= 1e-12 * abs(phi_ref)
    assert np.linalg.norm(gsum - g_ref) <= 1e-12 * np.linalg.norm(g_ref)
