"""Uneven batch (one persistent forward sweep and one persistent adjoint sweep
over problems of different sizes, models and time axes): every problem's
gradient and misfit equal a separate single-shot call and the oracle; graph
replay equals the eager path; the autograd wrapper returns the same
gradients."""
import numpy as np
import pytest
import torch

import oracle
from paper_2304_05592_gb300 import synth, wave
from paper_2304_05592_gb300.autograd import batch_misfit
from paper_2304_05592_gb300.wave import BatchProblem, Grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def rel(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ogrid(p):
    return oracle.Grid(p.ndim, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, ny=p.ny, vref=p.vref)


@pytest.fixture(scope="module")
def batch():
    probs = synth.uneven_batch(seed=11, nshot=6, scale=0.12)
    out = []
    for p in probs:
        q = oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)
        dobs = oracle.forward(ogrid(p), p.vel, p.src, q[None, :, None], p.rec)[0].astype(np.float32)
        v0 = (p.vel * 1.03).astype(np.float32)
        out.append((p, q, dobs, v0))
    return out


def _problems(batch):
    return [BatchProblem(Grid.of(p), torch.from_numpy(v0).cuda(), p.src[0], torch.from_numpy(q[:, None]).cuda(),
                         p.rec[0], torch.from_numpy(dobs).cuda()) for p, q, dobs, v0 in batch]


@pytest.mark.parametrize("store", [wave.STORE_FP32, wave.STORE_BF16])
def test_batch_matches_single_shot_calls_and_oracle(batch, store):
    probs = _problems(batch)
    misfits, grads = wave.wave_gradient_batch(probs, store=store, use_graph=False)
    assert len({p.nt for p, *_ in batch}) > 1 and len({(p.nx, p.nz) for p, *_ in batch}) > 1
    for (p, q, dobs, v0), bp, phi, gr in zip(batch, probs, misfits, grads):
        phi1, g1, _ = wave.wave_gradient(Grid.of(p), bp.vel, p.src, bp.wavelet[None].contiguous(), p.rec,
                                         bp.d_obs[None].contiguous(), store=store)
        assert abs(phi - phi1) <= 1e-6 * phi1
        assert float((gr - g1).norm() / g1.norm()) < 1e-5
        phi_r, g_r = oracle.gradient(ogrid(p), v0, p.src, q[None, :, None], p.rec, dobs)
        # the misfit is quadratic in records that match to 1e-4
        assert abs(phi - phi_r) <= 3e-4 * phi_r
        assert rel(gr.cpu().numpy(), g_r) < (1e-3 if store == wave.STORE_FP32 else 1e-2)


def test_graph_replay_equals_eager(batch):
    probs = _problems(batch)
    ws = wave.wave_workspace_size_batch(probs, wave.STORE_BF16)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    m0, g0 = wave.wave_gradient_batch(probs, use_graph=False, work=work)
    for _ in range(2):  # capture, then replay
        m1, g1 = wave.wave_gradient_batch(probs, use_graph=True, work=work)
        assert m1 == m0
        assert all(torch.equal(a, b) for a, b in zip(g0, g1))


def test_batch_autograd(batch):
    probs = _problems(batch)
    for bp in probs:
        bp.vel.requires_grad_(True)
    loss = batch_misfit(probs).sum()
    loss.backward()
    _, gv = wave.wave_gradient_batch(probs, wrt=wave.WRT_VELOCITY, use_graph=False)
    for bp, g in zip(probs, gv):
        assert float((bp.vel.grad - g).norm() / g.norm()) < 1e-6


@pytest.fixture(scope="module")
def wide_batch():
    # grids of 1-2 tiles across and 3-9 tile rows of 16 (ragged both ways), nt 687-1160
    probs = synth.uneven_batch(seed=12, nshot=4, scale=0.3)
    out = []
    for p in probs:
        q = oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)
        dobs = oracle.forward(ogrid(p), p.vel, p.src, q[None, :, None], p.rec)[0].astype(np.float32)
        v0 = (p.vel * 1.03).astype(np.float32)
        phi_r, g_r = oracle.gradient(ogrid(p), v0, p.src, q[None, :, None], p.rec, dobs)
        out.append((p, q, dobs, v0, phi_r, g_r))
    return out


@pytest.fixture
def restore_batch_variant():
    yield
    wave.wave_set_batch_variant(-1, -1)


def test_every_sweep_variant_matches_oracle(wide_batch, restore_batch_variant):
    """Each sweep kernel (direct loads; TMA producer/consumer with 16- or
    32-row tiles, 2-8 consumer warps, 2-3 stages) gives the oracle's misfits
    and gradients, and all of them agree to rounding of the imaging sums."""
    assert any(p.nx + 2 * p.nb > 128 for p, *_ in wide_batch)  # two tile columns or more
    probs = _problems([b[:4] for b in wide_batch])
    base = None
    for v in range(wave.wave_batch_variant_count()):
        wave.wave_set_batch_variant(v, v)
        misfits, grads = wave.wave_gradient_batch(probs, store=wave.STORE_FP32, use_graph=False)
        for (p, q, dobs, v0, phi_r, g_r), phi, gr in zip(wide_batch, misfits, grads):
            assert abs(phi - phi_r) <= 3e-4 * phi_r, (v, phi, phi_r)
            assert rel(gr.cpu().numpy(), g_r) < 1e-3, (v, rel(gr.cpu().numpy(), g_r))
        if base is None:
            base = grads
        else:
            for a, b in zip(grads, base):
                assert float((a - b).norm() / b.norm()) < 1e-5, v


def test_autotuned_batch_matches_oracle_bf16(wide_batch, restore_batch_variant):
    probs = _problems([b[:4] for b in wide_batch])
    vf, va = wave.wave_autotune_batch(probs, store=wave.STORE_BF16, steps=50)
    n = wave.wave_batch_variant_count()
    assert 0 <= vf < n and 0 <= va < n
    misfits, grads = wave.wave_gradient_batch(probs, store=wave.STORE_BF16)
    errs = []
    for (p, q, dobs, v0, phi_r, g_r), phi, gr in zip(wide_batch, misfits, grads):
        assert abs(phi - phi_r) <= 3e-4 * phi_r
        errs.append(rel(gr.cpu().numpy(), g_r))
    print(f"uneven batch, BF16 store, sweeps {vf}/{va}: gradient rel L2 vs oracle {errs}")
    assert max(errs) < 1e-2


def test_more_tiles_than_ctas_matches_single_shot_calls(restore_batch_variant):
    """A batch with several tiles per CTA (sweep variant 10: one CTA per SM), so
    that the host's cost-balanced round-robin order is in play: misfits and
    gradients equal one wave_gradient call per problem."""
    probs_s = synth.uneven_batch(seed=13, nshot=12, scale=0.45)
    probs = []
    for p in probs_s:
        q = torch.from_numpy(oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)[:, None]).cuda()
        v = torch.from_numpy(p.vel).cuda()
        dob = wave.wave_forward(Grid.of(p), v, p.src, q[None].contiguous(), p.rec)[0].contiguous()
        probs.append(BatchProblem(Grid.of(p), (v * 1.03).contiguous(), p.src[0], q, p.rec[0], dob))
    ntile = sum(-(-(p.nx + 2 * p.nb) // 128) * -(-(p.nz + 2 * p.nb) // 16) for p in probs_s)
    assert ntile > torch.cuda.get_device_properties(0).multi_processor_count  # several tiles per CTA
    wave.wave_set_batch_variant(10, 10)
    misfits, grads = wave.wave_gradient_batch(probs, store=wave.STORE_FP32, use_graph=False)
    for p, bp, phi, gr in zip(probs_s, probs, misfits, grads):
        phi1, g1, _ = wave.wave_gradient(Grid.of(p), bp.vel, p.src, bp.wavelet[None].contiguous(), p.rec,
                                         bp.d_obs[None].contiguous(), store=wave.STORE_FP32)
        assert abs(phi - phi1) <= 1e-6 * phi1
        assert float((gr - g1).norm() / g1.norm()) < 1e-5


def test_forced_variant_pair_must_share_tile_height(restore_batch_variant):
    with pytest.raises(wave.WaveError):
        wave.wave_set_batch_variant(0, 1)  # 32-row against 16-row tiles
    with pytest.raises(wave.WaveError):
        wave.wave_set_batch_variant(wave.wave_batch_variant_count(), 0)
