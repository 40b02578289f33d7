"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: the 32-shot config-2 gradient (one batched call, checkpointed, nt =
4000) is checked on sampled outputs the oracle computes one by one (records of
sampled shots, gradients of sampled shots), plus linearity of the shot sum;
config 3 runs on its full 480 x 480 x 380 padded grid with a shortened record."""
import numpy as np
import pytest
import torch

import oracle
from paper_2304_05592_gb300 import synth, wave
from paper_2304_05592_gb300.wave import Grid

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
def config2():
    from scipy.ndimage import gaussian_filter

    p = synth.config2()
    v0 = gaussian_filter(p.vel.astype(np.float64), 8.0).astype(np.float32)
    dev = torch.device("cuda")
    q1 = oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)
    wav = torch.from_numpy(np.repeat(q1[None, :, None], p.nshot, axis=0)).to(dev)
    g = Grid.of(p)
    d_obs = wave.wave_forward(g, torch.from_numpy(p.vel).to(dev), p.src, wav, p.rec)
    phi, grad, dsyn = wave.wave_gradient(g, torch.from_numpy(v0).to(dev), p.src, wav, p.rec, d_obs,
                                         store=wave.STORE_CHECKPOINT, nsnap=256, want_dsyn=True)
    return dict(p=p, v0=v0, q1=q1, wav=wav, d_obs=d_obs, phi=phi, grad=grad.cpu().numpy(),
                dsyn=dsyn.cpu().numpy())


def test_config2_records_of_sampled_shots(config2):
    p, v0, q1 = config2["p"], config2["v0"], config2["q1"]
    for s in (0, 13, 31):
        ref = oracle.forward(ogrid(p), v0, p.src[s:s + 1], q1[None, :, None], p.rec[s:s + 1])[0]
        assert rel(config2["dsyn"][s], ref) < 1e-4, s


def test_config2_batched_gradient_is_the_sum_of_shot_gradients(config2):
    p, v0 = config2["p"], config2["v0"]
    dev = torch.device("cuda")
    g = Grid.of(p)
    total = np.zeros_like(config2["grad"], dtype=np.float64)
    phis = 0.0
    vel = torch.from_numpy(v0).to(dev)
    for s in range(p.nshot):
        phi, gs, _ = wave.wave_gradient(g, vel, p.src[s:s + 1], config2["wav"][s:s + 1], p.rec[s:s + 1],
                                        config2["d_obs"][s:s + 1].contiguous(), nsnap=256)
        total += gs.cpu().numpy()
        phis += phi
    assert rel(config2["grad"], total) < 1e-5
    assert abs(config2["phi"] - phis) <= 1e-6 * phis


@pytest.fixture(scope="module")
def config2_oracle(config2):
    """Observed data of two sampled shots modelled by the oracle on the true
    model, and the oracle's misfit and gradient of each at the starting model."""
    p, v0, q1 = config2["p"], config2["v0"], config2["q1"]
    out = {}
    for s in (5, 26):
        d_obs = oracle.forward(ogrid(p), p.vel, p.src[s:s + 1], q1[None, :, None], p.rec[s:s + 1])
        phi_r, g_r = oracle.gradient(ogrid(p), v0, p.src[s:s + 1], q1[None, :, None], p.rec[s:s + 1], d_obs)
        out[s] = (d_obs, phi_r, g_r)
    return out


def _shot_gradient(config2, s, d_obs, store):
    p = config2["p"]
    dev = torch.device("cuda")
    vel = torch.from_numpy(config2["v0"]).to(dev)
    dd = torch.from_numpy(d_obs.astype(np.float32)).to(dev)
    return wave.wave_gradient(Grid.of(p), vel, p.src[s:s + 1], config2["wav"][s:s + 1], p.rec[s:s + 1], dd,
                              store=store, nsnap=256)


def test_config2_gradient_of_sampled_shots_matches_oracle(config2, config2_oracle):
    for s, (d_obs, phi_r, g_r) in config2_oracle.items():
        phi, gs, _ = _shot_gradient(config2, s, d_obs, wave.STORE_CHECKPOINT)
        assert abs(phi - phi_r) <= 1e-4 * phi_r
        assert rel(gs.cpu().numpy(), g_r) < 1e-3, (s, rel(gs.cpu().numpy(), g_r))


def test_config2_bf16_store_error_is_stated(config2, config2_oracle):
    """The BF16 wavefield store (stencil arithmetic and accumulation stay FP32)
    changes the gradient by a stated amount: against the FP64 oracle on two
    sampled shots of the benchmark survey, and against the FP32 checkpointed
    gradient of the whole 32-shot batch.  Both must stay below 1e-2."""
    errs = {}
    for s, (d_obs, phi_r, g_r) in config2_oracle.items():
        phi, g16, _ = _shot_gradient(config2, s, d_obs, wave.STORE_BF16)
        _, g32, _ = _shot_gradient(config2, s, d_obs, wave.STORE_CHECKPOINT)
        errs[s] = (rel(g16.cpu().numpy(), g_r), rel(g32.cpu().numpy(), g_r))
        assert abs(phi - phi_r) <= 1e-4 * phi_r
    for s, (e16, e32) in errs.items():
        print(f"config 2 shot {s}: gradient rel L2 vs FP64 oracle: BF16 store {e16:.3e}, "
              f"FP32 checkpointed {e32:.3e}")
    assert max(e for e, _ in errs.values()) < 1e-2
    p = config2["p"]
    dev = torch.device("cuda")
    _, g16, _ = wave.wave_gradient(Grid.of(p), torch.from_numpy(config2["v0"]).to(dev), p.src, config2["wav"],
                                   p.rec, config2["d_obs"], store=wave.STORE_BF16)
    e = rel(g16.cpu().numpy(), config2["grad"].astype(np.float64))
    print(f"config 2, 32 shots: BF16 store vs FP32 checkpointed gradient: rel L2 {e:.3e}")
    assert e < 1e-2


def test_config3_full_grid_short_record():
    p = synth.config3(nt=150)
    q1 = oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)
    dev = torch.device("cuda")
    d = wave.wave_forward(Grid.of(p), torch.from_numpy(p.vel).to(dev), p.src,
                          torch.from_numpy(q1[None, :, None].copy()).to(dev), p.rec).cpu().numpy()
    ref = oracle.forward(ogrid(p), p.vel, p.src, q1[None, :, None], p.rec)
    assert np.abs(ref).max() > 0
    assert rel(d, ref) < 1e-4, rel(d, ref)
