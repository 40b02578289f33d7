"""Failure detection without a GPU fault: the persistent sweep's bounded wait
gives up on a flag that nothing releases (WAVE_ERR_TIMEOUT, the context stays
usable), returns at once on a released flag, stops early on the abort word;
an undersized workspace is refused before any device work."""
import time

import numpy as np
import pytest
import torch

from paper_2304_05592_gb300 import synth, wave
from paper_2304_05592_gb300.wave import Grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def ints(*v):
    return torch.tensor(v, dtype=torch.int32, device="cuda")


def test_wait_that_nobody_releases_times_out_and_context_survives():
    flag, abort_word, err = ints(0), ints(0), ints(0)
    t = time.perf_counter()
    st = wave.wave_wait_probe(flag, 1, abort_word, err)
    el = time.perf_counter() - t
    assert st == 6 and int(err.item()) != 0  # WAVE_ERR_TIMEOUT
    assert el < 60.0
    # the context is still usable: a small forward run succeeds
    p = synth.small_2d(3, nt=60)
    q = wave.wave_ricker(p.f0, p.dt, p.nt)[None, :, None].repeat(p.nshot, 1, 1).contiguous()
    d = wave.wave_forward(Grid.of(p), torch.from_numpy(p.vel).cuda(), p.src, q, p.rec)
    assert torch.isfinite(d).all()


def test_released_flag_and_abort_word():
    assert wave.wave_wait_probe(ints(3), 3, ints(0), ints(0)) == 0
    t = time.perf_counter()
    assert wave.wave_wait_probe(ints(0), 1, ints(1), ints(0)) == 6
    assert time.perf_counter() - t < 5.0


def test_undersized_workspace_is_refused():
    # through the C entry point (the Python binding would allocate a larger one)
    import ctypes

    p = synth.small_2d(4, nt=80)
    g = Grid.of(p)
    q = wave.wave_ricker(p.f0, p.dt, p.nt)[None, :, None].repeat(p.nshot, 1, 1).contiguous()
    need = wave.wave_workspace_size(g, wave.OP_GRADIENT, p.src, p.rec, wave.STORE_CHECKPOINT, 4)
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    vel = torch.from_numpy(p.vel).cuda()
    d_obs = torch.zeros((p.nshot, p.nt, p.rec.shape[1]), dtype=torch.float32, device="cuda")
    grad = torch.full(g.phys_shape, 7.0, device="cuda")
    src = np.ascontiguousarray(p.src, np.float32)
    rec = np.ascontiguousarray(p.rec, np.float32)
    phi = ctypes.c_double(0.0)
    gc = g.c()
    st = wave._lib().wave_gradient(ctypes.byref(gc), vel.data_ptr(), p.nshot, 1, src.ctypes.data, q.data_ptr(),
                                   rec.shape[1], rec.ctypes.data, d_obs.data_ptr(), grad.data_ptr(), None,
                                   ctypes.byref(phi), wave.STORE_CHECKPOINT, 4, wave.WRT_SLOWNESS2,
                                   small.data_ptr(), small.numel(), None)
    assert st == 4  # WAVE_ERR_WORKSPACE, outputs untouched
    assert bool((grad == 7.0).all())
