"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function that include/*.h declares, and its host-only entry points
(workspace sizing, geometry validation, stability limit, checkpoint schedule)
behave as documented."""
import ctypes
import os
import re
from functools import lru_cache

import numpy as np
import pytest

import oracle
from paper_2304_05592_gb300 import synth, wave

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2304_05592_gb300 import build

    build.build()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:wave_status_t|double|long long|int|size_t|const char\*)\s+((?:wave|fno)_\w+)\s*\(",
                                text, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert {"wave_forward", "wave_adjoint", "wave_gradient", "wave_workspace_size", "fno_combine", "fno_dft_x",
            "fno_mix_backward", "fno_wgrad_work_floats"} <= set(names)
    lib = ctypes.CDLL(wave.library_path())
    for n in names:
        assert hasattr(lib, n), n


def test_fno_entry_points_reject_bad_sizes_before_any_launch():
    """Argument checks of the FNO calls run on the host: a size outside the
    documented limits returns WAVE_ERR_ARG, and an empty batch returns WAVE_OK,
    without touching the (fake, never dereferenced) device pointers."""
    from paper_2304_05592_gb300 import fno

    lib = fno._lib()
    P = ctypes.c_void_p
    fake = P(0x1000)
    ARG, OK = 1, 0
    # fno_project(B, Ci, H, Nz, Nx, in, in_bf16, Q1, q1, Q2, q2, out, stream)
    assert lib.fno_project(-1, 32, 64, 8, 8, fake, 1, fake, fake, fake, fake, fake, None) == ARG
    assert lib.fno_project(2, 65, 64, 8, 8, fake, 1, fake, fake, fake, fake, fake, None) == ARG
    assert lib.fno_project(2, 32, 0, 8, 8, fake, 1, fake, fake, fake, fake, fake, None) == ARG
    assert lib.fno_project(2, 32, 64, 8, 8, fake, 1, None, fake, fake, fake, fake, None) == ARG
    assert lib.fno_project(0, 32, 64, 8, 8, fake, 1, fake, None, fake, None, fake, None) == OK
    # fno_mix_idft_z(B, Ci, Co, Nz, mz, mx, X, R, tz, out, stream): mx <= 16, 2 mz <= Nz
    assert lib.fno_mix_idft_z(2, 32, 32, 256, 16, 17, fake, fake, fake, fake, None) == ARG
    assert lib.fno_mix_idft_z(2, 32, 32, 30, 16, 16, fake, fake, fake, fake, None) == ARG
    assert lib.fno_mix_idft_z(2, 65, 32, 256, 16, 16, fake, fake, fake, fake, None) == ARG
    assert lib.fno_mix_idft_z(0, 32, 32, 256, 16, 16, fake, fake, fake, fake, None) == OK
    # fno_combine(B, Ci, Co, Nz, Nx, mx, in, in_bf16, M, m_trans, bias, T, table, act, pre, out, out_bf16, stream)
    assert lib.fno_combine(2, 32, 65, 8, 8, 1, fake, 1, fake, 0, None, None, None, 0, None, fake, 1, None) == ARG
    assert lib.fno_combine(2, 32, 32, 8, 8, 17, fake, 1, fake, 0, None, fake, fake, 0, None, fake, 1, None) == ARG
    assert lib.fno_combine(2, 32, 32, 8, 8, 1, fake, 1, fake, 0, None, None, None, 7, None, fake, 1, None) == ARG
    assert lib.fno_combine(0, 32, 32, 8, 8, 1, fake, 1, fake, 0, None, None, None, 1, None, fake, 1, None) == OK
    # fno_dft_x(rows, Nx, mx, in, in_bf16, table, out, stream)
    assert lib.fno_dft_x(10, 64, 0, fake, 1, fake, fake, None) == ARG
    assert lib.fno_dft_x(0, 64, 16, fake, 1, fake, fake, None) == OK
    assert lib.fno_set_tensor_cores(2) == ARG
    assert lib.fno_wgrad_work_floats(-1, 32, 32, 100) == 0


def test_courant_limit_matches_oracle():
    for nd in (2, 3):
        assert abs(wave.wave_courant_limit(nd) - oracle.courant_limit(nd)) < 1e-12
    assert wave.wave_courant_limit(4) == 0.0


def _grid(p, **kw):
    return wave.Grid.of(p) if not kw else wave.Grid(**{**wave.Grid.of(p).__dict__, **kw})


def test_workspace_grows_with_store_and_snapshots():
    p = synth.small_2d(1, nt=200)
    g = _grid(p)
    f = wave.wave_workspace_size(g, wave.OP_FORWARD, p.src, p.rec)
    a = wave.wave_workspace_size(g, wave.OP_ADJOINT, p.src, p.rec)
    c4 = wave.wave_workspace_size(g, wave.OP_GRADIENT, p.src, p.rec, wave.STORE_CHECKPOINT, 4)
    c8 = wave.wave_workspace_size(g, wave.OP_GRADIENT, p.src, p.rec, wave.STORE_CHECKPOINT, 8)
    b16 = wave.wave_workspace_size(g, wave.OP_GRADIENT, p.src, p.rec, wave.STORE_BF16)
    f32 = wave.wave_workspace_size(g, wave.OP_GRADIENT, p.src, p.rec, wave.STORE_FP32)
    assert 0 < f and 0 < a < c4 < c8 < b16 < f32
    # padded fields: (nz+2nb) x pitch(nx+2nb) floats per shot
    cell = (p.nz + 2 * p.nb) * ((p.nx + 2 * p.nb + 31) // 32 * 32)
    assert f32 - b16 >= p.nt * p.nshot * cell * 2 - 4096  # up to alignment padding


def test_geometry_outside_grid_is_rejected_before_launch():
    p = synth.small_2d(2, nt=50)
    g = _grid(p)
    rec = p.rec.copy()
    rec[1, 3, 0] = (p.nx - 1) * p.h + 0.5
    with pytest.raises(wave.WaveError) as e:
        wave.wave_workspace_size(g, wave.OP_FORWARD, p.src, rec)
    assert e.value.status == 3
    rec[1, 3, 0] = (p.nx - 1) * p.h
    wave.wave_workspace_size(g, wave.OP_FORWARD, p.src, rec)
    src = p.src.copy()
    src[0, 0, 1] = -1.0
    with pytest.raises(wave.WaveError) as e:
        wave.wave_workspace_size(g, wave.OP_FORWARD, src, p.rec)
    assert e.value.status == 3


@pytest.mark.parametrize("bad", [dict(ndim=4), dict(nx=1), dict(nt=0), dict(h=0.0), dict(dt=-1.0),
                                 dict(nb=-1), dict(vref=float("nan"))])
def test_bad_grid_is_rejected(bad):
    p = synth.small_2d(3, nt=20)
    g = wave.Grid(**{**wave.Grid.of(p).__dict__, **bad})
    if "ndim" in bad:
        src = np.zeros(p.src.shape[:2] + (4,), np.float32)
        rec = np.zeros(p.rec.shape[:2] + (4,), np.float32)
    else:
        src, rec = p.src, p.rec
    with pytest.raises(wave.WaveError) as e:
        wave.wave_workspace_size(g, wave.OP_FORWARD, src, rec)
    assert e.value.status == 1


def test_bad_store_mode_is_rejected():
    p = synth.small_2d(3, nt=20)
    g = _grid(p)
    with pytest.raises(wave.WaveError):
        wave.wave_workspace_size(g, wave.OP_GRADIENT, p.src, p.rec, 7, 4)
    with pytest.raises(wave.WaveError):
        wave.wave_workspace_size(g, wave.OP_GRADIENT, p.src, p.rec, wave.STORE_CHECKPOINT, 0)


def test_cuda_calls_reject_host_tensors():
    import torch

    p = synth.small_2d(3, nt=20)
    with pytest.raises(TypeError):
        wave.wave_forward(_grid(p), torch.from_numpy(p.vel), p.src, torch.zeros(p.nshot, p.nt, 1), p.rec)


# ---------------------------------------------------------------------------
# Binomial checkpoint schedule.


@lru_cache(None)
def best_cost(l, s):
    """Fewest macro advances to run the adjoint pairs of positions a+l .. a
    with the state at a restorable and s free slots (exhaustive over every
    split point; a snapshot at a position serves that position)."""
    if l == 0:
        return 0
    if s == 0:
        return l * (l + 1) // 2
    return min(m + best_cost(l - m, s - 1) + best_cost(m - 1, s) for m in range(1, l + 1))


def simulate(nt, nsnap, acts):
    """Replays the action list on symbolic states and returns the adjoint
    steps in execution order with the time level each one was given."""
    K = nt - 1
    state = 0  # W holds (u^state, u^{state-1})
    slots = {}
    recorded = set()
    done = []
    finalized = False
    fwd = 0
    for kind, arg, st in acts:
        if kind == 0:
            assert arg == state
            for n in range(state, st):
                recorded.add(n)
                fwd += 1
            state = st
        elif kind == 1:
            assert 0 <= arg < max(1, nsnap)
            slots[arg] = state
            assert st == state
        elif kind == 2:
            state = 0 if arg == -1 else slots[arg]
            assert st == state
        elif kind == 3:
            assert finalized and arg == state
            done.append((state, state))
            if state - 1 >= 1:
                done.append((state - 1, state))
        elif kind == 4:
            assert recorded == set(range(K))
            finalized = True
    return done, fwd


@pytest.mark.parametrize("nt,nsnap", [(2, 1), (3, 1), (4, 1), (5, 2), (12, 1), (40, 3), (41, 3), (101, 5),
                                      (200, 64), (1000, 20)])
def test_schedule_reverses_every_step_in_order(nt, nsnap):
    steps, acts = wave.wave_checkpoint_schedule(nt, nsnap)
    done, fwd = simulate(nt, nsnap, acts.tolist())
    K = nt - 1
    assert [k for k, _ in done] == list(range(K, 0, -1))
    # each adjoint step k reads u^k from a state that holds it
    assert all(st == k or st == k + 1 for k, st in done)
    assert fwd == steps


@pytest.mark.parametrize("nt,nsnap", [(9, 1), (21, 2), (41, 3), (61, 4), (81, 2)])
def test_schedule_is_optimal_for_its_cost_model(nt, nsnap):
    steps, acts = wave.wave_checkpoint_schedule(nt, nsnap)
    K = nt - 1
    jmin = 1 if K % 2 else 2
    L = (K - jmin) // 2 + 1
    s = max(0, min(nsnap, L))
    # a macro advance between positions a < b covers state(b) - state(a) steps:
    # 2 per position, jmin for the first one
    macro = 0
    for kind, a, b in acts.tolist():
        if kind == 0:
            pa = 0 if a == 0 else (a - jmin) // 2 + 1
            pb = (b - jmin) // 2 + 1
            macro += pb - pa
    assert macro == best_cost(L, s)


def test_schedule_sweeps_shrink_with_slots():
    K = 3999
    full, _ = wave.wave_checkpoint_schedule(4000, 2000)
    assert full == K  # one slot per pair of steps: a single forward sweep
    many, _ = wave.wave_checkpoint_schedule(4000, 400)
    few, _ = wave.wave_checkpoint_schedule(4000, 20)
    assert K < many < 2 * K < few
