"""GPU FNO kernels against the FP64 oracle: each transform, the mode mix and
its backward, the whole network forward and backward (small case and the full
512x256, width-32, 16x16-mode network), BF16 inference, MSE, Adam, and
repeatability of the gradients."""
import numpy as np
import pytest
import torch

from oracle import fno as ofno
from paper_2304_05592_gb300 import fno

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(99)
# FP32 accumulation over up to Nz*Nx = 131072 terms per output: a relative
# error of a few 1e-6 per sum; 2e-5 on relative L2 norms leaves margin.
TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def rel(a, b):
    a = np.asarray(a, np.complex128 if np.iscomplexobj(b) else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def cplx(t):
    a = t.detach().cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def pack(c):
    return dev(np.stack([c.real, c.imag], axis=-1))


@pytest.mark.parametrize("Nz,Nx,mz,mx", [(24, 40, 4, 5), (256, 512, 16, 16), (37, 70, 3, 7)])
def test_tables_match_oracle(Nz, Nx, mz, mx):
    """fno_tables (double on the device, rounded to float) against the factors
    of the truncated transforms computed from their definition."""
    (tf, ti, tb, ta), tz = fno.fno_tables(Nz, Nx, mz, mx)
    for got, ref in zip((tf, ti, tb, ta, tz), ofno.twiddle_tables(Nz, Nx, mz, mx)):
        g = got.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(g[..., 0] + 1j * g[..., 1], ref, rtol=0, atol=2e-7 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(2, 3, 24, 40, 4, 5), (1, 32, 256, 512, 16, 16), (3, 2, 37, 70, 3, 7)])
def test_truncated_dft_and_inverse(shape):
    B, C, Nz, Nx, mz, mx = shape
    v = RNG.standard_normal((B, C, Nz, Nx))
    (tf, ti, tb, ta), tz = fno.fno_tables(Nz, Nx, mz, mx)
    T1 = fno.fno_dft_x(dev(v), mx, tf)
    X = fno.fno_dft_z(T1, B * C, Nz, mz, mx, tz)
    ref = ofno.dft_trunc(v, mz, mx)
    assert rel(cplx(X).reshape(ref.shape), ref) < TOL
    # inverse: S Y through the z inverse and the combine kernel (M = 0)
    Y = RNG.standard_normal(ref.shape) + 1j * RNG.standard_normal(ref.shape)
    T2 = fno.fno_idft_z(pack(Y), B * C, Nz, mz, mx, tz)
    zero = torch.zeros((C, C), dtype=torch.float32, device="cuda")
    y = fno.fno_combine(dev(np.zeros((B, C, Nz, Nx))), zero, C, T=T2, table=ti, mx=mx)
    assert rel(y.cpu().numpy(), ofno.idft_trunc(Y, Nz, Nx)) < TOL
    # the two adjoints used by the backward pass
    dy = RNG.standard_normal((B, C, Nz, Nx))
    dT2 = fno.fno_dft_x(dev(dy), mx, tb)
    dY = fno.fno_dft_z(dT2, B * C, Nz, mz, mx, tz)
    assert rel(cplx(dY).reshape(ref.shape), ofno.idft_trunc_adjoint(dy, mz, mx)) < TOL
    dT1 = fno.fno_idft_z(pack(Y), B * C, Nz, mz, mx, tz)
    dv = fno.fno_combine(dev(np.zeros((B, C, Nz, Nx))), zero, C, T=dT1, table=ta, mx=mx)
    assert rel(dv.cpu().numpy(), ofno.dft_trunc_adjoint(Y, Nz, Nx)) < TOL


@pytest.mark.parametrize("B,Ci,Co,Nz,mz,mx", [(2, 32, 32, 256, 16, 16), (3, 5, 7, 37, 3, 5), (1, 4, 64, 130, 32, 9)])
def test_fused_mix_and_inverse_z(B, Ci, Co, Nz, mz, mx):
    """fno_mix_idft_z against fno_mix followed by fno_idft_z, and against both
    sums evaluated in FP64 (einsum) with the same z table."""
    KZ = 2 * mz
    X = RNG.standard_normal((B, Ci, KZ, mx, 2))
    R = RNG.standard_normal((Ci, Co, KZ, mx, 2))
    _, tz = fno.fno_tables(Nz, 2 * mx, mz, mx)
    fused = fno.fno_mix_idft_z(dev(X), dev(R), B, Ci, Co, Nz, mz, mx, tz).cpu().numpy()
    Y = fno.fno_mix(dev(X), dev(R), B, Ci, Co, KZ * mx)
    two = fno.fno_idft_z(Y, B * Co, Nz, mz, mx, tz).cpu().numpy()
    assert rel(fused, two) < 1e-6
    Xc = X[..., 0] + 1j * X[..., 1]
    Rc = R[..., 0] + 1j * R[..., 1]
    Yc = np.einsum("biam,ioam->boam", Xc, Rc)
    Ec = ofno.twiddle_tables(Nz, 2 * mx, mz, mx)[4]  # [Nz][KZ], from the definition
    ref = np.einsum("boam,za->bozm", Yc, Ec)
    fc = fused.reshape(B, Co, Nz, mx, 2)
    assert rel(fc[..., 0] + 1j * fc[..., 1], ref) < 1e-5


@pytest.mark.parametrize("Nz,Nx,dtype", [(16, 36, torch.float32), (16, 36, torch.bfloat16), (7, 9, torch.float32)])
def test_lift_path_matches_reference(Nz, Nx, dtype):
    """fno_combine with few input channels and no spectral term (the lift; four
    pixels per thread when Nz Nx is a multiple of 4, the general kernel otherwise):
    pre-activation, GELU output and the transposed weight layout against FP64."""
    B, ci, co = 2, 3, 32
    x = RNG.standard_normal((B, ci, Nz, Nx))
    M, b = RNG.standard_normal((co, ci)), RNG.standard_normal(co)
    pre = torch.empty((B, co, Nz, Nx), dtype=torch.float32, device="cuda")
    out = fno.fno_combine(dev(x), dev(M), co, bias=dev(b), act=fno.ACT_GELU, pre=pre, out_dtype=dtype)
    ref = ofno.pointwise(M, b, x)
    assert rel(pre.cpu().numpy(), ref) < 1e-6
    assert rel(out.float().cpu().numpy(), ofno.gelu(ref)) < (1e-2 if dtype == torch.bfloat16 else 1e-6)
    outt = fno.fno_combine(dev(x), dev(np.ascontiguousarray(M.T)), co, m_trans=True, bias=dev(b))
    assert rel(outt.cpu().numpy(), ref) < 1e-6


def test_mode_mix_and_backward():
    B, Ci, Co, KZ, mx = 3, 5, 7, 8, 6
    X = RNG.standard_normal((B, Ci, KZ, mx)) + 1j * RNG.standard_normal((B, Ci, KZ, mx))
    R = RNG.standard_normal((Ci, Co, KZ, mx)) + 1j * RNG.standard_normal((Ci, Co, KZ, mx))
    dY = RNG.standard_normal((B, Co, KZ, mx)) + 1j * RNG.standard_normal((B, Co, KZ, mx))
    Y = fno.fno_mix(pack(X), pack(R), B, Ci, Co, KZ * mx)
    assert rel(cplx(Y).reshape(B, Co, KZ, mx), np.einsum("bikx,iokx->bokx", X, R)) < 1e-6
    dX = torch.empty((B, Ci, KZ, mx, 2), dtype=torch.float32, device="cuda")
    dR = torch.empty((Ci, Co, KZ, mx, 2), dtype=torch.float32, device="cuda")
    fno.fno_mix_backward(pack(X), pack(R), pack(dY), B, Ci, Co, KZ * mx, dX=dX, dR=dR)
    assert rel(cplx(dX), np.einsum("bokx,iokx->bikx", dY, np.conj(R))) < 1e-6
    assert rel(cplx(dR), np.einsum("bikx,bokx->iokx", np.conj(X), dY)) < 1e-6


def test_pointwise_gelu_and_weight_gradient():
    B, Ci, Co, Nz, Nx = 2, 6, 9, 11, 300
    x = RNG.standard_normal((B, Ci, Nz, Nx))
    M, b = RNG.standard_normal((Co, Ci)), RNG.standard_normal(Co)
    pre = torch.empty((B, Co, Nz, Nx), dtype=torch.float32, device="cuda")
    out = fno.fno_combine(dev(x), dev(M), Co, bias=dev(b), act=fno.ACT_GELU, pre=pre)
    ref = ofno.pointwise(M, b, x)
    assert rel(pre.cpu().numpy(), ref) < 1e-6
    assert rel(out.cpu().numpy(), ofno.gelu(ref)) < 1e-6
    dout = RNG.standard_normal(ref.shape)
    dpre = fno.fno_gelu_backward(dev(dout), pre)
    assert rel(dpre.cpu().numpy(), dout * ofno.gelu_grad(ref)) < 1e-6
    dM = torch.empty((Co, Ci), dtype=torch.float32, device="cuda")
    db = torch.empty(Co, dtype=torch.float32, device="cuda")
    work = torch.empty(fno.fno_wgrad_work_floats(B, Ci, Co, Nz * Nx), dtype=torch.float32, device="cuda")
    fno.fno_wgrad(dev(dout), dev(x), dM, db, work)
    gM, gb = ofno._wgrad(dout, x)
    assert rel(dM.cpu().numpy(), gM) < 1e-5 and rel(db.cpu().numpy(), gb) < 1e-5
    # the transposed matrix (used by the backward pass)
    back = fno.fno_combine(dev(ref), dev(M), Ci, m_trans=True)
    assert rel(back.cpu().numpy(), np.einsum("oi,bo...->bi...", M, ref)) < 1e-6


@pytest.mark.parametrize("Ci,Co,Nz,Nx,spectral,bf16_in", [(32, 32, 9, 300, True, False), (32, 64, 5, 260, False, False),
                                                          (17, 32, 6, 70, True, False), (32, 32, 6, 256, True, True),
                                                          (64, 64, 3, 132, True, False)])
def test_wide_channel_mix_paths(Ci, Co, Nz, Nx, spectral, bf16_in):
    """fno_combine for 32 or 64 output channels (the register-tiled kernels: rows
    marched with the next row's tile by cp.async when the input is FP32 with rows of
    a multiple of 4 pixels, one row per block otherwise), ragged 128-pixel strips
    and row groups, with and without the spectral term, against FP64."""
    B, mx = 2, 7
    x = RNG.standard_normal((B, Ci, Nz, Nx))
    M, b = RNG.standard_normal((Co, Ci)), RNG.standard_normal(Co)
    ref = ofno.pointwise(M, b, x)
    T = tab = None
    if spectral:
        Tn = RNG.standard_normal((B, Co, Nz, 2 * mx))
        tabn = RNG.standard_normal((Nx, mx, 2))
        ref = ref + np.einsum("bozk,xk->bozx", Tn[..., 0::2], tabn[..., 0]) - np.einsum(
            "bozk,xk->bozx", Tn[..., 1::2], tabn[..., 1])
        T, tab = dev(Tn), dev(tabn)
    xin = dev(x).to(torch.bfloat16) if bf16_in else dev(x)
    if bf16_in:
        ref = ofno.pointwise(M, b, xin.float().cpu().numpy().astype(np.float64)) + (ref - ofno.pointwise(M, b, x))
    pre = torch.empty((B, Co, Nz, Nx), dtype=torch.float32, device="cuda")
    fno.fno_set_tensor_cores(False)  # the CUDA-core kernels, also for BF16 inputs
    try:
        out = fno.fno_combine(xin, dev(M), Co, bias=dev(b), T=T, table=tab, mx=mx, act=fno.ACT_GELU, pre=pre)
        outt = fno.fno_combine(xin, dev(np.ascontiguousarray(M.T)), Co, m_trans=True, bias=dev(b), T=T, table=tab,
                               mx=mx)
    finally:
        fno.fno_set_tensor_cores(True)
    assert rel(pre.cpu().numpy(), ref) < 1e-6
    assert rel(out.cpu().numpy(), ofno.gelu(ref)) < 1e-6
    assert torch.equal(outt, pre)  # the same sums in the same order


@pytest.mark.parametrize("Ci,Co,Nz,Nx", [(32, 32, 13, 300), (32, 64, 7, 256), (64, 1, 9, 100), (3, 32, 5, 77)])
def test_weight_gradient_shapes(Ci, Co, Nz, Nx):
    """fno_wgrad for the network's layer shapes (and pixel counts that leave a
    ragged last tile or are not a multiple of 4) against FP64."""
    B = 3
    x, dout = RNG.standard_normal((B, Ci, Nz, Nx)), RNG.standard_normal((B, Co, Nz, Nx))
    dM = torch.empty((Co, Ci), dtype=torch.float32, device="cuda")
    db = torch.empty(Co, dtype=torch.float32, device="cuda")
    work = torch.empty(fno.fno_wgrad_work_floats(B, Ci, Co, Nz * Nx), dtype=torch.float32, device="cuda")
    fno.fno_wgrad(dev(dout), dev(x), dM, db, work)
    gM, gb = ofno._wgrad(dout, x)
    assert rel(dM.cpu().numpy(), gM) < 1e-5 and rel(db.cpu().numpy(), gb) < 1e-5
    dM2 = torch.empty_like(dM)
    db2 = torch.empty_like(db)
    fno.fno_wgrad(dev(dout), dev(x), dM2, db2, work)
    assert torch.equal(dM, dM2) and torch.equal(db, db2)


def _net(cfg, Nz, Nx, B, seed):
    p = ofno.init_params(ofno.Config(**cfg.__dict__), seed)
    net = fno.FNO2d(cfg, Nz, Nx, seed=seed)
    net.load(p)
    x = RNG.standard_normal((B, cfg.cin, Nz, Nx))
    t = RNG.standard_normal((B, 1, Nz, Nx))
    return p, net, x, t


@pytest.mark.parametrize("cfg,Nz,Nx,B", [
    (fno.FNOConfig(cin=3, width=8, hidden=12, layers=3, mz=4, mx=5), 32, 48, 2),
    (fno.FNOConfig(), 256, 512, 2),
])
def test_network_forward_backward_match_oracle(cfg, Nz, Nx, B):
    p, net, x, t = _net(cfg, Nz, Nx, B, seed=3)
    ocfg = ofno.Config(**cfg.__dict__)
    out_ref, cache = ofno.forward(p, x, ocfg)
    loss_ref, dout_ref = ofno.mse(out_ref, t)
    g_ref = ofno.backward(p, cache, dout_ref, ocfg)
    out = net.forward(dev(x), train=True)
    assert rel(out.cpu().numpy(), out_ref) < TOL
    dout = torch.empty_like(out)
    fno.fno_mse(out, dev(t), dout, net._loss, net._mse_work)
    assert abs(float(net._loss.item()) - loss_ref) <= 1e-5 * loss_ref
    net.backward(dout)
    g = net.export(grads=True)
    for name in g_ref:
        assert rel(g[name], g_ref[name]) < 1e-4, name
    # repeatable: a second pass gives the same bits
    first = net.grads.clone()
    net.forward(dev(x), train=True)
    net.backward(dout)
    assert torch.equal(first, net.grads)
    # FP32 inference (fused projection head) agrees like the training forward
    assert rel(net.forward(dev(x), train=False).cpu().numpy(), out_ref) < TOL
    # BF16 activations (inference): error stated, bounded by 1e-2
    out16 = net.forward(dev(x), train=False, bf16=True)
    e16 = rel(out16.cpu().numpy(), out_ref)
    assert e16 < 1e-2, e16


def test_adam_matches_oracle():
    n = 1000
    p0, g = RNG.standard_normal(n), RNG.standard_normal(n)
    m0, v0 = RNG.standard_normal(n) * 0.1, np.abs(RNG.standard_normal(n)) * 0.01
    p, m, v = dev(p0), dev(m0), dev(v0)
    fno.fno_adam(p, dev(g), m, v, 1e-3, 5)
    pr, mr, vr = ofno.adam(p0, g, m0, v0, 5, 1e-3)
    assert rel(p.cpu().numpy(), pr) < 1e-6 and rel(m.cpu().numpy(), mr) < 1e-6 and rel(v.cpu().numpy(), vr) < 1e-6


def test_training_reduces_loss():
    # learn a fixed smooth map (a shifted, scaled copy of the first channel)
    cfg = fno.FNOConfig(cin=3, width=16, hidden=32, layers=3, mz=6, mx=6)
    Nz, Nx, B = 48, 64, 4
    net = fno.FNO2d(cfg, Nz, Nx, seed=1)
    z, x = np.meshgrid(np.linspace(0, 1, Nz), np.linspace(0, 1, Nx), indexing="ij")
    data = []
    for k in range(8):
        f = np.sin(2 * np.pi * (RNG.uniform(0.5, 2) * z + RNG.uniform(0.5, 2) * x + RNG.uniform(0, 1)))
        inp = np.stack([f, z, x])[None].repeat(1, 0)
        data.append((inp, 0.5 * np.roll(f, 3, axis=1)[None, None]))
    X = dev(np.concatenate([d[0] for d in data]))
    T = dev(np.concatenate([d[1] for d in data]))
    l0 = net.loss(X, T)
    for it in range(150):
        sel = slice((it % 2) * B, (it % 2) * B + B)
        net.train_step(X[sel].contiguous(), T[sel].contiguous(), 3e-3)
    l1 = net.loss(X, T)
    assert l1 < 0.2 * l0, (l0, l1)


@pytest.mark.parametrize("co,spectral,Nz,Nx,mx", [
    (32, True, 12, 300, 7), (64, False, 12, 300, 7), (32, False, 12, 300, 7), (32, True, 12, 301, 7),
    # rows a multiple of 8 pixels and an even mode count: activations and T copied with cp.async;
    # Nz = 301 gives several rows per CTA and a last CTA with a single row
    (32, True, 301, 264, 8), (64, True, 301, 520, 16), (64, False, 40, 512, 16), (32, True, 301, 264, 7)])
def test_tensor_core_combine_matches_cuda_cores_and_reference(co, spectral, Nz, Nx, mx):
    """The tcgen05 channel mix (BF16 operands, FP32 accumulation in tensor
    memory) against the CUDA-core kernel and an FP64 reference computed from the
    same BF16 activations, on row lengths that leave a ragged 128-pixel tile
    (some not a multiple of 4 or 8) and ragged groups of rows."""
    B, ci, mz = 2, 32, 4
    x = torch.from_numpy(RNG.standard_normal((B, ci, Nz, Nx)).astype(np.float32)).to(torch.bfloat16).cuda()
    M, b = RNG.standard_normal((co, ci)) / np.sqrt(ci), RNG.standard_normal(co)
    (tf, ti, tb, ta), tz = fno.fno_tables(Nz, Nx, mz, mx)
    Th = RNG.standard_normal((B * co, Nz, mx, 2)) * 50.0
    T = dev(Th) if spectral else None
    kw = dict(bias=dev(b), act=fno.ACT_GELU, out_dtype=torch.bfloat16)
    if spectral:
        kw.update(T=T, table=ti, mx=mx)
    try:
        fno.fno_set_tensor_cores(True)
        out_tc = fno.fno_combine(x, dev(M), co, **kw).float().cpu().numpy()
        assert fno.fno_tensor_core_status() == 0
        fno.fno_set_tensor_cores(False)
        out_cc = fno.fno_combine(x, dev(M), co, **kw).float().cpu().numpy()
    finally:
        fno.fno_set_tensor_cores(True)
    xf = x.float().cpu().numpy().astype(np.float64)
    pre = ofno.pointwise(M, b, xf)
    if spectral:
        Tn = Th.astype(np.float32).astype(np.float64).reshape(B, co, Nz, mx, 2)
        inv = ofno.twiddle_tables(Nz, Nx, mz, mx)[1]  # [Nx][mx]
        pre += Tn[..., 0] @ inv.real.T - Tn[..., 1] @ inv.imag.T
    ref = ofno.gelu(pre)
    # BF16 operands and output: relative errors of a few 1e-3
    assert rel(out_tc, ref) < 1e-2, rel(out_tc, ref)
    assert rel(out_cc, ref) < 1e-2, rel(out_cc, ref)
    assert rel(out_tc, out_cc) < 1e-2


@pytest.mark.parametrize("shape", [(2, 32, 24, 512, 16), (3, 5, 37, 300, 7), (3, 5, 37, 264, 8), (1, 2, 40, 1024, 16),
                                   (1, 3, 20, 1032, 5)])
def test_tensor_core_x_transform_matches_reference(shape):
    """The tcgen05 x transform of BF16 activations (K = Nx in chunks of 64,
    ragged K and rows; rows of a multiple of 8 through the cp.async ring, others
    through the staged kernel) against the CUDA-core kernel and an FP64
    reference."""
    B, C, Nz, Nx, mx = shape
    v = torch.from_numpy(RNG.standard_normal((B, C, Nz, Nx)).astype(np.float32)).to(torch.bfloat16).cuda()
    (tf, ti, tb, ta), tz = fno.fno_tables(Nz, Nx, 4, mx)
    try:
        fno.fno_set_tensor_cores(True)
        out_tc = fno.fno_dft_x(v, mx, tf).cpu().numpy()
        assert fno.fno_tensor_core_status() == 0
        fno.fno_set_tensor_cores(False)
        out_cc = fno.fno_dft_x(v, mx, tf).cpu().numpy()
    finally:
        fno.fno_set_tensor_cores(True)
    vf = v.float().cpu().numpy().astype(np.float64).reshape(-1, Nx)
    fwd = ofno.twiddle_tables(Nz, Nx, 4, mx)[0]  # [Nx][mx]
    ref = (vf @ fwd).view(np.float64)  # interleaved (re, im) per mode
    assert rel(out_tc.reshape(ref.shape), ref) < 1e-2
    assert rel(out_cc.reshape(ref.shape), ref) < 1e-5


@pytest.mark.parametrize("dtype,Ci,H,Nz,Nx,tc", [
    (torch.bfloat16, 32, 64, 301, 264, True),  # tensor cores, cp.async staging, rows per CTA > 1, ragged tile
    (torch.bfloat16, 32, 32, 12, 300, True),   # tensor cores, element-wise staging
    (torch.bfloat16, 32, 64, 40, 512, False),  # CUDA cores on BF16 input
    (torch.float32, 32, 64, 37, 70, False),
    (torch.float32, 5, 7, 9, 33, False)])
def test_fused_projection_matches_two_layers_and_reference(dtype, Ci, H, Nz, Nx, tc):
    """fno_project (both head layers in one pass) against two fno_combine calls
    and an FP64 reference from the same input values."""
    B = 2
    x = torch.from_numpy(RNG.standard_normal((B, Ci, Nz, Nx)).astype(np.float32)).cuda().to(dtype)
    Q1, q1 = RNG.standard_normal((H, Ci)) / np.sqrt(Ci), RNG.standard_normal(H)
    Q2, q2 = RNG.standard_normal((1, H)) / np.sqrt(H), RNG.standard_normal(1)
    try:
        fno.fno_set_tensor_cores(tc)
        out = fno.fno_project(x, dev(Q1), dev(q1), dev(Q2), dev(q2)).cpu().numpy()
        assert fno.fno_tensor_core_status() == 0
    finally:
        fno.fno_set_tensor_cores(True)
    h = fno.fno_combine(x, dev(Q1), H, bias=dev(q1), act=fno.ACT_GELU)  # float hidden layer, CUDA cores
    two = fno.fno_combine(h, dev(Q2), 1, bias=dev(q2)).cpu().numpy()
    xf = x.float().cpu().numpy().astype(np.float64)
    ref = ofno.pointwise(Q2, q2, ofno.gelu(ofno.pointwise(Q1, q1, xf)))
    assert out.shape == (B, 1, Nz, Nx)
    assert rel(two, ref) < 1e-5
    # tensor cores: Q1 rounded to BF16 on its way in; otherwise float arithmetic throughout
    assert rel(out, ref) < (1e-2 if tc else 1e-5), rel(out, ref)
    if tc:
        # with the same BF16 weights the rest is float: FP32 accumulation, the bias
        # to 16 bits, GELU by Abramowitz-Stegun 7.1.26 (|erf error| <= 1.5e-7)
        Q1b = torch.from_numpy(Q1).to(torch.bfloat16).double().numpy()
        refb = ofno.pointwise(Q2, q2, ofno.gelu(ofno.pointwise(Q1b, q1, xf)))
        assert rel(out, refb) < 5e-5, rel(out, refb)
