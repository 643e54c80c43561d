"""The schedule network's CUDA kernels (through the C ABI) against the FP64 reference."""
import numpy as np
import pytest

import synth
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eik():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00009_gb300 import build
    build.build()
    import paper_1811_00009_gb300 as E
    return E


def _data(seed, B):
    w = (synth.normal(seed, 1, mlp.n_params()) * 0.3).astype(np.float32)
    X = synth.normal(seed, 2, B * mlp.D_IN).reshape(B, mlp.D_IN).astype(np.float32)
    act = (synth.uniform(seed, 3, B) * mlp.A).astype(np.int32)
    tgt = synth.normal(seed, 4, B).astype(np.float32)
    return w, X, act, tgt


def _cuda(*arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def test_forward_matches_fp64(eik):
    import torch
    w, X, act, tgt = _data(11, 1000)
    wd, Xd = _cuda(w, X)
    Y = torch.empty((1000, mlp.A), dtype=torch.float32, device="cuda")
    eik.eik_mlp_forward(wd, Xd, Y)
    ref, _, _ = mlp.forward(w.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(Y.cpu().numpy(), ref, rtol=1e-4, atol=1e-5)


def test_gradient_matches_fp64_and_is_deterministic(eik):
    import torch
    B = 2048
    w, X, act, tgt = _data(12, B)
    wd, Xd, ad, td = _cuda(w, X, act, tgt)
    g1 = torch.empty(mlp.n_params(), dtype=torch.float32, device="cuda")
    g2 = torch.empty_like(g1)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    work = torch.empty(eik.eik_mlp_work_floats(B), dtype=torch.float32, device="cuda")
    eik.eik_mlp_grad(wd, Xd, ad, td, g1, loss, work)
    eik.eik_mlp_grad(wd, Xd, ad, td, g2, loss, work)
    torch.cuda.synchronize()
    l_ref, g_ref = mlp.grad(w.astype(np.float64), X.astype(np.float64), act, tgt.astype(np.float64))
    g = g1.cpu().numpy()
    assert np.array_equal(g, g2.cpu().numpy())
    assert abs(loss.item() - l_ref) <= 1e-4 * abs(l_ref)
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-3 * scale


def test_adam_matches_fp64(eik):
    import torch
    n = mlp.n_params()
    w, X, act, tgt = _data(13, 8)
    g = (synth.normal(13, 9, n) * 0.01).astype(np.float32)
    wd, gd = _cuda(w, g)
    m = torch.zeros(n, dtype=torch.float32, device="cuda")
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    wr, mr, vr = w.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in (1, 2, 3):
        eik.eik_mlp_adam(wd, gd, m, v, t, lr=1e-2)
        wr, mr, vr = mlp.adam(wr, g.astype(np.float64), mr, vr, t, lr=1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(wd.cpu().numpy(), wr, rtol=0, atol=2e-6)


def test_training_on_the_gpu_reduces_loss(eik):
    import torch
    B = 4096
    w, X, act, tgt = _data(14, B)
    tgt = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * (act % 3 == 0)).astype(np.float32)
    wd, Xd, ad, td = _cuda(w, X, act, tgt)
    n = mlp.n_params()
    g = torch.empty(n, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(g); v = torch.zeros_like(g)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    work = torch.empty(eik.eik_mlp_work_floats(B), dtype=torch.float32, device="cuda")
    eik.eik_mlp_grad(wd, Xd, ad, td, g, loss, work)
    l0 = loss.item()
    for t in range(1, 301):
        eik.eik_mlp_grad(wd, Xd, ad, td, g, loss, work)
        eik.eik_mlp_adam(wd, g, m, v, t, lr=3e-3)
    eik.eik_mlp_grad(wd, Xd, ad, td, g, loss, work)
    assert loss.item() < 0.3 * l0
