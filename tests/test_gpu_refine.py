"""Differentiable refinement (fic_refine_*, through the C ABI and the
torch.autograd.Function): the FP32 loss and adjoint gradient against the FP64
oracle's (refine_grad), central finite differences of the GPU loss, bitwise
determinism, and the native Adam loop against the same loop driven through
autograd and torch.optim.Adam."""
import numpy as np
import pytest

import fic_synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fic():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1404_0774_gb300 import fic

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fic


def encoded(fic, size, seed, n=8, t=4):
    img = fic_synth.ct_slice(seed, size)
    p = fic.params(range_size=n, domain_stride=t, bit_depth=12)
    dimg = torch.from_numpy(img.astype(np.int16)).cuda()
    maps = fic.encode(dimg, p)
    s, o = fic.map_coefficients(maps)
    return img, dimg, p, maps, s, o


def gpu_loss_grad(fic, dimg, p, maps, s, o, iters):
    h, w = dimg.shape
    s = s.clone().requires_grad_(True)
    o = o.clone().requires_grad_(True)
    x = fic.decode_differentiable(s, o, maps, w, h, p, iters)
    loss = torch.mean((x - dimg.float()) ** 2)
    loss.backward()
    return float(loss.detach()), s.grad.double().cpu().numpy(), o.grad.double().cpu().numpy()


@pytest.mark.parametrize("size,iters", [(64, 8), (128, 3), (512, 8)])
def test_gradient_matches_fp64_oracle(fic, orc, size, iters):
    img, dimg, p, maps, s, o = encoded(fic, size, 80 + size)
    rng = torch.Generator(device="cuda").manual_seed(size)
    s = s + 0.02 * torch.randn(s.shape, device="cuda", generator=rng)  # off the quantisation grid
    o = o + 10.0 * torch.randn(o.shape, device="cuda", generator=rng)
    loss, gs, go = gpu_loss_grad(fic, dimg, p, maps, s, o, iters)
    m = fic.maps_to_numpy(maps)
    rl, rs, ro = orc.refine_grad(m["domain_idx"], m["iso"], s.double().cpu().numpy(), o.double().cpu().numpy(),
                                 img.astype(np.float64), n=8, t=4, bit_depth=12, iters=iters)
    assert abs(loss - rl) <= 1e-5 * rl
    assert np.max(np.abs(gs - rs)) <= 1e-4 * np.max(np.abs(rs))
    assert np.max(np.abs(go - ro)) <= 1e-4 * np.max(np.abs(ro))


def test_gradient_matches_central_differences(fic):
    img, dimg, p, maps, s, o = encoded(fic, 64, 90)
    h, w = dimg.shape
    loss, gs, go = gpu_loss_grad(fic, dimg, p, maps, s, o, 8)

    def L(ss, oo):
        with torch.no_grad():
            x = fic.decode_differentiable(ss, oo, maps, w, h, p, 8)
            return float(torch.mean((x.double() - dimg.double()) ** 2))

    # eps = 1e-3 in the optimised parameters (s, o/P): o moves by 1e-3 * P
    P = float((1 << 12) - 1)
    for g, which, eps in ((gs, 0, 1e-3), (go, 1, 1e-3 * P)):
        for r in np.argsort(-np.abs(g))[:6]:
            a, b = [s.clone(), o.clone()], [s.clone(), o.clone()]
            a[which][r] += eps
            b[which][r] -= eps
            fd = (L(*a) - L(*b)) / (2 * eps)
            assert abs(fd - g[r]) <= 2e-2 * abs(g[r]) + 1e-3, (which, r, fd, g[r])


def test_adjoint_is_deterministic(fic):
    img, dimg, p, maps, s, o = encoded(fic, 128, 91)
    a = gpu_loss_grad(fic, dimg, p, maps, s, o, 8)
    b = gpu_loss_grad(fic, dimg, p, maps, s, o, 8)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_native_adam_loop_matches_autograd_loop(fic):
    img, dimg, p, maps, s0, o0 = encoded(fic, 128, 92)
    h, w = dimg.shape
    P = float((1 << 12) - 1)
    steps, lr = 10, 2e-3
    s1, o1 = s0.clone(), o0.clone()
    loss = fic.refine(dimg, maps, s1, o1, p, steps=steps, iters=8, lr=lr)
    torch.cuda.synchronize()
    # the same optimisation through autograd: parameters (s, o/P), torch Adam
    s2 = s0.clone().requires_grad_(True)
    on = (o0 / P).clone().requires_grad_(True)
    opt = torch.optim.Adam([s2, on], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    ref_loss = []
    for _ in range(steps):
        opt.zero_grad()
        x = fic.decode_differentiable(s2, on * P, maps, w, h, p, 8)
        l = torch.mean((x - dimg.float()) ** 2)
        ref_loss.append(float(l))
        l.backward()
        opt.step()
    L = loss.cpu().numpy()
    assert np.allclose(L[:steps], ref_loss, rtol=1e-4)
    assert L[-1] < L[0]
    assert torch.allclose(s1, s2.detach(), rtol=1e-3, atol=1e-4)
    assert torch.allclose(o1, (on * P).detach(), rtol=1e-3, atol=1e-2)
