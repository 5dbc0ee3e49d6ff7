"""Pins of the oracle's refinement gradient (FP64 adjoint of the unrolled decode).

The gradient is checked against central finite differences of the oracle's
own loss (the definition of a derivative; eps = 1e-3 as the refinement
workload states), and against the closed form of a one-iteration decode from
a flat start, where x_1 = s_r * c + o_r on range r.
"""
import numpy as np
import pytest

import fic_synth


def setup_case(orc, seed, size=32, n=4, t=4, B=12):
    img = fic_synth.ct_slice(seed, size)
    fit = orc.encode(img, n=n, t=t, bit_depth=B)
    P = (1 << B) - 1
    return img.astype(np.float64), fit["d"], fit["k"], fit["s_hat"].copy(), fit["o_hat"].copy(), P


@pytest.mark.parametrize("iters", [1, 3, 8])
def test_gradient_matches_central_differences(orc, iters):
    ref, dom, sym, s, o, P = setup_case(orc, 51)
    rng = np.random.default_rng(iters)
    s = s + rng.normal(0, 0.05, s.shape)  # off the quantisation grid
    o = o + rng.normal(0, 20.0, o.shape)
    kw = dict(n=4, t=4, bit_depth=12, iters=iters)
    loss, gs, go = orc.refine_grad(dom, sym, s, o, ref, **kw)
    eps = 1e-3

    def central(vec_s, vec_o, r, which, e):
        a, b = (vec_s.copy(), vec_o.copy()), (vec_s.copy(), vec_o.copy())
        a[which][r] += e
        b[which][r] -= e
        return (orc.refine_grad(dom, sym, *a, ref, **kw)[0] - orc.refine_grad(dom, sym, *b, ref, **kw)[0]) / (2 * e)

    for r in rng.choice(len(s), 12, replace=False):
        for which, g in ((0, gs), (1, go)):
            scale = max(abs(g).max(), 1e-300)
            f1 = central(s, o, r, which, eps)
            f2 = central(s, o, r, which, eps / 2)
            # eps = 1e-3 central difference (truncation error O(eps^2))
            assert abs(f1 - g[r]) <= 1e-4 * scale, (r, which, f1, g[r])
            # Richardson extrapolation of eps and eps/2: error O(eps^4)
            assert abs((4 * f2 - f1) / 3 - g[r]) <= 1e-7 * scale, (r, which, (4 * f2 - f1) / 3, g[r])


def test_one_iteration_closed_form(orc):
    ref, dom, sym, s, o, P = setup_case(orc, 52)
    c = 1000.0
    loss, gs, go = orc.refine_grad(dom, sym, s, o, ref, n=4, t=4, bit_depth=12, iters=1, init=c)
    h, w = ref.shape
    N = h * w
    blocks = ref.reshape(h // 4, 4, w // 4, 4).transpose(0, 2, 1, 3).reshape(-1, 16)
    resid = s[:, None] * c + o[:, None] - blocks
    assert np.isclose(loss, np.sum(resid ** 2) / N, rtol=1e-13)
    assert np.allclose(go, 2.0 * resid.sum(1) / N, rtol=1e-12, atol=1e-15)
    assert np.allclose(gs, 2.0 * c * resid.sum(1) / N, rtol=1e-12, atol=1e-12)


def test_forward_is_the_unclamped_decode(orc):
    ref, dom, sym, s, o, P = setup_case(orc, 53)
    loss, _, _ = orc.refine_grad(dom, sym, s, o, ref, n=4, t=4, bit_depth=12, iters=5)
    x = orc.decode(dom, sym, s, o, 32, 32, n=4, t=4, bit_depth=12, iters=5, clamp=False)
    assert np.isclose(loss, np.mean((x - ref) ** 2), rtol=1e-13)
