"""The contraction stage alone (fic_cross_terms): the tensor-core and the FP32
CUDA-core paths against the exact integer cross terms.

Xt[r, c] = (m * X - Sq * Sb) / m with X = sum_i q_i b_i (eq 9's cross term),
computed here in int64 with numpy's own rotations/flips for the symmetries.
FP32 accumulation of centred integer products is exact while partial sums
stay below 2^24; beyond that the error is bounded by a small multiple of
2^-24 times the magnitude of the centred products: K = m terms, so for 16x16
ranges (K = 256, hi and lo parts each) the bound is 3 * 256 * 2^-24 < 2^-14
of the scale.
"""
import numpy as np
import pytest

import fic_synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NP_SYM = [lambda a: a, lambda a: np.rot90(a, -1), lambda a: np.rot90(a, 2), lambda a: np.rot90(a, 1),
          lambda a: np.fliplr(a), lambda a: np.flipud(a), lambda a: a.T, lambda a: np.rot90(a, 2).T]


def exact_xt(img, n, t):
    img = img.astype(np.int64)
    h, w = img.shape
    U, V = (w - 2 * n) // t + 1, (h - 2 * n) // t + 1
    q = []
    for d in range(U * V):
        y, x = (d // U) * t, (d % U) * t
        blk = img[y:y + 2 * n, x:x + 2 * n]
        qq = blk[0::2, 0::2] + blk[1::2, 0::2] + blk[0::2, 1::2] + blk[1::2, 1::2]
        q.extend(NP_SYM[k](qq).ravel() for k in range(8))
    q = np.array(q)
    nx = w // n
    b = np.array([img[(r // nx) * n:(r // nx + 1) * n, (r % nx) * n:(r % nx + 1) * n].ravel()
                  for r in range((h // n) * nx)])
    m = n * n
    X = b @ q.T
    xt = (m * X - b.sum(1)[:, None] * q.sum(1)[None, :]) / m
    qc = q - q.mean(1, keepdims=True)
    bc = b - b.mean(1, keepdims=True)
    scale = np.sqrt(((bc ** 2).sum(1) + m)[:, None] * ((qc ** 2).sum(1) + m)[None, :])
    return xt, scale


@pytest.fixture(scope="module")
def fic():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1404_0774_gb300 import fic

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fic


def gpu_xt(fic, img, p):
    t = torch.from_numpy(img.astype(np.int16) if img.dtype == np.uint16 else img).cuda()
    out = fic.cross_terms(t, p)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


CASES = [
    ("mr8", lambda: fic_synth.mr_slice(21, 64), 8, 4, 8),
    ("rand8", lambda: fic_synth.random_image(22, 64, 64, 8), 8, 4, 8),
    ("ct12", lambda: fic_synth.ct_slice(23, 64), 8, 4, 12),
    ("rand12", lambda: fic_synth.random_image(24, 48, 80, 12).astype(np.uint16), 8, 8, 12),
    ("ramp12", lambda: (np.add.outer(np.arange(64) * 40, np.arange(64) * 23) % 4096).astype(np.uint16), 8, 4, 12),
    ("ct12_n4", lambda: fic_synth.ct_slice(25, 64), 4, 2, 12),
    ("mr8_n4", lambda: fic_synth.mr_slice(26, 48), 4, 4, 8),
    ("extremes12", lambda: fic_synth.random_image(27, 64, 64, 1).astype(np.uint16) * 4095, 8, 4, 12),
    ("all4095", lambda: np.full((48, 64), 4095, np.uint16), 8, 4, 12),
    ("ct12_n16", lambda: fic_synth.ct_slice(28, 64), 16, 8, 12),
    ("rand12_n16", lambda: fic_synth.random_image(29, 64, 64, 12).astype(np.uint16), 16, 16, 12),
    ("mr8_n16", lambda: fic_synth.mr_slice(30, 64), 16, 8, 8),
    ("extremes12_n16", lambda: fic_synth.random_image(31, 64, 64, 1).astype(np.uint16) * 4095, 16, 16, 12),
]


@pytest.mark.parametrize("search", ["tc", "simt"])
@pytest.mark.parametrize("name,make,n,t,B", CASES, ids=[c[0] for c in CASES])
def test_cross_terms(fic, name, make, n, t, B, search):
    img = make()
    code = fic.FIC_SEARCH_TC if search == "tc" else fic.FIC_SEARCH_SIMT
    p = fic.params(range_size=n, domain_stride=t, bit_depth=B, search=code)
    got = gpu_xt(fic, img, p)
    ref, scale = exact_xt(img, n, t)
    err = np.abs(got - ref)
    assert np.isfinite(got).all()
    assert (err / scale).max() < (2.0 ** -14 if n == 16 else 2.0 ** -16), (err / scale).max()
    if B == 8 and search == "tc" and n < 16:
        # 8-bit: every product and partial sum of the centred integers is below
        # 2^24, so only the final fractional centring term can round
        assert (err <= np.abs(ref) * 2.0 ** -23 + 2.0 ** -6).all(), err.max()
