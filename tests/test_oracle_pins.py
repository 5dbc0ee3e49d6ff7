"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to numpy/scipy library routines, a closed
form, brute force on a tiny input, an invariant, or a count the paper prints,
so that a dropped term, a wrong sign or index, or a transposed operand in
oracle/fic_oracle.c fails at least one of them.  No GPU needed.
"""
import os

import numpy as np
import pytest

import fic_synth

# numpy statement of the eight symmetries (Section V: rotations and mirroring),
# in the oracle's numbering: identity, rot90 cw, rot180, rot270 cw, mirror L-R,
# mirror T-B, transpose, anti-transpose.
NP_SYM = [
    lambda a: a,
    lambda a: np.rot90(a, -1),
    lambda a: np.rot90(a, 2),
    lambda a: np.rot90(a, 1),
    lambda a: np.fliplr(a),
    lambda a: np.flipud(a),
    lambda a: a.T,
    lambda a: np.rot90(a, 2).T,
]


def np_tau(block):
    n = block.shape[0] // 2
    return block.reshape(n, 2, n, 2).mean(axis=(1, 3))


def np_range(img, r, n):
    nx = img.shape[1] // n
    y, x = (r // nx) * n, (r % nx) * n
    return img[y:y + n, x:x + n].astype(np.float64)


def np_domain(img, d, n, t):
    u_count = (img.shape[1] - 2 * n) // t + 1
    y, x = (d // u_count) * t, (d % u_count) * t
    return img[y:y + 2 * n, x:x + 2 * n].astype(np.float64)


def np_code_block(img, d, k, n, t):
    return NP_SYM[k](np_tau(np_domain(img, d, n, t)))


def lstsq_fit(a, b):
    """Slope/intercept of b ~ s*a + o by numpy least squares (flat a -> s = 0)."""
    a, b = a.ravel(), b.ravel()
    if np.all(a == a[0]):
        return 0.0, float(b.mean())
    A = np.stack([a, np.ones_like(a)], 1)
    (s, o), *_ = np.linalg.lstsq(A, b, rcond=None)
    return float(s), float(o)


def grid_fit(a, b, bit_depth, s_bits, o_bits):
    """Quantised fit characterised without the oracle's formulas:
    s code = grid point nearest the lstsq slope (clamped to [-1,1]);
    o code = brute-force minimiser of the residual over every o grid point."""
    P = (1 << bit_depth) - 1
    Ls, Lo = (1 << (s_bits - 1)) - 1, (1 << (o_bits - 1)) - 1
    s, _ = lstsq_fit(a, b)
    c = int(np.round(np.clip(s, -1, 1) * Ls))
    sh = c / Ls
    oh = np.arange(-Lo, Lo + 1) * P / Lo
    res = ((sh * a.ravel()[None, :] + oh[:, None] - b.ravel()[None, :]) ** 2).sum(1)
    e = int(np.argmin(res)) - Lo
    return c, e, float(res.min())


# ---------------------------------------------------------------- symmetries
def _planted(n=4, t=4, k=0, seed=0):
    """32x32 float image: random domain 0, range 36 (at (16,16)) = S_k(tau(domain 0))."""
    rng = np.random.default_rng(seed)
    img = rng.uniform(0, 200, (32, 32))
    dom = rng.uniform(0, 255, (2 * n, 2 * n))
    img[:2 * n, :2 * n] = dom
    img[16:16 + n, 16:16 + n] = NP_SYM[k](np_tau(dom))
    return img


@pytest.mark.parametrize("k", range(8))
def test_symmetry_numbering_matches_numpy(orc, k):
    img = _planted(k=k, seed=k)
    r = (16 // 4) * (32 // 4) + 16 // 4
    for kk in range(8):
        f = orc.fit_candidate(img, r, 0, kk, n=4, t=4, bit_depth=8, s_bits=0, o_bits=0)
        if kk == k:
            assert f["err"] < 1e-18 and abs(f["s_ls"] - 1) < 1e-12 and abs(f["o_raw"]) < 1e-9
        else:
            assert f["err"] > 1.0


def test_symmetries_form_the_dihedral_group():
    a = np.arange(16.0).reshape(4, 4)
    imgs = {NP_SYM[k](a).tobytes() for k in range(8)}
    assert len(imgs) == 8
    r90 = NP_SYM[1]
    assert np.array_equal(r90(r90(r90(r90(a)))), a)
    for k in (4, 5, 6, 7):
        assert np.array_equal(NP_SYM[k](NP_SYM[k](a)), a)


@pytest.mark.parametrize("k", range(8))
def test_contraction_commutes_with_symmetries(k):
    """S_k(tau(c)) == tau(S_k(c)): symmetries can be applied after the 2x2 mean."""
    c = np.random.default_rng(k).integers(0, 4096, (16, 16)).astype(np.float64)
    assert np.array_equal(NP_SYM[k](np_tau(c)), np_tau(NP_SYM[k](c)))


# ---------------------------------------------------------------- least squares
def test_least_squares_matches_lstsq(orc):
    img = fic_synth.random_image(7, 32, 32, 8).astype(np.float64)
    rng = np.random.default_rng(1)
    for _ in range(40):
        r, d, k = int(rng.integers(16)), int(rng.integers(9)), int(rng.integers(8))
        f = orc.fit_candidate(img, r, d, k, n=8, t=8, bit_depth=8, s_bits=0, o_bits=0)
        a, b = np_code_block(img, d, k, 8, 8), np_range(img, r, 8)
        s, o = lstsq_fit(a, b)
        assert f["s_ls"] == pytest.approx(s, rel=1e-10, abs=1e-12)
        assert f["o_hat"] == pytest.approx(o, rel=1e-10, abs=1e-9)
        resid = s * a + o - b
        assert f["err"] == pytest.approx((resid ** 2).sum(), rel=1e-9, abs=1e-9)
        # normal equations: residual orthogonal to 1 and to a
        assert abs(resid.sum()) < 1e-8 and abs((resid * a).sum()) < 1e-5


def test_flat_domain_gives_zero_slope_and_mean_offset(orc):
    img = fic_synth.random_image(3, 32, 32, 8).astype(np.float64)
    img[:16, :16] = 77.0  # domain 0 (n=8, t=8) is flat
    for r in (5, 10, 15):
        f = orc.fit_candidate(img, r, 0, 3, n=8, t=8, bit_depth=8, s_bits=0, o_bits=0)
        assert f["s_ls"] == 0.0
        assert f["o_hat"] == pytest.approx(np_range(img, r, 8).mean(), rel=1e-13)


# ---------------------------------------------------------------- quantisers
@pytest.mark.parametrize("bits", [(8, 5, 7), (12, 5, 7), (12, 4, 6)])
def test_quantised_codes_are_grid_optimal(orc, bits):
    B, sb, ob = bits
    img = fic_synth.random_image(11 + B, 32, 32, B).astype(np.float64)
    img[8:16, 0:8] = 5.0  # a shadow range
    rng = np.random.default_rng(B)
    for _ in range(60):
        r, d, k = int(rng.integers(16)), int(rng.integers(9)), int(rng.integers(8))
        f = orc.fit_candidate(img, r, d, k, n=8, t=8, bit_depth=B, s_bits=sb, o_bits=ob)
        c, e, res = grid_fit(np_code_block(img, d, k, 8, 8), np_range(img, r, 8), B, sb, ob)
        assert (f["c"], f["e"]) == (c, e)
        assert f["err"] == pytest.approx(res, rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("slope,mb,c_end,e_end", [(3.0, 128.0, 15, None), (-3.0, 128.0, -15, None),
                                                  (-2.0, 200.0, -15, 63)])
def test_codes_at_the_grid_ends(orc, slope, mb, c_end, e_end):
    """Planted blocks whose fit lies outside the code grids: a slope of +-3
    clamps s to +-1, and with s = -1 an offset mean(b) + mean(a) ~ 400 > P = 255
    clamps o to P.  The codes are the grid ends and equal the brute-force grid
    fit; the residual is that of the clamped codes."""
    n, t, B, sb, ob = 4, 4, 8, 5, 7
    rng = np.random.default_rng(int(10 * slope + mb))
    img = rng.uniform(0, 255, (32, 32))
    dom = 200.0 + rng.uniform(-10, 10, (2 * n, 2 * n))
    img[:2 * n, :2 * n] = dom
    a = np_tau(dom)
    img[16:16 + n, 16:16 + n] = slope * (a - a.mean()) + mb
    r = (16 // n) * (32 // n) + 16 // n
    f = orc.fit_candidate(img, r, 0, 0, n=n, t=t, bit_depth=B, s_bits=sb, o_bits=ob)
    c, e, res = grid_fit(a, np_range(img, r, n), B, sb, ob)
    assert (f["c"], f["e"]) == (c, e)
    assert f["c"] == c_end and f["s_hat"] == c_end / 15
    if e_end is not None:
        assert f["e"] == e_end and f["o_hat"] == 255.0 and f["o_raw"] > 255.0
    assert f["err"] == pytest.approx(res, rel=1e-12, abs=1e-9)


def test_nearest_s_level_is_optimal_for_free_offset():
    """With o free, the residual is a convex quadratic in s, so the nearest grid
    level to the least-squares slope is the best level (brute force over levels)."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        a = rng.uniform(0, 255, 64)
        b = rng.uniform(-0.8, 0.8) * a + rng.normal(0, 20, 64)
        s, _ = lstsq_fit(a, b)
        levels = np.arange(-15, 16) / 15.0
        cost = [((lv * a - b) - (lv * a - b).mean()) @ ((lv * a - b) - (lv * a - b).mean()) for lv in levels]
        best = levels[int(np.argmin(cost))]
        assert abs(best - np.clip(s, -1, 1)) <= 1 / 30 + 1e-12


# ---------------------------------------------------------------- search
@pytest.mark.parametrize("seed,B", [(1, 8), (2, 12), (3, 8)])
def test_search_equals_brute_force(orc, seed, B):
    """Every range of a 16x16 image (n=4, t=4): 9 domains x 8 symmetries each,
    characterised independently; the oracle must return the lexicographically
    first (d, k) among the minima of the residual."""
    img = fic_synth.random_image(seed, 16, 16, B).astype(np.float64)
    if seed == 3:
        img[0:4, 0:4] = 9.0      # shadow range
        img[8:16, 8:16] = 100.0  # flat domains -> massive exact ties
    got = orc.encode(img, n=4, t=4, bit_depth=B, s_bits=5, o_bits=7)
    for r in range(16):
        b = np_range(img, r, 4)
        best = None
        for d in range(9):
            for k in range(8):
                _, _, res = grid_fit(np_code_block(img, d, k, 4, 4), b, B, 5, 7)
                if best is None or res < best[0] - 1e-9 * max(1.0, res):
                    best = (res, d, k)
        assert got[r]["err"] == pytest.approx(best[0], rel=1e-12, abs=1e-9)
        assert (got[r]["d"], got[r]["k"]) == best[1:]


def test_linear_ramp_is_reproduced_exactly(orc):
    """A ramp I = 2x + 3y: every range is its own domain 0 contracted with s = 1/2
    (quantisation off), residual exactly 0 (closed form)."""
    yy, xx = np.mgrid[0:64, 0:64]
    img = (2 * xx + 3 * yy).astype(np.float64)
    got = orc.encode(img, n=8, t=8, bit_depth=12, s_bits=0, o_bits=0)
    assert np.all(got["err"] == 0.0)
    assert np.all(got["d"] == 0) and np.all(got["k"] == 0) and np.all(got["s_hat"] == 0.5)


def test_constant_image_shadow_ranges(orc):
    """Every range of a constant image is a shadow block: the first candidate
    (0, 0) with s = 0 and the nearest offset level."""
    c = 1234.0
    img = np.full((64, 64), c)
    got = orc.encode(img, n=8, t=4, bit_depth=12, s_bits=5, o_bits=7)
    e = int(np.round(c * 63 / 4095))
    assert np.all(got["d"] == 0) and np.all(got["k"] == 0) and np.all(got["c"] == 0)
    assert np.all(got["e"] == e)
    assert np.allclose(got["err"], 64 * (e * 4095 / 63 - c) ** 2, rtol=1e-12)


def test_exact_attractor_is_encoded_with_zero_error(orc):
    """Random contractive maps with on-grid (s, o): decode to the fixed point x*,
    then encode x*; the generating maps have zero collage error, so every
    range's minimum must be ~0."""
    rng = np.random.default_rng(42)
    h = w = 64
    n, t = 8, 8
    R, D = orc.counts(h, w, n, t)
    dom = rng.integers(0, D, R).astype(np.int32)
    sym = rng.integers(0, 8, R).astype(np.int32)
    c = rng.integers(-10, 11, R)
    c[c == 0] = 7
    e = rng.integers(0, 20, R)
    s_hat, o_hat = c / 15.0, e * 255 / 63.0
    x, _ = orc.decode(dom, sym, s_hat, o_hat, h, w, n=n, t=t, bit_depth=8, iters=300,
                      init=128.0, clamp=False, trace=True)
    got = orc.encode(x, n=n, t=t, bit_depth=8, s_bits=5, o_bits=7)
    assert got["err"].max() < 1e-12 * 64 * 255 ** 2
    # the generating map of every range reproduces it: decode and encode agree
    # on domain placement and on the symmetry numbering
    for r in range(R):
        f = orc.fit_candidate(x, r, dom[r], sym[r], n=n, t=t, bit_depth=8, s_bits=5, o_bits=7)
        assert (f["c"], f["e"]) == (c[r], e[r]) and f["err"] < 1e-12 * 64 * 255 ** 2


# ---------------------------------------------------------------- decoding
def test_decode_converges_to_the_ramp(orc):
    """Maps of the ramp (s = 1/2, domain 0, identity) have the ramp as attractor:
    the decode error halves (at least) every iteration."""
    yy, xx = np.mgrid[0:64, 0:64]
    img = (2 * xx + 3 * yy).astype(np.float64)
    got = orc.encode(img, n=8, t=8, bit_depth=12, s_bits=0, o_bits=0)
    _, tr = orc.decode(got["d"], got["k"], got["s_hat"], got["o_hat"], 64, 64, n=8, t=8,
                       bit_depth=12, iters=40, init=2048.0, clamp=False, trace=True)
    errs = [np.abs(it - img).max() for it in tr]
    for a, b in zip(errs[:-1], errs[1:]):
        assert b <= 0.5 * a + 1e-9
    assert errs[-1] < 1e-6


def test_decode_iterates_contract(orc):
    """|x_{t+1} - x_t|_inf <= max|s| * |x_t - x_{t-1}|_inf (contraction, Section III-A)."""
    img = fic_synth.mr_slice(size=64)
    got = orc.encode(img, n=8, t=8, bit_depth=8)
    _, tr = orc.decode(got["d"], got["k"], got["s_hat"], got["o_hat"], 64, 64, n=8, t=8,
                       bit_depth=8, iters=12, clamp=False, trace=True)
    smax = np.abs(got["s_hat"]).max()
    steps = [np.abs(b - a).max() for a, b in zip(tr[:-1], tr[1:])]
    for a, b in zip(steps[:-1], steps[1:]):
        assert b <= smax * a * (1 + 1e-12) + 1e-9


@pytest.mark.parametrize("s,o,init", [(0.5, 4000.0, 100.0), (0.75, -300.0, 2048.0), (-0.5, 1000.0, 0.0)])
def test_decode_of_uniform_maps_closed_form(orc, s, o, init):
    """With one (s, o) for every range, a flat image stays flat whatever the
    domains and symmetries (the 2x2 mean of a constant is the constant), so
    x_t = s^t x_0 + o (1 - s^t) / (1 - s).  The first two cases leave [0, P]
    (towards 8000 and -1200 for P = 4095): the clamped decode is the clip of
    that value, the unclamped decode the value itself."""
    h = w = 32
    n, t, B, T = 8, 4, 12, 9
    R = (h // n) * (w // n)
    U = (w - 2 * n) // t + 1
    rng = np.random.default_rng(5)
    dom = rng.integers(0, U * U, R).astype(np.int32)
    sym = rng.integers(0, 8, R).astype(np.int32)
    sv, ov = np.full(R, s), np.full(R, o)
    want = s ** T * init + o * (1 - s ** T) / (1 - s)
    raw = orc.decode(dom, sym, sv, ov, h, w, n=n, t=t, bit_depth=B, iters=T, init=init, clamp=False)
    assert np.allclose(raw, want, rtol=0, atol=1e-9 * (abs(want) + abs(o)))
    got = orc.decode(dom, sym, sv, ov, h, w, n=n, t=t, bit_depth=B, iters=T, init=init)
    assert np.array_equal(got, np.clip(raw, 0, (1 << B) - 1))
    assert np.all((got >= 0) & (got <= (1 << B) - 1))


def test_psnr_closed_form(orc):
    ref = np.zeros((16, 16))
    assert orc.psnr(ref, ref + 1.0, 8) == pytest.approx(20 * np.log10(255.0), rel=1e-14)
    assert orc.psnr(ref, ref + 2.0, 12) == pytest.approx(20 * np.log10(4095.0 / 2.0), rel=1e-14)


# ---------------------------------------------------------------- paper counts
def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(v) for v in line.split()])
    return rows


def test_paper_counts(orc):
    for size, n, t, ranges, domains, tests in _golden("paper_counts.txt"):
        R, D = orc.counts(size, size, n, t)
        assert (R, D) == (ranges, domains)
        assert R * D == tests


def test_scaled_decode_averages_down_to_the_unscaled_decode(orc):
    """Resolution-independent decoding: the same maps at twice the size (ranges
    2n at 2x, domains 4n at stride 2t) average 2x2 down to the decode at the
    original size, iterate by iterate, because the 2x2 contraction commutes
    with the symmetries; likewise the original averages down to half size."""
    img = fic_synth.ct_slice(34, 64)
    fit = orc.encode(img, n=8, t=4, bit_depth=12)
    args = (fit["d"], fit["k"], fit["s_hat"], fit["o_hat"])

    def dec(z_num, z_den):
        n, t, size = 8 * z_num // z_den, 4 * z_num // z_den, 64 * z_num // z_den
        return orc.decode(*args, size, size, n=n, t=t, bit_depth=12, iters=6, clamp=False)

    def down(x):
        return 0.25 * (x[0::2, 0::2] + x[1::2, 0::2] + x[0::2, 1::2] + x[1::2, 1::2])

    x1, x2, xh = dec(1, 1), dec(2, 1), dec(1, 2)
    assert x2.shape == (128, 128) and xh.shape == (32, 32)
    assert np.allclose(down(x2), x1, rtol=0, atol=1e-9 * 4095)
    assert np.allclose(down(x1), xh, rtol=0, atol=1e-9 * 4095)


def test_exact_ties_round_half_away_from_zero(orc):
    # eq 11-12 quantise s and o to the nearest code; on an exact half the
    # reading is "half away from zero" (C round()).  The two crafted ranges
    # of rounding_tie_image land exactly on s * Ls = 7.5 and o * Lo / P = 1.5:
    # the codes must be 8 and 2, and the neighbouring codes must give the
    # same least-squares distance (the tie is real, not a near miss).
    img = fic_synth.rounding_tie_image().astype(np.float64)
    ref = orc.encode(img, n=8, t=16, bit_depth=12)
    assert (ref["d"][15], ref["k"][15], ref["s_ls"][15], ref["c"][15]) == (0, 0, 0.5, 8)
    assert (ref["d"][8], ref["k"][8], ref["c"][8], ref["o_raw"][8], ref["e"][8]) == (0, 0, 0, 97.5, 2)
    assert abs(0.5 * 15 - 8) == abs(0.5 * 15 - 7)
    assert abs(97.5 * 63 / 4095 - 2) == abs(97.5 * 63 / 4095 - 1)
