"""Parity of the CUDA encoder/decoder (through the C ABI) with the FP64 oracle.

For every checked range:
  * the map the GPU returns, re-scored by the oracle for the same
    (domain, symmetry), has identical s/o codes (both sides decide them in
    FP64 with the operation order of eq 9-12) and the same residual to
    1e-12 relative (the GPU reports the exact residual rounded once, the
    oracle sums squares in FP64);
  * its residual is within 1e-5 relative (plus 1e-9*m*P^2 absolute, for exact
    zeros) of the oracle's per-range minimum over all candidates;
  * index agreement with the oracle's choice is reported; it is not required,
    because equal residuals admit several correct maps.
Decoding: GPU FP32 decode of the same maps as the FP64 oracle decode, pixel
by pixel, and the decoded PSNR within 0.01 dB.
"""
import numpy as np
import pytest

import fic_synth
from parity import check_against_oracle, encode_pinned

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


def gpu_encode(fic, img, p):
    dev = torch.device("cuda:0")
    t = torch.from_numpy(img.astype(np.int16) if img.dtype == np.uint16 else img).to(dev)
    maps = fic.encode(t, p)
    torch.cuda.synchronize()
    return fic.maps_to_numpy(maps)


CASES = [
    # (name, image factory, n, t, B)
    ("mr64_t4", lambda: fic_synth.mr_slice(5, 64), 8, 4, 8),
    ("ct64_t4", lambda: fic_synth.ct_slice(6, 64), 8, 4, 12),
    ("rand12_96x64", lambda: fic_synth.random_image(7, 64, 96, 12), 8, 8, 12),
    ("rand8_n4", lambda: fic_synth.random_image(8, 32, 32, 8), 4, 2, 8),
    ("ct12_n4", lambda: fic_synth.ct_slice(13, 96), 4, 2, 12),
    ("mr8_n4_t4", lambda: fic_synth.mr_slice(14, 80), 4, 4, 8),
    ("ct_n16", lambda: fic_synth.ct_slice(9, 64), 16, 8, 12),
    ("min_size", lambda: fic_synth.random_image(10, 16, 16, 8), 8, 8, 8),
    ("constant", lambda: np.full((48, 48), 1234, np.uint16), 8, 4, 12),
    ("flat_regions", lambda: np.where(fic_synth.random_image(11, 64, 64, 8) > 128, 200, 10).astype(np.uint8), 8, 4, 8),
    ("b10_rand", lambda: fic_synth.random_image(12, 48, 48, 10).astype(np.uint16), 8, 4, 10),
    # extreme magnitudes: every pixel 0 or 4095 (the largest centred products)
    ("extremes12", lambda: fic_synth.random_image(15, 64, 64, 1).astype(np.uint16) * 4095, 8, 4, 12),
    ("extremes12_n4", lambda: fic_synth.random_image(16, 48, 48, 1).astype(np.uint16) * 4095, 4, 2, 12),
]


SEARCH = ["simt", "tc"]


def search_code(fic, search):
    return {"simt": fic.FIC_SEARCH_SIMT, "tc": fic.FIC_SEARCH_TC}[search]


@pytest.mark.parametrize("name,make,n,t,B", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("search", SEARCH)
def test_encode_parity_small(fic, orc, name, make, n, t, B, search):
    img = make()
    p = fic.params(range_size=n, domain_stride=t, bit_depth=B, search=search_code(fic, search))
    got = gpu_encode(fic, img, p)
    check_against_oracle(orc, img, got, n, t, B)


@pytest.mark.parametrize("n_split", [1, 3, 0])
@pytest.mark.parametrize("search", SEARCH)
def test_encode_parity_splits(fic, orc, n_split, search):
    img = fic_synth.ct_slice(13, 96)
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12, search=search_code(fic, search), n_split=n_split)
    check_against_oracle(orc, img, gpu_encode(fic, img, p), 8, 4, 12)


@pytest.mark.parametrize("search", SEARCH)
def test_mr_slice_256_full(fic, orc, search):
    """256x256 8-bit MR-like slice, 8x8 ranges, domains at stride 8: every range."""
    img = fic_synth.mr_slice()
    p = fic.params(range_size=8, domain_stride=8, bit_depth=8, search=search_code(fic, search))
    same = check_against_oracle(orc, img, gpu_encode(fic, img, p), 8, 8, 8)
    assert same > 0.99


@pytest.fixture(scope="module")
def ct512_oracle(orc):
    """The oracle's exhaustive search of every range of the 512x512 CT-like
    slice (4096 ranges x 125000 candidates; seconds on the host's threads)."""
    img = fic_synth.ct_slice()
    return img, orc.encode(img, n=8, t=4, bit_depth=12)


@pytest.mark.parametrize("search", SEARCH)
def test_ct_slice_512_full(fic, orc, ct512_oracle, search):
    """512x512 12-bit CT-like slice, 8x8 ranges, domains at stride 4 (5.12e8
    comparisons), in the bench's launch configuration: every map re-scored by
    the oracle and every range's residual checked against the oracle's
    per-range minimum."""
    img, ref = ct512_oracle
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12, search=search_code(fic, search))
    got = gpu_encode(fic, img, p)
    same = check_against_oracle(orc, img, got, 8, 4, 12, ref=ref)
    print(f"index agreement with the oracle: {same:.4f}")


@pytest.fixture(scope="module")
def ct512_n4_oracle(orc):
    """The oracle's exhaustive search of every 4x4 range of the 512x512 slice
    (16384 ranges x 16129 domains x 8 = 2.1e9 comparisons)."""
    img = fic_synth.ct_slice()
    return img, orc.encode(img, n=4, t=4, bit_depth=12)


@pytest.mark.parametrize("search", SEARCH)
def test_ct_slice_512_n4_full(fic, orc, ct512_n4_oracle, search):
    """4x4 ranges on the 512x512 12-bit CT-like slice, 8x8 domains at stride 4
    (the geometry of the quadtree's last level): many near-ties, so lists
    fail certification and the exact re-scans decide; every map re-scored by
    the oracle, every range's residual checked against its minimum."""
    img, ref = ct512_n4_oracle
    p = fic.params(range_size=4, domain_stride=4, bit_depth=12, search=search_code(fic, search))
    got = gpu_encode(fic, img, p)
    check_against_oracle(orc, img, got, 4, 4, 12, ref=ref)
    print(f"maps resolved by exact re-scans: {int((got['info'] & fic.FIC_MAP_FALLBACK != 0).sum())}")


@pytest.mark.parametrize("t", [16, 8])
@pytest.mark.parametrize("search", SEARCH)
def test_ct_slice_512_n16_full(fic, orc, search, t):
    """16x16 ranges on the 512x512 12-bit CT-like slice (the quadtree's first
    level at stride 16, and stride 8): K = 256 per part on the tensor cores;
    every map re-scored, every range's minimum checked."""
    img = fic_synth.ct_slice()
    p = fic.params(range_size=16, domain_stride=t, bit_depth=12, search=search_code(fic, search))
    check_against_oracle(orc, img, gpu_encode(fic, img, p), 16, t, 12)


@pytest.mark.parametrize("search", SEARCH)
def test_ct_slice_1024_sampled(fic, orc, search):
    """The largest size of the paper's experiments (1024x1024), 12-bit CT-like,
    8x8 ranges, domains at stride 4 (16384 ranges x 64009 domains x 8 =
    8.4e9 comparisons): every map re-scored, the minimum checked on sampled
    ranges."""
    img = fic_synth.ct_slice(fic_synth.CT_SEED + 3, 1024)
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12, search=search_code(fic, search))
    got = gpu_encode(fic, img, p)
    rng = np.random.default_rng(1)
    sample = np.sort(rng.choice(16384, 40, replace=False))
    check_against_oracle(orc, img, got, 8, 4, 12, ranges=sample)


@pytest.mark.parametrize("search", SEARCH)
def test_ct_slice_1024_stride2_sampled(fic, orc, search):
    """1024x1024 12-bit CT-like, 8x8 ranges, domains at stride 2 (16384 ranges
    x 255025 domains): more statistics blocks (8482) than one block of the
    fused compaction + rows + seed launch can prefix-sum, so this size takes
    the separate compaction + seed and rows launches.  Every map re-scored,
    the minimum checked on sampled ranges."""
    img = fic_synth.ct_slice(fic_synth.CT_SEED + 4, 1024)
    p = fic.params(range_size=8, domain_stride=2, bit_depth=12, search=search_code(fic, search))
    got = gpu_encode(fic, img, p)
    rng = np.random.default_rng(2)
    sample = np.sort(rng.choice(16384, 24, replace=False))
    check_against_oracle(orc, img, got, 8, 2, 12, ranges=sample)


DENSE_CASES = [
    ("ct128", lambda: fic_synth.ct_slice(16, 128), 8, 4, 12),
    ("mr128", lambda: fic_synth.mr_slice(17, 128), 8, 4, 8),
    ("flat_regions", lambda: np.where(fic_synth.random_image(18, 64, 64, 8) > 100, 200, 10).astype(np.uint8), 8, 4, 8),
    ("constant", lambda: np.full((48, 48), 77, np.uint8), 8, 4, 8),
]


@pytest.mark.parametrize("name,make,n,t,B", DENSE_CASES, ids=[c[0] for c in DENSE_CASES])
@pytest.mark.parametrize("search", SEARCH)
def test_skipping_shadow_ranges_and_flat_domains_changes_nothing(fic, orc, name, make, n, t, B, search):
    """The default search skips shadow ranges and flat domains (Section V);
    FIC_FLAG_DENSE screens everything.  Both must give the same maps, and the
    dense maps must meet the oracle parity bar too."""
    img = make()
    p = fic.params(range_size=n, domain_stride=t, bit_depth=B, search=search_code(fic, search))
    pd = fic.params(range_size=n, domain_stride=t, bit_depth=B, search=search_code(fic, search),
                    flags=fic.FIC_FLAG_DENSE)
    a = gpu_encode(fic, img, p)
    b = gpu_encode(fic, img, pd)
    for f in ("domain_idx", "iso", "s_code", "o_code", "err"):
        assert np.array_equal(a[f], b[f]), f
    check_against_oracle(orc, img, b, n, t, B)


def test_host_and_device_pointers_agree(fic):
    img = fic_synth.ct_slice(14, 64)
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12)
    dev = gpu_encode(fic, img, p)
    host = fic.encode(img, p)
    assert np.array_equal(dev, host)


@pytest.mark.parametrize("layout", ["contiguous", "pitched", "unaligned"])
@pytest.mark.parametrize("B,n,t", [(12, 8, 4), (8, 8, 8)])
def test_pinned_host_buffers_agree(fic, B, n, t, layout):
    img = fic_synth.ct_slice(14, 64) if B == 12 else fic_synth.mr_slice(size=64)
    p = fic.params(range_size=n, domain_stride=t, bit_depth=B)
    rc, got = encode_pinned(fic, img, p, layout)
    assert rc == 0
    assert np.array_equal(got, gpu_encode(fic, img, p))
    assert np.array_equal(got, fic.encode(img, p))  # pageable host buffers: copy-engine path


@pytest.mark.parametrize("B,n,t", [(8, 8, 8), (12, 8, 4)])
def test_decode_parity(fic, orc, B, n, t):
    img = fic_synth.mr_slice(size=128) if B == 8 else fic_synth.ct_slice(15, 128)
    p = fic.params(range_size=n, domain_stride=t, bit_depth=B, decode_iters=10)
    maps = fic.encode(torch.from_numpy(img.astype(np.int16) if B > 8 else img).cuda(), p)
    out = fic.decode(maps, 128, 128, p)
    torch.cuda.synchronize()
    got = fic.maps_to_numpy(maps)
    ref = orc.decode(got["domain_idx"], got["iso"], got["s_code"] / ((1 << 4) - 1),
                     got["o_code"] * ((1 << B) - 1) / 63.0, 128, 128, n=n, t=t, bit_depth=B, iters=10)
    diff = np.abs(out.cpu().numpy().astype(np.float64) - ref)
    assert diff.max() < 2e-6 * (1 << B) * 10
    assert abs(orc.psnr(img, out.cpu().numpy(), B) - orc.psnr(img, ref, B)) < 0.01
    # host maps / host output path
    host = fic.decode(got, 128, 128, p)
    assert np.array_equal(host, out.cpu().numpy())


PSNR_CASES = [
    # the MR-like 256x256 8-bit slice, 8x8 ranges, domains at stride 8; the
    # CT-like 512x512 12-bit slice, 8x8 ranges, domains at stride 4
    ("mr256_t8", lambda: fic_synth.mr_slice(), 8, 8, 8),
    ("ct512_t4", lambda: fic_synth.ct_slice(), 8, 4, 12),
]


@pytest.fixture(scope="module")
def psnr_oracle(orc):
    """Per case: the oracle's own maps (exhaustive FP64 search) decoded by the
    FP64 oracle decoder (10 iterations from 2^(B-1)) and their PSNR."""
    cache = {}

    def get(name, img, n, t, B):
        if name not in cache:
            ref = orc.encode(img, n=n, t=t, bit_depth=B)
            Ls, Lo, P = 15.0, 63.0, float((1 << B) - 1)
            x = orc.decode(ref["d"], ref["k"], ref["c"] / Ls, ref["e"] * P / Lo, img.shape[0], img.shape[1], n=n,
                           t=t, bit_depth=B, iters=10)
            cache[name] = (ref, orc.psnr(img, x, B))
        return cache[name]

    return get


@pytest.mark.parametrize("name,make,n,t,B", PSNR_CASES, ids=[c[0] for c in PSNR_CASES])
@pytest.mark.parametrize("search", SEARCH)
def test_decoded_psnr_matches_oracle_maps(fic, orc, psnr_oracle, name, make, n, t, B, search):
    """The decoded PSNR of the GPU's own maps (GPU FP32 decode) within 0.01 dB
    of the oracle's own maps decoded by the FP64 oracle.  The two searches may
    pick different maps among equal residuals, so this checks the whole
    encode-decode chain, not the decoder alone."""
    img = make()
    ref, psnr_ref = psnr_oracle(name, img, n, t, B)
    p = fic.params(range_size=n, domain_stride=t, bit_depth=B, decode_iters=10, search=search_code(fic, search))
    dev_img = torch.from_numpy(img.astype(np.int16) if B > 8 else img).cuda()
    maps = fic.encode(dev_img, p)
    out = fic.decode(maps, img.shape[1], img.shape[0], p)
    torch.cuda.synchronize()
    psnr_gpu = orc.psnr(img, out.cpu().numpy(), B)
    assert abs(psnr_gpu - psnr_ref) < 0.01, (psnr_gpu, psnr_ref)
    # and the collage errors agree range by range (the maps' own parity)
    got = fic.maps_to_numpy(maps)
    assert np.all(got["err"] <= ref["err"] * (1 + 1e-5) + 1e-9 * n * n * ((1 << B) - 1) ** 2)


def test_decode_rejects_invalid_host_maps(fic):
    p = fic.params(range_size=8, domain_stride=8, bit_depth=8)
    maps = np.zeros(16, fic.MAP_DTYPE)
    maps["domain_idx"][3] = 10 ** 6
    with pytest.raises(fic.FicError):
        fic.decode(maps, 32, 32, p)


EXACT_CASES = [
    ("ct64_t4", lambda: fic_synth.ct_slice(19, 64), 8, 4, 12),
    ("mr64_t4", lambda: fic_synth.mr_slice(20, 64), 8, 4, 8),
    ("rand8_n4", lambda: fic_synth.random_image(21, 32, 32, 8), 4, 2, 8),
    ("ct12_n4", lambda: fic_synth.ct_slice(23, 64), 4, 2, 12),
    ("flat_regions", lambda: np.where(fic_synth.random_image(22, 48, 48, 8) > 100, 200, 10).astype(np.uint8), 8, 4, 8),
]


@pytest.mark.parametrize("name,make,n,t,B", EXACT_CASES, ids=[c[0] for c in EXACT_CASES])
@pytest.mark.parametrize("search", SEARCH)
def test_exact_scan_gives_the_screened_maps(fic, orc, name, make, n, t, B, search):
    """FIC_FLAG_EXACT_SCAN sends every screened range to the exhaustive exact
    scan (the path uncertified ranges take): the maps must be the screened
    search's, each flagged as resolved by the scan, and meet the oracle bar."""
    img = make()
    p = fic.params(range_size=n, domain_stride=t, bit_depth=B, search=search_code(fic, search))
    px = fic.params(range_size=n, domain_stride=t, bit_depth=B, search=search_code(fic, search),
                    flags=fic.FIC_FLAG_EXACT_SCAN)
    a = gpu_encode(fic, img, p)
    b = gpu_encode(fic, img, px)
    for f in ("domain_idx", "iso", "s_code", "o_code", "err"):
        assert np.array_equal(a[f], b[f]), f
    blocks = img.reshape(img.shape[0] // n, n, img.shape[1] // n, n).transpose(0, 2, 1, 3).reshape(-1, n * n)
    screened = blocks.max(1) != blocks.min(1)
    assert np.array_equal((b["info"] & fic.FIC_MAP_FALLBACK) != 0, screened)
    check_against_oracle(orc, img, b, n, t, B)


@pytest.mark.parametrize("search", SEARCH)
@pytest.mark.parametrize("n,sb,ob", [(8, 8, 10), (16, 6, 9), (8, 3, 4), (4, 8, 10)])
def test_encode_parity_other_code_widths(fic, orc, search, n, sb, ob):
    """s and o quantised to other bit widths (the 8/10-bit and 6/9-bit cases
    need 128-bit exact residuals; 3/4 bits is a coarse grid)."""
    img = fic_synth.ct_slice(23 + n + sb, 64)
    p = fic.params(range_size=n, domain_stride=4, bit_depth=12, s_bits=sb, o_bits=ob, search=search_code(fic, search))
    check_against_oracle(orc, img, gpu_encode(fic, img, p), n, 4, 12, sb=sb, ob=ob)


@pytest.mark.parametrize("scale_log2", [-1, 1, 2])
def test_decode_scaled_parity(fic, orc, scale_log2):
    img = fic_synth.ct_slice(24, 64)
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12, decode_iters=10)
    maps = fic.encode(torch.from_numpy(img.astype(np.int16)).cuda(), p)
    out = fic.decode_scaled(maps, 64, 64, p, scale_log2)
    torch.cuda.synchronize()
    got = fic.maps_to_numpy(maps)
    z = 2.0 ** scale_log2
    size, n, t = int(64 * z), int(8 * z), int(4 * z)
    ref = orc.decode(got["domain_idx"], got["iso"], got["s_code"] / 15.0, got["o_code"] * 4095 / 63.0, size, size,
                     n=n, t=t, bit_depth=12, iters=10)
    diff = np.abs(out.cpu().numpy().astype(np.float64) - ref)
    assert out.shape == (size, size)
    assert diff.max() < 2e-6 * 4096 * 10
    host = fic.decode_scaled(got, 64, 64, p, scale_log2)
    assert np.array_equal(host, out.cpu().numpy())
    if scale_log2 == 1:
        # 2x2 averages of the 2x decode match the unscaled decode (before the clamp: compare inside [0, P])
        base = fic.decode(maps, 64, 64, p).cpu().numpy().astype(np.float64)
        o = out.cpu().numpy().astype(np.float64)
        down = 0.25 * (o[0::2, 0::2] + o[1::2, 0::2] + o[0::2, 1::2] + o[1::2, 1::2])
        fine_in = (o > 0) & (o < 4095)
        inside = (base > 0) & (base < 4095) & fine_in[0::2, 0::2] & fine_in[1::2, 0::2] & fine_in[0::2, 1::2] \
            & fine_in[1::2, 1::2]
        assert np.abs(down - base)[inside].max() < 2e-6 * 4096 * 10


@pytest.mark.parametrize("search", SEARCH)
def test_failed_lists_rescan_gives_the_exact_maps(fic, orc, search):
    """High-contrast slices (a smooth bone ring offers many near-equal edge
    matches) leave some lists uncertified; those lists' candidates are then
    re-scanned exactly.  The maps must equal the all-exact scan's and meet the
    oracle bar, and the re-scan path must actually have run."""
    img = fic_synth.ct_slice(fic_synth.CT_SEED + 1000 + 72, 512)
    code = search_code(fic, search)
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12, search=code)
    px = fic.params(range_size=8, domain_stride=4, bit_depth=12, search=code, flags=fic.FIC_FLAG_EXACT_SCAN)
    a = gpu_encode(fic, img, p)
    b = gpu_encode(fic, img, px)
    assert int((a["info"] & fic.FIC_MAP_FALLBACK).sum()) > 0
    for f in ("domain_idx", "iso", "s_code", "o_code", "err"):
        assert np.array_equal(a[f], b[f]), f
    rng = np.random.default_rng(3)
    resc = np.nonzero(a["info"] & fic.FIC_MAP_FALLBACK)[0]
    sample = np.unique(np.concatenate([resc[:24], rng.choice(len(a), 24, replace=False)]))
    check_against_oracle(orc, img, a, 8, 4, 12, ranges=sample)



@pytest.mark.parametrize("search", SEARCH)
def test_codes_on_exact_rounding_ties(fic, orc, search):
    # the GPU decides the codes in FP32 from exact integers and defers to the
    # FP64 operation sequence next to a rounding boundary; here both ties are
    # exact, so that sequence (and the oracle) must give the rounded-away codes
    img = fic_synth.rounding_tie_image()
    ref = orc.encode(img.astype(np.float64), n=8, t=16, bit_depth=12)
    assert (ref["d"][15], ref["k"][15], ref["c"][15]) == (0, 0, 8) and ref["s_ls"][15] == 0.5
    assert (ref["d"][8], ref["k"][8], ref["c"][8], ref["e"][8]) == (0, 0, 0, 2) and ref["o_raw"][8] == 97.5
    p = fic.params(range_size=8, domain_stride=16, bit_depth=12, search=search_code(fic, search))
    got = gpu_encode(fic, img, p)
    check_against_oracle(orc, img.astype(np.float64), got, 8, 16, 12)
    for r in (15, 8):
        assert (got["domain_idx"][r], got["iso"][r], got["s_code"][r], got["o_code"][r]) == \
            (ref["d"][r], ref["k"][r], ref["c"][r], ref["e"][r]), r
