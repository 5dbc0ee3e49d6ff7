"""Parity of the adaptive quadtree encode (fic_encode_quadtree, through the C
ABI) with the FP64 oracle's quadtree.

Small images: the leaf sets (level, position, size) must be identical, and
every leaf's map must meet the encode parity bar at its level (codes equal to
the oracle's for the same candidate, residual within 1e-12, and within 1e-5
relative of the oracle's minimum).  The 512x512 CT slice: the tree must tile
the image, and sampled leaves and parents must satisfy the split rule against
the oracle's per-range minima.
"""
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


def gpu_quadtree(fic, img, p, min_size, thr, device=True):
    if device:
        t = torch.from_numpy(img.astype(np.int16) if img.dtype == np.uint16 else img).cuda()
        maps, n = fic.encode_quadtree(t, p, min_size, thr)
        torch.cuda.synchronize()
        return fic.qmaps_to_numpy(maps, n)
    leaves, n = fic.encode_quadtree(img, p, min_size, thr)
    return leaves


def check_leaves(orc, img, got, B, sb=5, ob=7):
    h, w = img.shape
    m_all = got["map"]
    for lf, mp in zip(got, m_all):
        n = int(lf["size"])
        f = orc.fit_candidate(img, int(mp["range_idx"]), int(mp["domain_idx"]), int(mp["iso"]), n=n, t=n,
                              bit_depth=B, s_bits=sb, o_bits=ob)
        assert (f["c"], f["e"]) == (mp["s_code"], mp["o_code"])
        assert abs(f["err"] - mp["err"]) <= 1e-12 * f["err"] + 1e-9
        assert mp["range_idx"] == (lf["y"] // n) * (w // n) + lf["x"] // n


CASES = [
    ("ct64", lambda: fic_synth.ct_slice(41, 64), 12, 16, 4),
    ("mr64", lambda: fic_synth.mr_slice(42, 64), 8, 16, 4),
    ("ct96x64_8to4", lambda: fic_synth.ct_slice(43, 96)[:64], 12, 8, 4),
    ("rand_16to8", lambda: fic_synth.random_image(44, 64, 64, 8), 8, 16, 8),
    ("constant", lambda: np.full((64, 64), 700, np.uint16), 12, 16, 4),
]


@pytest.mark.parametrize("name,make,B,nmax,nmin", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("search", ["auto", "simt"])
def test_quadtree_parity_small(fic, orc, name, make, B, nmax, nmin, search):
    img = make()
    code = {"auto": fic.FIC_SEARCH_AUTO, "simt": fic.FIC_SEARCH_SIMT}[search]
    p = fic.params(range_size=nmax, domain_stride=nmax, bit_depth=B, search=code)
    got = gpu_quadtree(fic, img, p, nmin, 8.0)
    ref = orc.encode_quadtree(img, nmax, nmin, 8.0, bit_depth=B)
    key = lambda a, lvl, x, y, n: list(zip(a[lvl], a[x], a[y], a[n]))
    assert key(got, "level", "x", "y", "size") == key(ref, "level", "x", "y", "n")
    check_leaves(orc, img, got, B)
    e_gpu = got["map"]["err"]
    bound = ref["err"] * (1 + 1e-5) + 1e-9 * (nmax * nmax) * ((1 << B) - 1) ** 2
    assert np.all(e_gpu <= bound)


def test_quadtree_host_and_device_agree(fic):
    img = fic_synth.ct_slice(45, 64)
    p = fic.params(range_size=16, domain_stride=16, bit_depth=12)
    a = gpu_quadtree(fic, img, p, 4, 8.0, device=True)
    b = gpu_quadtree(fic, img, p, 4, 8.0, device=False)
    assert np.array_equal(a, b)


def test_quadtree_pinned_host_buffers_agree(fic):
    """A page-locked host image (read by a copy kernel) and page-locked host
    leaves (written in place by the gather kernel) give the device path's leaves."""
    img = fic_synth.ct_slice(45, 64)
    p = fic.params(range_size=16, domain_stride=16, bit_depth=12)
    a = gpu_quadtree(fic, img, p, 4, 8.0, device=True)
    h_img = torch.from_numpy(img.astype(np.int16)).pin_memory()
    cap = (64 // 4) ** 2
    h_maps = torch.zeros(cap * fic.QMAP_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    leaves, n = fic.encode_quadtree(h_img.numpy().view(np.uint16), p, 4, 8.0,
                                    maps=h_maps.numpy().view(fic.QMAP_DTYPE))
    assert n == len(a)
    assert np.array_equal(np.asarray(leaves), a)


def test_quadtree_rejects_bad_sizes(fic):
    img = np.zeros((64, 64), np.uint8)
    with pytest.raises(fic.FicError):
        fic.encode_quadtree(img, fic.params(range_size=16, bit_depth=8), 2, 8.0)
    with pytest.raises(fic.FicError):
        fic.encode_quadtree(img, fic.params(range_size=8, bit_depth=8), 16, 8.0)
    with pytest.raises(fic.FicError):
        fic.encode_quadtree(np.zeros((40, 64), np.uint8), fic.params(range_size=16, bit_depth=8), 4, 8.0)


def test_quadtree_ct512_sampled(fic, orc):
    """The 512x512 12-bit CT slice, 16 -> 8 -> 4, RMS 8.0, in the bench's configuration."""
    img = fic_synth.ct_slice()
    p = fic.params(range_size=16, domain_stride=16, bit_depth=12)
    got = gpu_quadtree(fic, img, p, 4, 8.0)
    cover = np.zeros(img.shape, np.int32)
    for lf in got:
        cover[lf["y"]:lf["y"] + lf["size"], lf["x"]:lf["x"] + lf["size"]] += 1
    assert np.all(cover == 1)
    stats = fic.last_quadtree_stats()
    assert stats[0] == 3
    rng = np.random.default_rng(1)
    for level in range(3):
        n = 16 >> level
        sel = got[got["level"] == level]
        if not len(sel):
            continue
        pick = sel[rng.choice(len(sel), min(12, len(sel)), replace=False)]
        check_leaves(orc, img, pick, 12)
        ref = orc.encode(img, n=n, t=n, bit_depth=12, ranges=pick["map"]["range_idx"].astype(np.int32))
        assert np.all(pick["map"]["err"] <= ref["err"] * (1 + 1e-5) + 1e-9 * n * n * 4095 ** 2)
        if level < 2:
            assert np.all(np.sqrt(ref["err"] / (n * n)) <= 8.0)
        if level > 0:
            pn = 2 * n
            parents = np.unique((pick["y"] // pn) * (512 // pn) + pick["x"] // pn).astype(np.int32)
            pref = orc.encode(img, n=pn, t=pn, bit_depth=12, ranges=parents)
            assert np.all(np.sqrt(pref["err"] / (pn * pn)) > 8.0)
