"""Pins of the oracle's adaptive quadtree against its definition (CPU).

The quadtree's per-level search is the oracle's exhaustive ``encode`` (pinned
in test_oracle_pins.py); these tests pin the tree logic: the split rule
(collage RMS sqrt(E/m) above the threshold splits a range into its four
quadrants, down to the minimum size), the level geometry (domains 2n x 2n at
stride n), exact tiling of the image by the leaves, and planted structures
whose tree is known in advance.
"""
import numpy as np
import pytest

import fic_synth


def tiles_exactly(leaves, h, w):
    cover = np.zeros((h, w), np.int32)
    for lf in leaves:
        cover[lf["y"]:lf["y"] + lf["n"], lf["x"]:lf["x"] + lf["n"]] += 1
    return np.all(cover == 1)


def test_constant_image_is_not_split(orc):
    img = np.full((64, 64), 128, np.uint8)
    lv = orc.encode_quadtree(img, 16, 4, 8.0, bit_depth=8)
    assert len(lv) == 16 and np.all(lv["level"] == 0) and np.all(lv["n"] == 16)
    assert tiles_exactly(lv, 64, 64)
    # s = 0 and the o code nearest 128 on the 7-bit grid: e = round(128*63/255) = 32
    assert np.all(lv["c"] == 0) and np.all(lv["e"] == 32)
    o_hat = 32 * 255 / 63
    assert np.allclose(lv["err"], 256 * (o_hat - 128) ** 2, rtol=1e-12)


def test_planted_noise_block_splits_to_the_minimum(orc):
    rng = np.random.default_rng(5)
    img = np.full((64, 64), 100, np.uint8)
    img[16:32, 16:32] = rng.integers(0, 256, (16, 16))
    lv = orc.encode_quadtree(img, 16, 4, 8.0, bit_depth=8)
    assert tiles_exactly(lv, 64, 64)
    big = lv[lv["level"] == 0]
    small = lv[lv["level"] == 2]
    assert len(big) == 15 and len(small) == 16 and len(lv) == 31
    assert not np.any((big["x"] == 16) & (big["y"] == 16))
    assert np.all((small["x"] >= 16) & (small["x"] < 32) & (small["y"] >= 16) & (small["y"] < 32))


def test_min_equal_max_is_a_plain_encode(orc):
    img = fic_synth.ct_slice(31, 64)
    lv = orc.encode_quadtree(img, 8, 8, 8.0, bit_depth=12)
    ref = orc.encode(img, n=8, t=8, bit_depth=12)
    assert np.array_equal(lv["range_idx"], np.arange(64))
    assert np.array_equal(lv["d"], ref["d"]) and np.array_equal(lv["k"], ref["k"])
    assert np.array_equal(lv["err"], ref["err"])


@pytest.mark.parametrize("make,B", [(lambda: fic_synth.ct_slice(32, 64), 12), (lambda: fic_synth.mr_slice(33, 64), 8)])
def test_tree_follows_the_split_rule(orc, make, B):
    img = make()
    thr = 8.0
    lv = orc.encode_quadtree(img, 16, 4, thr, bit_depth=B)
    h, w = img.shape
    assert tiles_exactly(lv, h, w)
    assert np.all(lv["n"] == 16 >> lv["level"])
    for level in range(3):
        n = 16 >> level
        nx = w // n
        sel = lv[lv["level"] == level]
        # every leaf's map is the exhaustive search at its level (domains at stride n)
        if len(sel):
            ref = orc.encode(img, n=n, t=n, bit_depth=B, ranges=sel["range_idx"])
            assert np.array_equal(sel["err"], ref["err"]) and np.array_equal(sel["d"], ref["d"])
            assert np.array_equal(sel["range_idx"], (sel["y"] // n) * nx + sel["x"] // n)
            if level < 2:  # kept above the minimum size: RMS at most the threshold
                assert np.all(np.sqrt(ref["err"] / (n * n)) <= thr)
        # every parent of a leaf below level 0 was split: its RMS exceeds the threshold
        if level > 0 and len(sel):
            pn = 2 * n
            pnx = w // pn
            parents = np.unique((sel["y"] // pn) * pnx + sel["x"] // pn).astype(np.int32)
            pref = orc.encode(img, n=pn, t=pn, bit_depth=B, ranges=parents)
            assert np.all(np.sqrt(pref["err"] / (pn * pn)) > thr)
