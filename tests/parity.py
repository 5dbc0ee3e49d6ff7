"""Shared parity check of GPU maps against the FP64 oracle (test helper).

For every map the GPU returns, the oracle re-scores the same (range, domain,
symmetry): the s/o codes must be identical (both sides decide them in FP64
with the operation order of eq 9-12), the residual equal to 1e-12 relative
(the GPU reports the exact residual rounded once, the oracle sums squares in
FP64), and the stored s_hat, o_hat the FP32 roundings of the oracle's.  On
the checked ranges the residual must be within 1e-5 relative (plus
1e-9*m*P^2 absolute, for exact zeros) of the oracle's per-range minimum over
all 8*D candidates (Algorithm 2).  Index agreement with the oracle's choice is
returned, not required: equal residuals admit several correct maps.
"""
import numpy as np

REL = 1e-5


def abs_tol(n, B):
    return 1e-9 * n * n * ((1 << B) - 1) ** 2


def check_maps_rescored(orc, img, got, n, t, B, sb=5, ob=7):
    h, w = img.shape
    R = (h // n) * (w // n)
    assert len(got) == R
    assert np.array_equal(got["range_idx"], np.arange(R))
    for r in range(R):
        f = orc.fit_candidate(img, r, int(got["domain_idx"][r]), int(got["iso"][r]), n=n, t=t,
                              bit_depth=B, s_bits=sb, o_bits=ob)
        assert (f["c"], f["e"]) == (got["s_code"][r], got["o_code"][r]), r
        assert abs(f["err"] - got["err"][r]) <= 1e-12 * f["err"] + 1e-9, (r, f["err"], got["err"][r])
        assert np.float32(f["s_hat"]) == got["s"][r] and np.float32(f["o_hat"]) == got["o"][r]


def check_minima(got, ref, sel, n, B):
    e_gpu = got["err"][sel]
    bound = ref["err"] * (1 + REL) + abs_tol(n, B)
    bad = np.nonzero(e_gpu > bound)[0]
    assert bad.size == 0, f"ranges {np.asarray(sel)[bad][:10]} worse than the oracle minimum"
    return float(np.mean((got["domain_idx"][sel] == ref["d"]) & (got["iso"][sel] == ref["k"])))


def check_against_oracle(orc, img, got, n, t, B, sb=5, ob=7, ranges=None, ref=None):
    """Every map re-scored; minima on `ranges` (all by default).  `ref`: the
    oracle's encode of those ranges when the caller already has it."""
    check_maps_rescored(orc, img, got, n, t, B, sb, ob)
    h, w = img.shape
    sel = np.arange((h // n) * (w // n)) if ranges is None else np.asarray(ranges)
    if ref is None:
        ref = orc.encode(img, n=n, t=t, bit_depth=B, s_bits=sb, o_bits=ob, ranges=sel)
    return check_minima(got, ref, sel, n, B)


def encode_pinned(fic, img, p, layout="contiguous"):
    """fic_encode through the C ABI with the image and the maps in page-locked
    host memory: a contiguous, 16-byte aligned image is read by a copy kernel
    (layout "pitched": rows 8 elements longer than the image is wide, "unaligned":
    an image starting 2 bytes past an aligned address -- both go through the
    copy engines), and the maps are written by the map output kernel straight
    into the host buffer."""
    import ctypes

    import torch

    h, w = img.shape
    R, _ = fic.counts(w, h, p)
    src = img.astype(np.int16) if img.dtype == np.uint16 else img
    elem = src.dtype.itemsize
    if layout == "pitched":
        buf = torch.zeros((h, w + 8), dtype=torch.from_numpy(src[:1, :1].copy()).dtype).pin_memory()
        buf[:, :w] = torch.from_numpy(src.copy())
        ptr, pitch = buf.data_ptr(), w + 8
    elif layout == "unaligned":
        buf = torch.zeros(h * w + 16 // elem, dtype=torch.from_numpy(src[:1, :1].copy()).dtype).pin_memory()
        off = 2 // elem if elem == 2 else 2
        buf[off:off + h * w] = torch.from_numpy(src.copy().ravel())
        ptr, pitch = buf.data_ptr() + off * elem, w
    else:
        buf = torch.from_numpy(src.copy()).pin_memory()
        ptr, pitch = buf.data_ptr(), w
    h_maps = torch.full((R * 40,), 0xAB, dtype=torch.uint8).pin_memory()
    nm = ctypes.c_int()
    rc = fic.lib().fic_encode(ptr, w, h, pitch, ctypes.byref(p), h_maps.data_ptr(), R, ctypes.byref(nm),
                              None, 0, torch.cuda.current_stream().cuda_stream)
    return rc, h_maps.numpy().view(fic.MAP_DTYPE).copy()
