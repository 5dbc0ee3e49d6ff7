"""Seeded synthetic medical-like slices (inputs only).

The paper evaluates on unnamed black-and-white medical images (Section IV,
Section VIII) that are not available, so seeded synthetic slices with the
paper's sizes (256x256, 512x512, Section IV item 1) stand in for them.

This module holds no part of the encoding method: it only draws images.  It is
the one module that both the CUDA path's tests/bench and the FP64 oracle's
tests use, so that both sides see the same pixels.

Recipes (all float64 construction, then rint, clip, cast):

* ``mr_slice``  -- 8-bit MR-like slice: black background, one filled ellipse of
  intensity U(60,120), 3-6 Gaussian blobs (sigma U(5,20) px, amplitude
  U(-80,80)) centred inside it, a radial gradient g*(1-rho) inside it with
  g ~ U(10,30), additive N(0,4^2) noise everywhere, clipped to [0,255].
* ``ct_slice``  -- 12-bit CT-like slice (values 0..4095 in uint16): body
  ellipse U(900,1200), an elliptical bone ring at 0.85x the body axes with
  thickness U(0.02N,0.04N) and value U(2500,3500), N(0,20^2) texture inside
  the body, then 2-4 air pockets set to exactly 0, background 0.
* ``ct_stack``  -- a list of CT-like slices of mixed sizes (volume batches).
"""
from __future__ import annotations

import numpy as np

MR_SEED = 1404077401
CT_SEED = 1404077402


def _ellipse_frame(rng: np.random.Generator, h: int, w: int):
    """Random ellipse: returns (rho, inside) where rho is the normalised radius."""
    n = min(h, w)
    cy = h / 2.0 + rng.uniform(-0.05, 0.05) * n
    cx = w / 2.0 + rng.uniform(-0.05, 0.05) * n
    ay = rng.uniform(0.30, 0.45) * h
    ax = rng.uniform(0.30, 0.45) * w
    th = rng.uniform(0.0, np.pi)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    dy, dx = yy - cy, xx - cx
    u = dx * np.cos(th) + dy * np.sin(th)
    v = -dx * np.sin(th) + dy * np.cos(th)
    rho = np.sqrt((u / ax) ** 2 + (v / ay) ** 2)
    return rho, rho <= 1.0, (cy, cx, ay, ax, th), (yy, xx)


def _point_inside(rng, frame, rmax=0.8):
    cy, cx, ay, ax, th = frame
    r = rmax * np.sqrt(rng.uniform(0.0, 1.0))
    phi = rng.uniform(0.0, 2.0 * np.pi)
    u, v = r * ax * np.cos(phi), r * ay * np.sin(phi)
    x = cx + u * np.cos(th) - v * np.sin(th)
    y = cy + u * np.sin(th) + v * np.cos(th)
    return y, x


def mr_slice(seed: int = MR_SEED, size: int = 256) -> np.ndarray:
    """8-bit MR-like slice, shape (size, size), dtype uint8."""
    rng = np.random.default_rng(seed)
    h = w = size
    rho, inside, frame, (yy, xx) = _ellipse_frame(rng, h, w)
    img = np.zeros((h, w), np.float64)
    img[inside] = rng.uniform(60.0, 120.0)
    for _ in range(int(rng.integers(3, 7))):
        by, bx = _point_inside(rng, frame)
        sig = rng.uniform(5.0, 20.0)
        amp = rng.uniform(-80.0, 80.0)
        img += inside * amp * np.exp(-((yy - by) ** 2 + (xx - bx) ** 2) / (2.0 * sig * sig))
    g = rng.uniform(10.0, 30.0)
    img += inside * g * (1.0 - np.minimum(rho, 1.0))
    img += rng.normal(0.0, 4.0, (h, w))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def ct_slice(seed: int = CT_SEED, size: int = 512, width: int | None = None) -> np.ndarray:
    """12-bit CT-like slice, shape (size, width or size), dtype uint16, values 0..4095."""
    rng = np.random.default_rng(seed)
    h, w = size, (width or size)
    rho, inside, frame, (yy, xx) = _ellipse_frame(rng, h, w)
    n = min(h, w)
    img = np.zeros((h, w), np.float64)
    img[inside] = rng.uniform(900.0, 1200.0)
    mean_axis = 0.5 * (frame[2] + frame[3])
    thick = rng.uniform(0.02, 0.04) * n
    ring = np.abs(rho - 0.85) * mean_axis <= 0.5 * thick
    img[ring] = rng.uniform(2500.0, 3500.0)
    img += inside * rng.normal(0.0, 20.0, (h, w))
    for _ in range(int(rng.integers(2, 5))):
        py, px = _point_inside(rng, frame, rmax=0.6)
        ry = rng.uniform(0.03, 0.08) * n
        rx = rng.uniform(0.03, 0.08) * n
        img[((yy - py) / ry) ** 2 + ((xx - px) / rx) ** 2 <= 1.0] = 0.0
    return np.clip(np.rint(img), 0, 4095).astype(np.uint16)


def ct_stack(seed: int = CT_SEED, sizes=((256, 32), (384, 32), (512, 32))) -> list[np.ndarray]:
    """Mixed-size 12-bit CT-like volume: ``count`` slices of each ``size``."""
    out = []
    k = 0
    for size, count in sizes:
        for _ in range(count):
            out.append(ct_slice(seed + 1000 + k, size))
            k += 1
    return out


def random_image(seed: int, h: int, w: int, bit_depth: int) -> np.ndarray:
    """I.i.d. uniform pixels (worst-case texture) for parity tests."""
    rng = np.random.default_rng(seed)
    p = (1 << bit_depth) - 1
    dt = np.uint8 if bit_depth <= 8 else np.uint16
    return rng.integers(0, p + 1, (h, w)).astype(dt)


def rounding_tie_image(seed: int = 1404077499) -> np.ndarray:
    """32x32 12-bit image (8x8 ranges, 16x16 domains at stride 16) with two
    ranges whose best maps sit exactly on a rounding boundary of the 5-bit s /
    7-bit o quantiser: range 15 (rows/cols 24..31) equals a/2 + 1000 for the
    2x2 mean a of domain 0 (2x2-constant blocks of even values, so a/2 is an
    integer: least-squares s = 1/2, s * 15 = 7.5); range 8 (rows 16..23, cols
    0..7) is a 97/98 checkerboard (every candidate has |s * 15| < 1/2, so the
    offset is the mean 97.5 and o * 63 / 4095 = 1.5).  Uniform noise elsewhere."""
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 4096, size=(32, 32)).astype(np.uint16)
    w = rng.integers(50, 901, size=(8, 8))
    img[0:16, 0:16] = np.kron(2 * w, np.ones((2, 2), dtype=np.int64))
    img[24:32, 24:32] = w + 1000
    img[16:24, 0:8] = 97 + (np.add.outer(np.arange(8), np.arange(8)) % 2)
    return img
