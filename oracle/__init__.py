"""FP64 CPU oracle for PIFS fractal encoding (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  The product library (``paper_1404_0774_gb300``)
never imports it, and the two share no code: the arithmetic lives in
``fic_oracle.c`` (plain C, IEEE double, no FMA contraction), this module only
marshals numpy arrays through ctypes.

Functions follow Haque et al. (arXiv 1404.0774), Section V:
``encode`` is the exhaustive search of Algorithm 2/3 with the least squares of
eq 9-12 and the residual of eq 8; ``fit_candidate`` evaluates one
(range, domain, symmetry) triple; ``decode`` iterates the maps (the decoder the
abstract and Section VI refer to); ``psnr`` scores a decoded image.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fic_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libfic_oracle.so")
_lock = threading.Lock()
_lib = None


class OrcParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("t", ctypes.c_int32), ("bit_depth", ctypes.c_int32),
                ("s_bits", ctypes.c_int32), ("o_bits", ctypes.c_int32)]


class OrcFit(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("k", ctypes.c_int32), ("c", ctypes.c_int32),
                ("e", ctypes.c_int32), ("s_ls", ctypes.c_double), ("s_hat", ctypes.c_double),
                ("o_raw", ctypes.c_double), ("o_hat", ctypes.c_double), ("err", ctypes.c_double)]


FIT_DTYPE = np.dtype([("d", np.int32), ("k", np.int32), ("c", np.int32), ("e", np.int32),
                      ("s_ls", np.float64), ("s_hat", np.float64), ("o_raw", np.float64),
                      ("o_hat", np.float64), ("err", np.float64)])
assert FIT_DTYPE.itemsize == ctypes.sizeof(OrcFit)


def build(force: bool = False) -> str:
    """Compile fic_oracle.c into a shared library (gcc, -O2, OpenMP if available)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                "-shared", _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)  # serial build
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        pp = ctypes.POINTER(OrcParams)
        fp = ctypes.POINTER(OrcFit)
        lib.orc_encode.argtypes = [dp, ctypes.c_int, ctypes.c_int, pp, ip, ctypes.c_int, fp, ctypes.c_int]
        lib.orc_fit_candidate.argtypes = [dp, ctypes.c_int, ctypes.c_int, pp, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, fp]
        lib.orc_decode.argtypes = [ctypes.c_int, ctypes.c_int, pp, ip, ip, dp, dp, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, dp, dp]
        lib.orc_refine_grad.argtypes = [ctypes.c_int, ctypes.c_int, pp, ip, ip, dp, dp, ctypes.c_int,
                                        ctypes.c_double, dp, dp, dp, dp]
        lib.orc_psnr.argtypes = [dp, dp, ctypes.c_size_t, ctypes.c_int]
        lib.orc_psnr.restype = ctypes.c_double
        lib.orc_num_domains_x.argtypes = [ctypes.c_int, pp]
        lib.orc_num_domains_y.argtypes = [ctypes.c_int, pp]
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def params(n=8, t=8, bit_depth=8, s_bits=5, o_bits=7) -> OrcParams:
    return OrcParams(n, t, bit_depth, s_bits, o_bits)


def counts(h: int, w: int, n: int, t: int):
    """(ranges, domains) of an h x w image: (h/n)(w/n) and ((h-2n)/t+1)((w-2n)/t+1)."""
    return (h // n) * (w // n), ((h - 2 * n) // t + 1) * ((w - 2 * n) // t + 1)


def encode(img, n=8, t=8, bit_depth=8, s_bits=5, o_bits=7, ranges=None, threads=None):
    """Exhaustive search; returns a FIT_DTYPE record per listed range (all by default)."""
    lib = _load()
    im = np.ascontiguousarray(img, dtype=np.float64)
    h, w = im.shape
    if h % n or w % n or h < 2 * n or w < 2 * n:
        raise ValueError("image sides must be multiples of n and at least 2n")
    if ranges is None:
        ranges = np.arange((h // n) * (w // n), dtype=np.int32)
    rl = np.ascontiguousarray(ranges, dtype=np.int32)
    out = np.zeros(len(rl), FIT_DTYPE)
    p = params(n, t, bit_depth, s_bits, o_bits)
    nt = threads if threads is not None else (os.cpu_count() or 1)
    rc = lib.orc_encode(_dptr(im), w, h, ctypes.byref(p), _iptr(rl), len(rl),
                        out.ctypes.data_as(ctypes.POINTER(OrcFit)), nt)
    if rc != 0:
        raise MemoryError("oracle encode failed")
    return out


def fit_candidate(img, r, d, k, n=8, t=8, bit_depth=8, s_bits=5, o_bits=7):
    """Least squares, quantisation and residual of one (range, domain, symmetry)."""
    lib = _load()
    im = np.ascontiguousarray(img, dtype=np.float64)
    h, w = im.shape
    p = params(n, t, bit_depth, s_bits, o_bits)
    f = OrcFit()
    if lib.orc_fit_candidate(_dptr(im), w, h, ctypes.byref(p), int(r), int(d), int(k), ctypes.byref(f)):
        raise MemoryError("oracle fit failed")
    out = np.zeros((), FIT_DTYPE)
    ctypes.memmove(out.ctypes.data, ctypes.addressof(f), FIT_DTYPE.itemsize)
    return out[()]


def decode(dom, sym, s_hat, o_hat, h, w, n=8, t=8, bit_depth=8, iters=10, init=None,
           clamp=True, trace=False):
    """Iterate the maps; returns the decoded image (and all iterates if trace)."""
    lib = _load()
    p = params(n, t, bit_depth, 0, 0)
    dom = np.ascontiguousarray(dom, np.int32)
    sym = np.ascontiguousarray(sym, np.int32)
    sh = np.ascontiguousarray(s_hat, np.float64)
    oh = np.ascontiguousarray(o_hat, np.float64)
    if init is None:
        init = float(1 << (bit_depth - 1))
    out = np.zeros((h, w), np.float64)
    tr = np.zeros((iters + 1, h, w), np.float64) if trace else None
    rc = lib.orc_decode(w, h, ctypes.byref(p), _iptr(dom), _iptr(sym), _dptr(sh), _dptr(oh),
                        int(iters), float(init), int(bool(clamp)), _dptr(out),
                        _dptr(tr) if trace else ctypes.POINTER(ctypes.c_double)())
    if rc != 0:
        raise MemoryError("oracle decode failed")
    return (out, tr) if trace else out


def psnr(ref, img, bit_depth):
    lib = _load()
    a = np.ascontiguousarray(ref, np.float64)
    b = np.ascontiguousarray(img, np.float64)
    return float(lib.orc_psnr(_dptr(a), _dptr(b), a.size, bit_depth))


QT_DTYPE = np.dtype([("level", np.int32), ("x", np.int32), ("y", np.int32), ("n", np.int32),
                     ("range_idx", np.int32), ("d", np.int32), ("k", np.int32), ("c", np.int32),
                     ("e", np.int32), ("err", np.float64)])


def encode_quadtree(img, n_max=16, n_min=4, rms_split=8.0, bit_depth=8, s_bits=5, o_bits=7, threads=None):
    """Adaptive quadtree by its definition: level 0 tiles the image with n_max
    ranges; every range whose best map (the exhaustive search of ``encode`` at
    that level: domains 2n x 2n at stride n) has collage RMS error
    sqrt(E/m) > rms_split is replaced by its four quadrants at the next level,
    down to n_min, whose ranges are all kept.  Returns the kept leaves
    (QT_DTYPE) ordered by level, then range index within the level."""
    im = np.asarray(img)
    h, w = im.shape
    thr = float(rms_split)
    leaves = []
    n, level = n_max, 0
    active = np.arange((h // n) * (w // n), dtype=np.int32)
    while len(active):
        nx = w // n
        fits = encode(im, n=n, t=n, bit_depth=bit_depth, s_bits=s_bits, o_bits=o_bits, ranges=active,
                      threads=threads)
        rms = np.sqrt(fits["err"] / float(n * n))
        split = (rms > thr) & (n > n_min)
        for r, f in zip(active[~split], fits[~split]):
            leaves.append((level, (r % nx) * n, (r // nx) * n, n, r, f["d"], f["k"], f["c"], f["e"], f["err"]))
        children = []
        for r in active[split]:
            ry, rx = divmod(int(r), nx)
            for dy in (0, 1):
                for dx in (0, 1):
                    children.append((2 * ry + dy) * (2 * nx) + 2 * rx + dx)
        active = np.array(sorted(children), dtype=np.int32)
        n //= 2
        level += 1
    out = np.array(leaves, dtype=QT_DTYPE)
    return out[np.lexsort((out["range_idx"], out["level"]))]


def refine_grad(dom, sym, s, o, ref, n=8, t=8, bit_depth=8, iters=8, init=None):
    """Loss (1/N) sum (x_T - ref)^2 of the unrolled unclamped decode with real
    s, o per range, and its FP64 gradient (dL/ds, dL/do) by the adjoint of
    the iteration.  Returns (loss, grad_s, grad_o)."""
    lib = _load()
    ref = np.ascontiguousarray(ref, np.float64)
    h, w = ref.shape
    p = params(n, t, bit_depth, 0, 0)
    dom = np.ascontiguousarray(dom, np.int32)
    sym = np.ascontiguousarray(sym, np.int32)
    s = np.ascontiguousarray(s, np.float64)
    o = np.ascontiguousarray(o, np.float64)
    if init is None:
        init = float(1 << (bit_depth - 1))
    gs = np.zeros(len(s), np.float64)
    go = np.zeros(len(s), np.float64)
    loss = ctypes.c_double()
    rc = lib.orc_refine_grad(w, h, ctypes.byref(p), _iptr(dom), _iptr(sym), _dptr(s), _dptr(o), int(iters),
                             float(init), _dptr(ref), ctypes.byref(loss), _dptr(gs), _dptr(go))
    if rc != 0:
        raise MemoryError("oracle refine_grad failed")
    return loss.value, gs, go
