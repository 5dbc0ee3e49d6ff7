"""Thin ctypes binding of libfic.so (include/fic.h).

Argument marshalling only: every step of encoding and decoding runs in the
library's CUDA kernels.  Device buffers are torch CUDA tensors (torch is used
for device memory and streams only); host buffers are numpy arrays.  If the
compiled library is missing this module raises on import of any entry point:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libfic.so")

FIC_OK = 0
FIC_SEARCH_AUTO, FIC_SEARCH_TC, FIC_SEARCH_SIMT = 0, 1, 2
FIC_MAP_FALLBACK = 0x1
FIC_FLAG_PHASE_TIMING = 0x1
FIC_FLAG_DENSE = 0x2
FIC_FLAG_EXACT_SCAN = 0x4
STATUS = {0: "ok", -1: "bad argument", -2: "bad size", -3: "bad bit depth", -4: "capacity",
          -5: "cuda error", -6: "timeout", -7: "unsupported"}


class FicError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


class fic_params(ctypes.Structure):
    _fields_ = [("range_size", ctypes.c_int32), ("domain_stride", ctypes.c_int32),
                ("bit_depth", ctypes.c_int32), ("s_bits", ctypes.c_int32), ("o_bits", ctypes.c_int32),
                ("decode_iters", ctypes.c_int32), ("search", ctypes.c_int32), ("n_split", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


MAP_DTYPE = np.dtype([("range_idx", np.uint32), ("domain_idx", np.uint32), ("iso", np.int32),
                      ("s_code", np.int32), ("o_code", np.int32), ("s", np.float32), ("o", np.float32),
                      ("info", np.uint32), ("err", np.float64)])
assert MAP_DTYPE.itemsize == 40
QMAP_DTYPE = np.dtype([("x", np.uint32), ("y", np.uint32), ("size", np.uint32), ("level", np.uint32),
                       ("map", MAP_DTYPE)])
assert QMAP_DTYPE.itemsize == 56

_lib = None


def lib():
    """Load libfic.so (build it first with paper_1404_0774_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libfic.so not built: {_LIB_PATH} is missing (run __graft_entry__.build())")
        L = ctypes.CDLL(_LIB_PATH)
        vp, sz, i64p = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)
        pp = ctypes.POINTER(fic_params)
        L.fic_default_params.argtypes = [pp]
        L.fic_default_params.restype = None
        L.fic_counts.argtypes = [ctypes.c_int, ctypes.c_int, pp, i64p, i64p]
        L.fic_encode_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int, pp, ctypes.POINTER(sz)]
        L.fic_decode_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int, pp, ctypes.POINTER(sz)]
        L.fic_encode.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, pp, vp, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int), vp, sz, vp]
        L.fic_decode.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, pp, ctypes.c_float, vp, vp,
                                 sz, vp]
        L.fic_status_str.argtypes = [ctypes.c_int]
        L.fic_status_str.restype = ctypes.c_char_p
        L.fic_last_encode_stats.argtypes = [i64p]
        L.fic_last_encode_phase_ms.argtypes = [ctypes.POINTER(ctypes.c_double)]
        L.fic_cross_terms.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, pp, vp, vp, sz, vp]
        L.fic_encode_static.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, pp, vp, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), vp]
        L.fic_encode_quadtree.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, pp, ctypes.c_int,
                                          ctypes.c_float, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp, sz, vp]
        L.fic_quadtree_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int, pp, ctypes.c_int, ctypes.POINTER(sz)]
        L.fic_last_quadtree_stats.argtypes = [i64p]
        L.fic_last_quadtree_phase_ms.argtypes = [ctypes.POINTER(ctypes.c_double)]
        L.fic_encode_batch.argtypes = [vp, ctypes.c_int, pp, vp, sz, vp]
        L.fic_batch_workspace_size.argtypes = [vp, ctypes.c_int, pp, ctypes.POINTER(sz)]
        L.fic_last_batch_slice_ms.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_int]
        L.fic_decode_scaled.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, pp, ctypes.c_int,
                                        ctypes.c_float, vp, vp, sz, vp]
        L.fic_decode_scaled_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int, pp, ctypes.c_int,
                                                       ctypes.POINTER(sz)]
        L.fic_refine_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int, pp, ctypes.c_int, ctypes.POINTER(sz)]
        L.fic_refine_forward.argtypes = [vp, ctypes.c_int, ctypes.c_int, pp, vp, vp, ctypes.c_float, ctypes.c_int,
                                         vp, vp, vp, sz, vp]
        L.fic_refine_backward.argtypes = [vp, ctypes.c_int, ctypes.c_int, pp, vp, vp, ctypes.c_int, vp, vp, vp, vp,
                                          vp, sz, vp]
        L.fic_refine.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, pp, vp, vp, vp, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_float, vp, vp, sz, vp]
        L.fic_set_wait_limit_ns.argtypes = [ctypes.c_uint64]
        L.fic_get_wait_limit_ns.argtypes = []
        L.fic_get_wait_limit_ns.restype = ctypes.c_uint64
        _lib = L
    return _lib


def params(range_size=8, domain_stride=8, bit_depth=8, s_bits=5, o_bits=7, decode_iters=10,
           search=FIC_SEARCH_AUTO, n_split=0, flags=0) -> fic_params:
    return fic_params(range_size, domain_stride, bit_depth, s_bits, o_bits, decode_iters, search, n_split,
                      flags)


def _check(rc: int, what: str):
    if rc != FIC_OK:
        raise FicError(rc, what)


def counts(w: int, h: int, p: fic_params):
    r, d = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().fic_counts(w, h, ctypes.byref(p), ctypes.byref(r), ctypes.byref(d)), "fic_counts")
    return r.value, d.value


def encode_workspace_size(w: int, h: int, p: fic_params) -> int:
    b = ctypes.c_size_t()
    _check(lib().fic_encode_workspace_size(w, h, ctypes.byref(p), ctypes.byref(b)), "fic_encode_workspace_size")
    return b.value


def decode_workspace_size(w: int, h: int, p: fic_params) -> int:
    b = ctypes.c_size_t()
    _check(lib().fic_decode_workspace_size(w, h, ctypes.byref(p), ctypes.byref(b)), "fic_decode_workspace_size")
    return b.value


def _stream_ptr(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def encode(img, p: fic_params, maps=None, workspace=None, stream=None):
    """Encode one image.

    img: torch CUDA tensor (uint8, or int16/uint16 holding values < 2^12) or a
    numpy array (host).  Returns maps: for a CUDA image a torch uint8 tensor of
    R*40 bytes on the same device (view with ``maps_to_numpy``), for a host
    image a numpy MAP_DTYPE array.  ``workspace`` is an optional device byte
    tensor of at least ``encode_workspace_size`` bytes.
    """
    h, w = int(img.shape[0]), int(img.shape[1])
    R, _ = counts(w, h, p)
    if _is_torch(img):
        import torch

        if not img.is_cuda:
            raise ValueError("torch image must be on a CUDA device")
        pitch = int(img.stride(0))
        if img.stride(1) != 1:
            raise ValueError("image rows must be contiguous")
        if maps is None:
            maps = torch.empty(R * MAP_DTYPE.itemsize, dtype=torch.uint8, device=img.device)
        img_ptr, maps_ptr = img.data_ptr(), maps.data_ptr()
        st = _stream_ptr(stream)
    else:
        a = np.ascontiguousarray(img, dtype=np.uint8 if p.bit_depth <= 8 else np.uint16)
        img = a
        pitch = w
        if maps is None:
            maps = np.zeros(R, MAP_DTYPE)
        img_ptr, maps_ptr = a.ctypes.data, maps.ctypes.data
        st = 0 if stream is None else _stream_ptr(stream)
    ws_ptr, ws_bytes = (None, 0)
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    n = ctypes.c_int()
    _check(lib().fic_encode(img_ptr, w, h, pitch, ctypes.byref(p), maps_ptr, R, ctypes.byref(n), ws_ptr,
                            ws_bytes, st), "fic_encode")
    return maps


def decode(maps, w: int, h: int, p: fic_params, init: float | None = None, out=None, workspace=None,
           stream=None):
    """Decode maps (device tensor or host MAP_DTYPE array) into a w x h float32 image."""
    R, _ = counts(w, h, p)
    if init is None:
        init = float(1 << (p.bit_depth - 1))
    if _is_torch(maps):
        import torch

        if out is None:
            out = torch.empty((h, w), dtype=torch.float32, device=maps.device)
        maps_ptr, out_ptr, st = maps.data_ptr(), out.data_ptr(), _stream_ptr(stream)
    else:
        maps = np.ascontiguousarray(maps, MAP_DTYPE)
        if out is None:
            out = np.zeros((h, w), np.float32)
        maps_ptr, out_ptr = maps.ctypes.data, out.ctypes.data
        st = 0 if stream is None else _stream_ptr(stream)
    ws_ptr, ws_bytes = (None, 0)
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    _check(lib().fic_decode(maps_ptr, R, w, h, ctypes.byref(p), ctypes.c_float(init), out_ptr, ws_ptr, ws_bytes,
                            st), "fic_decode")
    return out


def quadtree_workspace_size(w: int, h: int, p: fic_params, min_size: int = 4) -> int:
    b = ctypes.c_size_t()
    _check(lib().fic_quadtree_workspace_size(w, h, ctypes.byref(p), min_size, ctypes.byref(b)),
           "fic_quadtree_workspace_size")
    return b.value


def encode_quadtree(img, p: fic_params, min_size: int = 4, rms_split: float = 8.0, maps=None, workspace=None,
                    stream=None):
    """Adaptive quadtree encode (p.range_size = largest block).  Returns
    (leaves, n): for a CUDA image a torch uint8 tensor of capacity*56 bytes on
    the device whose first n records are the leaves (view with
    ``qmaps_to_numpy``), for a host image a QMAP_DTYPE numpy array of n leaves."""
    h, w = int(img.shape[0]), int(img.shape[1])
    cap = (w // min_size) * (h // min_size)
    if _is_torch(img):
        import torch

        if not img.is_cuda or img.stride(1) != 1:
            raise ValueError("torch image must be on a CUDA device with contiguous rows")
        pitch = int(img.stride(0))
        if maps is None:
            maps = torch.empty(cap * QMAP_DTYPE.itemsize, dtype=torch.uint8, device=img.device)
        img_ptr, maps_ptr, st = img.data_ptr(), maps.data_ptr(), _stream_ptr(stream)
    else:
        a = np.ascontiguousarray(img, dtype=np.uint8 if p.bit_depth <= 8 else np.uint16)
        img = a
        pitch = w
        if maps is None:
            maps = np.zeros(cap, QMAP_DTYPE)
        img_ptr, maps_ptr = a.ctypes.data, maps.ctypes.data
        st = 0 if stream is None else _stream_ptr(stream)
    ws_ptr, ws_bytes = (None, 0)
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    n = ctypes.c_int()
    _check(lib().fic_encode_quadtree(img_ptr, w, h, pitch, ctypes.byref(p), int(min_size), ctypes.c_float(rms_split),
                                     maps_ptr, cap, ctypes.byref(n), ws_ptr, ws_bytes, st), "fic_encode_quadtree")
    if not _is_torch(maps):
        return maps[: n.value], n.value
    return maps, n.value


def qmaps_to_numpy(maps, n: int) -> np.ndarray:
    """The first n leaves of a device quadtree maps tensor as a host QMAP_DTYPE array."""
    if _is_torch(maps):
        return maps[: n * QMAP_DTYPE.itemsize].detach().cpu().numpy().view(QMAP_DTYPE)
    return np.asarray(maps, QMAP_DTYPE)[:n]


def last_quadtree_stats():
    """[levels, then per level: search kernel, CTA target, ranges screened, leaves]."""
    out = (ctypes.c_int64 * 17)()
    _check(lib().fic_last_quadtree_stats(out), "fic_last_quadtree_stats")
    return list(out)


def last_quadtree_phase_ms():
    """Search ms of each level of the last quadtree encode run with
    FIC_FLAG_PHASE_TIMING (waits for its events)."""
    out = (ctypes.c_double * 3)()
    _check(lib().fic_last_quadtree_phase_ms(out), "fic_last_quadtree_phase_ms")
    return list(out)


class fic_slice(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("w", ctypes.c_int32), ("h", ctypes.c_int32), ("pitch_px", ctypes.c_int32),
                ("maps", ctypes.c_void_p)]


def slice_table(imgs, maps):
    """ctypes array of fic_slice for lists of CUDA image tensors and maps tensors."""
    tab = (fic_slice * len(imgs))()
    for i, (im, mp) in enumerate(zip(imgs, maps)):
        if not (im.is_cuda and mp.is_cuda) or im.stride(1) != 1:
            raise ValueError("batch images and maps must be CUDA tensors with contiguous rows")
        tab[i] = fic_slice(im.data_ptr(), int(im.shape[1]), int(im.shape[0]), int(im.stride(0)), mp.data_ptr())
    return tab


def batch_workspace_size(table, p: fic_params) -> int:
    b = ctypes.c_size_t()
    _check(lib().fic_batch_workspace_size(table, len(table), ctypes.byref(p), ctypes.byref(b)),
           "fic_batch_workspace_size")
    return b.value


def encode_batch(table, p: fic_params, workspace, stream=None):
    """Encode every slice of ``table`` (from ``slice_table``); asynchronous on the stream."""
    _check(lib().fic_encode_batch(table, len(table), ctypes.byref(p), workspace.data_ptr(),
                                  workspace.numel() * workspace.element_size(), _stream_ptr(stream)),
           "fic_encode_batch")


def last_batch_slice_ms(n: int):
    out = (ctypes.c_float * n)()
    _check(lib().fic_last_batch_slice_ms(out, n), "fic_last_batch_slice_ms")
    return list(out)


def refine_workspace_size(w: int, h: int, p: fic_params, iters: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().fic_refine_workspace_size(w, h, ctypes.byref(p), iters, ctypes.byref(b)),
           "fic_refine_workspace_size")
    return b.value


def map_coefficients(maps):
    """(s, o) as float32 CUDA tensors (one per range) from a device maps tensor."""
    import torch

    f = maps.view(-1, MAP_DTYPE.itemsize)[:, 20:28].contiguous().view(torch.float32)
    return f[:, 0].clone(), f[:, 1].clone()


def _decode_fn():
    import torch

    class DecodeFn(torch.autograd.Function):
        """x_T of the unrolled decoder as a function of (s, o); backward runs
        the library's adjoint kernels (checkpointed every second iterate)."""

        @staticmethod
        def forward(ctx, s, o, maps, w, h, p, iters, init, ws):
            x = torch.empty((h, w), dtype=torch.float32, device=s.device)
            ckpt = torch.empty(((iters + 1) // 2) * h * w, dtype=torch.float32, device=s.device)
            st = _stream_ptr(None)
            _check(lib().fic_refine_forward(maps.data_ptr(), w, h, ctypes.byref(p), s.data_ptr(), o.data_ptr(),
                                            ctypes.c_float(init), iters, x.data_ptr(), ckpt.data_ptr(),
                                            ws.data_ptr(), ws.numel(), st), "fic_refine_forward")
            ctx.save_for_backward(s, o, ckpt)
            ctx.meta = (maps, w, h, p, iters, ws)
            return x

        @staticmethod
        def backward(ctx, gx):
            s, o, ckpt = ctx.saved_tensors
            maps, w, h, p, iters, ws = ctx.meta
            gx = gx.contiguous()
            gs, go = torch.empty_like(s), torch.empty_like(o)
            _check(lib().fic_refine_backward(maps.data_ptr(), w, h, ctypes.byref(p), s.data_ptr(), o.data_ptr(),
                                             iters, ckpt.data_ptr(), gx.data_ptr(), gs.data_ptr(), go.data_ptr(),
                                             ws.data_ptr(), ws.numel(), _stream_ptr(None)), "fic_refine_backward")
            return gs, go, None, None, None, None, None, None, None

    return DecodeFn


_DecodeFn = None


def decode_differentiable(s, o, maps, w: int, h: int, p: fic_params, iters: int = 8, init: float | None = None,
                          workspace=None):
    """x_T (h x w float32 CUDA tensor) of the unrolled, unclamped decoder with
    real-valued s, o (CUDA float32, one per range); differentiable in s and o
    through the library's adjoint (a torch.autograd.Function)."""
    global _DecodeFn
    import torch

    if _DecodeFn is None:
        _DecodeFn = _decode_fn()
    if init is None:
        init = float(1 << (p.bit_depth - 1))
    if workspace is None:
        workspace = torch.empty(refine_workspace_size(w, h, p, iters), dtype=torch.uint8, device=s.device)
    return _DecodeFn.apply(s.contiguous(), o.contiguous(), maps, w, h, p, iters, float(init), workspace)


def refine(img, maps, s, o, p: fic_params, steps: int = 200, iters: int = 8, lr: float = 1e-3, loss=None,
           workspace=None, stream=None):
    """The library's whole refinement loop (Adam on s and o/P, CUDA graph per
    step); s, o updated in place; returns the loss tensor (steps + 1 values)."""
    import torch

    h, w = int(img.shape[0]), int(img.shape[1])
    if loss is None:
        loss = torch.empty(steps + 1, dtype=torch.float32, device=s.device)
    if workspace is None:
        workspace = torch.empty(refine_workspace_size(w, h, p, iters), dtype=torch.uint8, device=s.device)
    _check(lib().fic_refine(img.data_ptr(), w, h, int(img.stride(0)), ctypes.byref(p), maps.data_ptr(),
                            s.data_ptr(), o.data_ptr(), steps, iters, ctypes.c_float(lr), loss.data_ptr(),
                            workspace.data_ptr(), workspace.numel(), _stream_ptr(stream)), "fic_refine")
    return loss


def decode_scaled(maps, w: int, h: int, p: fic_params, scale_log2: int, init: float | None = None, out=None,
                  stream=None):
    """Decode maps of a w x h encode at 2^scale_log2 times the size (returns
    an (h*z) x (w*z) float32 array / tensor, z = 2^scale_log2)."""
    R, _ = counts(w, h, p)
    z = 2.0 ** scale_log2
    ow, oh = int(round(w * z)), int(round(h * z))
    if init is None:
        init = float(1 << (p.bit_depth - 1))
    if _is_torch(maps):
        import torch

        if out is None:
            out = torch.empty((oh, ow), dtype=torch.float32, device=maps.device)
        maps_ptr, out_ptr, st = maps.data_ptr(), out.data_ptr(), _stream_ptr(stream)
    else:
        maps = np.ascontiguousarray(maps, MAP_DTYPE)
        if out is None:
            out = np.zeros((oh, ow), np.float32)
        maps_ptr, out_ptr = maps.ctypes.data, out.ctypes.data
        st = 0 if stream is None else _stream_ptr(stream)
    _check(lib().fic_decode_scaled(maps_ptr, R, w, h, ctypes.byref(p), int(scale_log2), ctypes.c_float(init), out_ptr,
                                   None, 0, st), "fic_decode_scaled")
    return out


def cross_terms(img, p: fic_params, out=None, stream=None):
    """Raw cross terms Xt[r, c] = (m*X - Sq*Sb)/m of the selected search path
    (testing aid).  img: torch CUDA tensor; returns a (R, 8D) float32 tensor."""
    import torch

    h, w = int(img.shape[0]), int(img.shape[1])
    R, D = counts(w, h, p)
    if out is None:
        out = torch.empty((R, 8 * D), dtype=torch.float32, device=img.device)
    _check(lib().fic_cross_terms(img.data_ptr(), w, h, int(img.stride(0)), ctypes.byref(p), out.data_ptr(), None,
                                 0, _stream_ptr(stream)), "fic_cross_terms")
    return out


def maps_to_numpy(maps) -> np.ndarray:
    """View a device maps tensor (uint8, R*40 bytes) as a host MAP_DTYPE array."""
    if _is_torch(maps):
        return maps.detach().cpu().numpy().view(MAP_DTYPE)
    return np.asarray(maps, MAP_DTYPE)


def set_wait_limit_ns(ns: int) -> None:
    """Wall-clock limit of each bounded device wait of the tensor-core search
    (0 restores the default of 2 s); applies to later launches."""
    _check(lib().fic_set_wait_limit_ns(int(ns)), "fic_set_wait_limit_ns")


def get_wait_limit_ns() -> int:
    return int(lib().fic_get_wait_limit_ns())


def last_encode_stats():
    out = (ctypes.c_int64 * 4)()
    lib().fic_last_encode_stats(out)
    return list(out)


def last_encode_phase_ms():
    """[prep, search, rescore, fallback, output] ms of the last encode run with
    FIC_FLAG_PHASE_TIMING (waits for its events)."""
    out = (ctypes.c_double * 5)()
    _check(lib().fic_last_encode_phase_ms(out), "fic_last_encode_phase_ms")
    return list(out)


def header_symbols() -> list[str]:
    """Function names declared in include/fic.h (for the ABI-export test)."""
    import re

    hdr = os.path.join(os.path.dirname(_HERE), "include", "fic.h")
    with open(hdr) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fic_\w+)\s*\(", text, re.M)))
