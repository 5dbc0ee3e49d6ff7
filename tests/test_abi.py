"""The C ABI library loads and exports every entry point include/fic.h
declares; host-side validation works without a GPU (no compute calls)."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def fic():
    from paper_1404_0774_gb300 import build

    build.build()
    from paper_1404_0774_gb300 import fic

    return fic


def test_exports_every_declared_symbol(fic):
    names = fic.header_symbols()
    assert "fic_encode" in names and "fic_decode" in names
    lib = fic.lib()
    for name in names:
        assert hasattr(lib, name), name


def test_binding_declares_argument_types_for_every_entry_point(fic):
    """ctypes passes undeclared integer arguments as 32-bit ints, which would
    truncate 64-bit device pointers: every entry point must declare its types."""
    import re

    lib = fic.lib()
    hdr = open(fic.os.path.join(fic.os.path.dirname(fic._HERE), "include", "fic.h")).read()
    for name in fic.header_symbols():
        decl = re.search(r"^\s*(?:const\s+)?\w+\s*\*?\s*" + name + r"\s*\(([^)]*)\)", hdr, re.M).group(1).strip()
        n_args = 0 if decl in ("", "void") else decl.count(",") + 1
        fn = getattr(lib, name)
        assert fn.argtypes is not None and len(fn.argtypes) == n_args, name


def test_counts_and_validation(fic):
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12)
    assert fic.counts(512, 512, p) == (4096, 15625)
    p1 = fic.params(range_size=8, domain_stride=8, bit_depth=8)
    assert fic.counts(256, 256, p1) == (1024, 961)
    for bad in [(250, 256, p1), (8, 256, p1), (256, 0, p1)]:
        with pytest.raises(fic.FicError) as ei:
            fic.counts(*bad)
        assert ei.value.code == -2
    with pytest.raises(fic.FicError) as ei:
        fic.counts(256, 256, fic.params(bit_depth=13))
    assert ei.value.code == -3
    with pytest.raises(fic.FicError) as ei:
        fic.counts(256, 256, fic.params(range_size=6))
    assert ei.value.code == -1


def test_status_strings(fic):
    lib = fic.lib()
    for code in range(-7, 1):
        assert lib.fic_status_str(code)


def test_encode_rejects_bad_arguments_before_any_gpu_work(fic):
    lib = fic.lib()
    p = fic.params()
    n = ctypes.c_int()
    # null image / maps
    assert lib.fic_encode(None, 64, 64, 64, ctypes.byref(p), None, 64, ctypes.byref(n), None, 0, None) == -1
    buf = (ctypes.c_uint8 * 4096)()
    maps = (ctypes.c_uint8 * (40 * 64))()
    # maps capacity below the range count
    assert lib.fic_encode(buf, 64, 64, 64, ctypes.byref(p), maps, 10, ctypes.byref(n), None, 0, None) == -4
    # pitch smaller than width
    assert lib.fic_encode(buf, 64, 64, 32, ctypes.byref(p), maps, 64, ctypes.byref(n), None, 0, None) == -1


def test_batch_workspace_size_and_limits(fic):
    """The batch plan is host arithmetic: sizes grow with the slices, more
    than 1024 slices is a capacity error, phase timing is rejected."""
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12)

    def table(sizes):
        return (fic.fic_slice * len(sizes))(*[fic.fic_slice(None, s, s, s, None) for s in sizes])

    size = ctypes.c_size_t()
    lib = fic.lib()
    assert lib.fic_batch_workspace_size(table([64]), 1, ctypes.byref(p), ctypes.byref(size)) == 0
    one = size.value
    assert lib.fic_batch_workspace_size(table([64, 128]), 2, ctypes.byref(p), ctypes.byref(size)) == 0
    assert size.value > one
    assert lib.fic_batch_workspace_size(table([64] * 1025), 1025, ctypes.byref(p), ctypes.byref(size)) == -4
    pt = fic.params(range_size=8, domain_stride=4, bit_depth=12, flags=fic.FIC_FLAG_PHASE_TIMING)
    assert lib.fic_batch_workspace_size(table([64]), 1, ctypes.byref(pt), ctypes.byref(size)) == -1


def test_wait_limit_setter_is_host_state(fic):
    """The search's wait limit is host state read at each launch: setting,
    reading back and restoring the default need no GPU."""
    assert fic.get_wait_limit_ns() == 2_000_000_000
    fic.set_wait_limit_ns(12345)
    assert fic.get_wait_limit_ns() == 12345
    fic.set_wait_limit_ns(0)
    assert fic.get_wait_limit_ns() == 2_000_000_000


def test_missing_library_raises_instead_of_falling_back(fic, monkeypatch, tmp_path):
    """Without libfic.so every entry point raises: there is no CPU path."""
    import numpy as np

    monkeypatch.setattr(fic, "_LIB_PATH", str(tmp_path / "libfic.so"))
    monkeypatch.setattr(fic, "_lib", None)
    img = np.zeros((64, 64), np.uint16)
    p = fic.params(range_size=8, domain_stride=8, bit_depth=12)
    with pytest.raises(ImportError):
        fic.encode(img, p)
    with pytest.raises(ImportError):
        fic.decode(np.zeros(64, fic.MAP_DTYPE), 64, 64, p)
    with pytest.raises(ImportError):
        fic.lib()


def test_product_sources_never_reach_the_oracle():
    """The library, its binding and its build name nothing of the oracle
    package (no import, include, link or call): the CUDA path and the oracle
    share no code."""
    import os
    import re

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pat = re.compile(r"\boracle\b|\borc_\w+|fic_oracle", re.I)
    seen = 0
    for top in ("paper_1404_0774_gb300", "include"):
        for dirpath, dirnames, files in os.walk(os.path.join(root, top)):
            dirnames[:] = [d for d in dirnames if d not in ("_lib", "_build", "__pycache__")]
            for f in files:
                if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp", ".c")):
                    seen += 1
                    with open(os.path.join(dirpath, f)) as fh:
                        hits = [ln for ln in fh if pat.search(ln)]
                    assert not hits, (f, hits[:3])
    assert seen >= 5
