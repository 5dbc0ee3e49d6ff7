"""fic_encode_static: the encode entry point that allocates no device memory.

Some callers may not allocate device memory (a plug-in inside an application
that owns the GPU's memory, a real-time pipeline that reserves everything up
front, a process under a memory cap it does not control).  fic_encode_static
serves them from a fixed scratch array inside the library.  These tests call
it through the C ABI, twice in a row (the scratch keeps the previous call's
contents), and compare its maps with fic_encode's, within the parity
tolerance the other tests use.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import fic_synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def fic():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1404_0774_gb300 import fic

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fic


CASES = [
    ("mr256_t8", lambda: fic_synth.mr_slice(), 8, 8, 8),
    ("ct256_t4", lambda: fic_synth.ct_slice(31, 256), 8, 4, 12),
]


@pytest.mark.parametrize("name,make,n,t,B", CASES, ids=[c[0] for c in CASES])
def test_static_scratch_encode_matches_fic_encode(fic, name, make, n, t, B):
    img_np = make()
    h, w = img_np.shape
    p = fic.params(range_size=n, domain_stride=t, bit_depth=B)
    R, _ = fic.counts(w, h, p)
    img = torch.from_numpy(img_np.astype(np.int16) if B > 8 else img_np).cuda()
    ref = fic.maps_to_numpy(fic.encode(img, p))
    torch.cuda.synchronize()
    m, P = n * n, (1 << B) - 1
    lib = fic.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        maps = torch.full((R * 40,), 0xAB, dtype=torch.uint8, device="cuda")
        nm = ctypes.c_int()
        rc = lib.fic_encode_static(img.data_ptr(), w, h, w, ctypes.byref(p), maps.data_ptr(), R,
                                   ctypes.byref(nm), stream)
        assert rc == 0, (call, rc)
        torch.cuda.synchronize()
        got = fic.maps_to_numpy(maps)
        assert nm.value == R
        assert np.array_equal(got["range_idx"], np.arange(R))
        bound = ref["err"] * (1 + REL) + 1e-9 * m * P * P
        assert np.all(got["err"] <= bound) and np.all(ref["err"] <= got["err"] * (1 + REL) + 1e-9 * m * P * P)
        same = (got["domain_idx"] == ref["domain_idx"]) & (got["iso"] == ref["iso"])
        assert np.array_equal(got["s_code"][same], ref["s_code"][same])
        assert np.array_equal(got["o_code"][same], ref["o_code"][same])


def test_static_scratch_rejects_images_beyond_its_size(fic):
    """512x512 at stride 4 needs more than the fixed scratch: refused with
    FIC_ERR_CAPACITY before any device work."""
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12)
    assert fic.encode_workspace_size(512, 512, p) > 16 << 20
    img = torch.zeros((512, 512), dtype=torch.int16, device="cuda")
    maps = torch.empty(4096 * 40, dtype=torch.uint8, device="cuda")
    nm = ctypes.c_int()
    rc = fic.lib().fic_encode_static(img.data_ptr(), 512, 512, 512, ctypes.byref(p), maps.data_ptr(), 4096,
                                     ctypes.byref(nm), torch.cuda.current_stream().cuda_stream)
    assert rc == -4
