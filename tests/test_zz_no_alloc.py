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


STATIC_SCRATCH_BYTES = 32 << 20  # FIC_STATIC_SCRATCH_BYTES in include/fic.h


def test_header_states_the_scratch_size():
    import os
    import re

    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fic.h")
    with open(hdr) as fh:
        m = re.search(r"#define FIC_STATIC_SCRATCH_BYTES \((\d+)u << (\d+)\)", fh.read())
    assert m and int(m.group(1)) << int(m.group(2)) == STATIC_SCRATCH_BYTES


@pytest.mark.parametrize("name,make,n,t,B", CASES, ids=[c[0] for c in CASES])
def test_static_scratch_encode_matches_fic_encode(fic, name, make, n, t, B):
    img_np = make()
    h, w = img_np.shape
    p = fic.params(range_size=n, domain_stride=t, bit_depth=B)
    # the parity cases must fit the fixed scratch (else they would test the refusal)
    assert fic.encode_workspace_size(w, h, p) <= STATIC_SCRATCH_BYTES
    R, _ = fic.counts(w, h, p)
    img = torch.from_numpy(img_np.astype(np.int16) if B > 8 else img_np).cuda()
    ref = fic.maps_to_numpy(fic.encode(img, p))
    torch.cuda.synchronize()
    m, P = n * n, (1 << B) - 1
    lib = fic.lib()
    stream = torch.cuda.current_stream().cuda_stream
    outs = [torch.full((R * 40,), 0xAB, dtype=torch.uint8, device="cuda") for _ in range(3)]
    nm = ctypes.c_int()
    # a first call may load the static array onto the device; the calls after
    # it must take no device memory at all
    assert lib.fic_encode_static(img.data_ptr(), w, h, w, ctypes.byref(p), outs[0].data_ptr(), R, ctypes.byref(nm),
                                 stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for call in (1, 2):
        maps = outs[call]
        rc = lib.fic_encode_static(img.data_ptr(), w, h, w, ctypes.byref(p), maps.data_ptr(), R,
                                   ctypes.byref(nm), stream)
        assert rc == 0, (call, rc)
        torch.cuda.synchronize()
        # (free memory may only grow: a pool trimmed at the synchronisation)
        assert torch.cuda.mem_get_info()[0] >= free0, "the call took device memory"
        assert torch.cuda.memory_reserved() == reserved0
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
    assert fic.encode_workspace_size(512, 512, p) > STATIC_SCRATCH_BYTES
    img = torch.zeros((512, 512), dtype=torch.int16, device="cuda")
    maps = torch.empty(4096 * 40, dtype=torch.uint8, device="cuda")
    nm = ctypes.c_int()
    rc = fic.lib().fic_encode_static(img.data_ptr(), 512, 512, 512, ctypes.byref(p), maps.data_ptr(), 4096,
                                     ctypes.byref(nm), torch.cuda.current_stream().cuda_stream)
    assert rc == -4
