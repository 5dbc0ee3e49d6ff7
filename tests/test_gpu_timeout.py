"""Failure detection without a fault: the tensor-core search's bounded waits.

Every mbarrier wait of the search gives up after a wall-clock limit, records
the error, drains the copies and MMAs already issued, frees its TMEM and
exits.  Here the limit is set so short (1 ns) that waits run out on a small
image: the synchronous call must return FIC_ERR_TIMEOUT with every map
flagged FIC_MAP_ERROR, and the GPU must stay usable -- an encode right after,
with the default limit, gives oracle-correct maps (which also shows that the
aborted CTAs released their TMEM: a leaked allocation would stall the next
search's CTAs).  Nothing faults, traps or hangs: the wait that runs out is an
ordinary bounded wait returning an error status.
"""
import numpy as np
import pytest

import fic_synth
from parity import check_against_oracle, encode_pinned

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIC_MAP_ERROR = 0x2


@pytest.fixture(scope="module")
def fic():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1404_0774_gb300 import fic

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fic


@pytest.mark.parametrize("n,t", [(8, 4), (4, 2)])
def test_expired_waits_return_timeout_and_leave_the_gpu_usable(fic, orc, n, t):
    img = fic_synth.ct_slice(91, 64)
    p = fic.params(range_size=n, domain_stride=t, bit_depth=12, search=fic.FIC_SEARCH_TC)
    R, _ = fic.counts(64, 64, p)
    fired = 0
    try:
        fic.set_wait_limit_ns(1)
        for _ in range(3):
            maps = np.zeros(R, fic.MAP_DTYPE)
            try:
                fic.encode(img, p, maps=maps)  # host image and maps: synchronous, reads the error flag
            except fic.FicError as e:
                assert e.code == -6
                assert np.all(maps["info"] & FIC_MAP_ERROR)
                fired += 1
    finally:
        fic.set_wait_limit_ns(0)
    # a wait for the first accumulator spans a TMA copy and the MMAs: far
    # longer than 1 ns, so the limit runs out
    assert fired >= 1
    # page-locked host maps are written by the map output kernel directly; the
    # call takes the error from the maps' flags
    fired_pinned = 0
    try:
        fic.set_wait_limit_ns(1)
        for _ in range(3):
            rc, pm = encode_pinned(fic, img, p)
            if rc != 0:
                assert rc == -6
                assert np.all(pm["info"] & FIC_MAP_ERROR)
                fired_pinned += 1
    finally:
        fic.set_wait_limit_ns(0)
    assert fired_pinned >= 1
    assert fic.get_wait_limit_ns() == 2_000_000_000
    # the context is intact and the search runs normally again
    got = fic.encode(img, p)
    assert not np.any(got["info"] & FIC_MAP_ERROR)
    check_against_oracle(orc, img, got, n, t, 12)
    dev = fic.maps_to_numpy(fic.encode(torch.from_numpy(img.astype(np.int16)).cuda(), p))
    torch.cuda.synchronize()
    assert np.array_equal(dev, got)
