"""The batched encode (fic_encode_batch through the C ABI): every slice of a
mixed-size batch must get exactly the maps fic_encode gives that slice alone,
on the first call (run eagerly) and on graph replays; and the batch's own maps
of one slice per size of the volume workload are checked against the FP64
oracle directly (every map re-scored, every range's residual against the
oracle's per-range minimum)."""
import numpy as np
import pytest

import fic_synth
from parity import check_against_oracle

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


@pytest.mark.parametrize("search", ["auto", "simt"])
def test_batch_equals_single_slice_encodes(fic, search):
    sizes = [64, 128, 96, 64, 128, 160]
    imgs_np = [fic_synth.ct_slice(60 + i, s) for i, s in enumerate(sizes)]
    code = {"auto": fic.FIC_SEARCH_AUTO, "simt": fic.FIC_SEARCH_SIMT}[search]
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12, search=code)
    imgs = [torch.from_numpy(a.astype(np.int16)).cuda() for a in imgs_np]
    maps = [torch.zeros((s // 8) ** 2 * 40, dtype=torch.uint8, device="cuda") for s in sizes]
    tab = fic.slice_table(imgs, maps)
    ws = torch.empty(fic.batch_workspace_size(tab, p), dtype=torch.uint8, device="cuda")
    ref = [fic.maps_to_numpy(fic.encode(im, p)) for im in imgs]
    for call in range(3):
        for m in maps:
            m.zero_()
        fic.encode_batch(tab, p, ws)
        torch.cuda.synchronize()
        for i, m in enumerate(maps):
            assert np.array_equal(fic.maps_to_numpy(m), ref[i]), (call, i)
    t = fic.last_batch_slice_ms(len(sizes))
    assert all(x > 0 for x in t)


def test_batch_rejects_host_pointers_and_short_workspace(fic):
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12)
    im = torch.from_numpy(fic_synth.ct_slice(70, 64).astype(np.int16)).cuda()
    mp = torch.zeros(64 * 40, dtype=torch.uint8, device="cuda")
    tab = fic.slice_table([im], [mp])
    need = fic.batch_workspace_size(tab, p)
    with pytest.raises(fic.FicError):
        fic.encode_batch(tab, p, torch.empty(need // 2, dtype=torch.uint8, device="cuda"))
    host = fic.fic_slice(fic_synth.ct_slice(70, 64).astype(np.int16).ctypes.data, 64, 64, 64, mp.data_ptr())
    bad = (fic.fic_slice * 1)(host)
    with pytest.raises(fic.FicError):
        fic.encode_batch(bad, p, torch.empty(need, dtype=torch.uint8, device="cuda"))


def test_batch_of_stack_slices_equals_single_encodes(fic):
    """Slices of the CT-like stack at the three sizes of the volume workload
    (several per size, so the batch forms groups and two half pipelines):
    every map equals the single-slice encode of that slice."""
    seed = fic_synth.CT_SEED + 11
    pick = [0, 1, 2, 32, 33, 34, 64, 65, 66, 95]  # slices of fic_synth.ct_stack(seed)
    size = {0: 256, 1: 384, 2: 512}
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12)
    imgs = [torch.from_numpy(fic_synth.ct_slice(seed + 1000 + k, size[k // 32]).astype(np.int16)).cuda() for k in pick]
    maps = [torch.zeros((im.shape[0] // 8) ** 2 * 40, dtype=torch.uint8, device="cuda") for im in imgs]
    tab = fic.slice_table(imgs, maps)
    ws = torch.empty(fic.batch_workspace_size(tab, p), dtype=torch.uint8, device="cuda")
    ref = [fic.maps_to_numpy(fic.encode(im, p)) for im in imgs]
    for call in range(2):  # eager run, then a graph replay
        for m in maps:
            m.zero_()
        fic.encode_batch(tab, p, ws)
        torch.cuda.synchronize()
        for i, m in enumerate(maps):
            got = fic.maps_to_numpy(m)
            assert np.array_equal(got, ref[i]), (call, pick[i])


def test_batch_of_one_slice(fic):
    im = torch.from_numpy(fic_synth.ct_slice(71, 128).astype(np.int16)).cuda()
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12)
    mp = torch.zeros(256 * 40, dtype=torch.uint8, device="cuda")
    tab = fic.slice_table([im], [mp])
    ws = torch.empty(fic.batch_workspace_size(tab, p), dtype=torch.uint8, device="cuda")
    fic.encode_batch(tab, p, ws)
    torch.cuda.synchronize()
    assert np.array_equal(fic.maps_to_numpy(mp), fic.maps_to_numpy(fic.encode(im, p)))


@pytest.mark.parametrize("search", ["auto", "simt"])
def test_batch_maps_match_the_oracle(fic, orc, search):
    """One CT-like slice of each size of the volume workload (256, 384 and 512
    pixels square, 8x8 ranges, 16x16 domains at stride 4, 12-bit) in one
    batch, plus repeats so that the batch forms size groups: the batch's maps
    of the first slice of each size pass the oracle parity bar on every range
    (Section V search, eq 8-12), on the eager call and on a graph replay."""
    seed = fic_synth.CT_SEED + 23
    sizes = [256, 384, 512, 256, 384]
    imgs_np = [fic_synth.ct_slice(seed + 1000 + i, s) for i, s in enumerate(sizes)]
    code = {"auto": fic.FIC_SEARCH_AUTO, "simt": fic.FIC_SEARCH_SIMT}[search]
    p = fic.params(range_size=8, domain_stride=4, bit_depth=12, search=code)
    imgs = [torch.from_numpy(a.astype(np.int16)).cuda() for a in imgs_np]
    maps = [torch.zeros((s // 8) ** 2 * 40, dtype=torch.uint8, device="cuda") for s in sizes]
    tab = fic.slice_table(imgs, maps)
    ws = torch.empty(fic.batch_workspace_size(tab, p), dtype=torch.uint8, device="cuda")
    refs = {}
    for call in range(2):  # eager run, then a graph replay
        for m in maps:
            m.zero_()
        fic.encode_batch(tab, p, ws)
        torch.cuda.synchronize()
        for i in range(3):
            got = fic.maps_to_numpy(maps[i])
            if i not in refs:
                refs[i] = orc.encode(imgs_np[i], n=8, t=4, bit_depth=12)
            check_against_oracle(orc, imgs_np[i], got, 8, 4, 12, ref=refs[i])
