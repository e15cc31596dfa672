"""The no-allocation entry point isx_encode_tile_static, through the C ABI.

Collected last (file name) so that it runs both after the other GPU tests
and, when started on its own, in a fresh process whose first call does the
per-device set-up.  Its streams must equal those of the context entry point
isx_encode_tiles for the same tile, on calls made one after another on the
one shared scratch array."""
import numpy as np
import pytest

from gpu_helpers import gpu_encode, to_device, torch_cuda

pytestmark = pytest.mark.gpu


def _tile(img, levels, bits, q=()):
    from paper_2005_08713_gb300 import isx
    return isx.tile_from_tensor(to_device(img), levels, bits, q)


def _static(tile, capacity):
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    out = torch.full((capacity,), 0xA5, dtype=torch.uint8, device="cuda")
    n = isx.encode_tile_static(tile, out)
    return out[:n].cpu().numpy().tobytes(), out


def _cases(synth):
    rng = np.random.default_rng(7)
    return [
        # fused shared-memory transform, lossy RGB
        (synth.slide(synth.config_seed(3), 4096, 2048, 256, 256), 5, 8, (3, 2, 1, 0, 0, 0)),
        # global transform path (16-bit samples), lossless, odd size
        ((rng.integers(0, 1 << 16, size=(509, 347))).astype(np.uint16), 3, 16, ()),
    ]


def test_static_encode_matches_context_entry_on_calls_in_a_row(synth):
    from paper_2005_08713_gb300 import isx
    torch = torch_cuda()
    cases = _cases(synth)
    with isx.Codec() as codec:
        refs = [gpu_encode(codec, [img], L, bits, [q])[0][0] for img, L, bits, q in cases]
    tiles = [_tile(img, L, bits, q) for img, L, bits, q in cases]
    got = []
    for t, img in zip(tiles, cases):
        got.append(_static(t, img[0].nbytes * 3 + 4096)[0])
    for i, (g, r) in enumerate(zip(got, refs)):
        assert g == r, f"case {i}: static stream ({len(g)} bytes) differs from isx_encode_tiles ({len(r)} bytes)"
    # the first tile again, after the second one has used the scratch
    again = _static(tiles[0], cases[0][0].nbytes * 3 + 4096)[0]
    assert again == refs[0]
    torch.cuda.synchronize()


def test_static_encode_allocates_nothing(synth):
    torch = torch_cuda()
    cases = _cases(synth)
    tiles = [_tile(img, L, bits, q) for img, L, bits, q in cases]
    outs = [torch.zeros(img.nbytes * 3 + 4096, dtype=torch.uint8, device="cuda") for img, *_ in cases]
    from paper_2005_08713_gb300 import isx
    for t, o in zip(tiles, outs):           # set-up and first launch of every kernel
        isx.encode_tile_static(t, o)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for t, o in zip(tiles, outs):
            isx.encode_tile_static(t, o)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"


def test_static_encode_matches_oracle_at_the_largest_documented_tile(orc, synth):
    img = synth.slide(synth.config_seed(3), 8192, 4096, 512, 512)
    ref = orc.encode_tile(img, 15, 8)
    got, _ = _static(_tile(img, 15, 8), img.nbytes * 3 + 4096)
    assert got == ref
    rng = np.random.default_rng(11)
    g16 = rng.integers(0, 1 << 16, size=(512, 512)).astype(np.uint16)
    ref16 = orc.encode_tile(g16, 2, 16)
    got16, _ = _static(_tile(g16, 2, 16), g16.nbytes * 4 + 4096)
    assert got16 == ref16


def test_static_encode_capacity_and_size_errors(synth):
    from paper_2005_08713_gb300 import isx
    torch = torch_cuda()
    img, L, bits, q = _cases(synth)[0]
    t = _tile(img, L, bits, q)
    ref, _ = _static(t, img.nbytes * 3 + 4096)
    small = torch.full((64,), 0x5A, dtype=torch.uint8, device="cuda")
    with pytest.raises(isx.IsxError) as ei:
        isx.encode_tile_static(t, small)
    assert ei.value.status == isx.ISX_ERR_CAPACITY
    assert ei.value.needed == (len(ref) + 3) // 4 * 4
    assert bool((small == 0x5A).all()), "a rejected stream must leave d_out untouched"
    # a tile beyond the static scratch is refused before anything runs
    big = np.zeros((1024, 1024, 3), np.uint8)
    out = torch.full((16,), 0x5A, dtype=torch.uint8, device="cuda")
    with pytest.raises(isx.IsxError) as ei:
        isx.encode_tile_static(_tile(big, 4, 8), out)
    assert ei.value.status == isx.ISX_ERR_OOM
    assert "static scratch holds %d" % isx.STATIC_SCRATCH_BYTES in str(ei.value)
    assert bool((out == 0x5A).all())
    # the scratch is usable again right after both errors
    assert _static(t, img.nbytes * 3 + 4096)[0] == ref


def test_static_encode_reports_samples_above_bit_depth(synth):
    from paper_2005_08713_gb300 import isx
    torch = torch_cuda()
    img = synth.slide(synth.config_seed(3), 4096, 2048, 128, 128)
    out = torch.zeros(img.nbytes * 3 + 4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(isx.IsxError) as ei:
        isx.encode_tile_static(_tile(img, 4, 5), out)   # 8-bit samples declared as 5-bit
    assert ei.value.status == isx.ISX_ERR_ARG
    assert "bit depth" in str(ei.value)
    # the status word starts at zero again on the next call
    ok = (img >> 3).astype(np.uint8)
    n = isx.encode_tile_static(_tile(ok, 4, 5), out)
    assert n > 0
