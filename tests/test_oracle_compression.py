"""Lossless compression of the synthetic workloads against PNG-style deflate
(the paper's Fig. 4 compares lossless file sizes with PNG and JPEG 2000 on
real radiology and pathology images, which are not available here).

PNG-style deflate: every row filtered with the PNG filter (none, sub, up,
average, Paeth) whose output has the smallest sum of absolute values, one
filter byte per row, then zlib at level 9; 16-bit samples big endian.  The
codec's sizes are those of the oracle's streams, tile headers included.
The bounds are loose: they catch a codec that stops compressing (a lost
zero-run or plane-removal step inflates every stream), not small changes.
"""
import zlib

import numpy as np
import pytest


def _rows(img: np.ndarray) -> np.ndarray:
    a = img.astype(">u2").view(np.uint8) if img.dtype == np.uint16 else img
    return a.reshape(a.shape[0], -1).astype(np.int32)


def _paeth(left, up, upleft):
    p = left + up - upleft
    pa, pb, pc = np.abs(p - left), np.abs(p - up), np.abs(p - upleft)
    return np.where((pa <= pb) & (pa <= pc), left, np.where(pb <= pc, up, upleft))


def png_deflate(img: np.ndarray, bpp: int) -> bytes:
    a = _rows(img)
    out = bytearray()
    prev = np.zeros(a.shape[1], np.int32)
    for row in a:
        left = np.concatenate([np.zeros(bpp, np.int32), row[:-bpp]])
        upleft = np.concatenate([np.zeros(bpp, np.int32), prev[:-bpp]])
        cands = [(c & 0xFF).astype(np.uint8) for c in (row, row - left, row - prev, row - (left + prev) // 2,
                                                        row - _paeth(left, prev, upleft))]
        best = min(range(5), key=lambda i: int(np.abs(cands[i].view(np.int8).astype(np.int32)).sum()))
        out.append(best)
        out += cands[best].tobytes()
        prev = row
    return zlib.compress(bytes(out), 9)


def png_inflate(data: bytes, rows: int, rowlen: int, bpp: int) -> np.ndarray:
    raw = np.frombuffer(zlib.decompress(data), np.uint8).reshape(rows, rowlen + 1)
    out = np.zeros((rows, rowlen), np.int32)
    prev = np.zeros(rowlen, np.int32)
    for y in range(rows):
        f, d = int(raw[y, 0]), raw[y, 1:].astype(np.int32)
        row = np.zeros(rowlen, np.int32)
        for x in range(rowlen):   # left neighbours are reconstructed first
            left = row[x - bpp] if x >= bpp else 0
            ul = prev[x - bpp] if x >= bpp else 0
            pred = [0, left, prev[x], (left + prev[x]) // 2, int(_paeth(np.int32(left), prev[x], np.int32(ul)))][f]
            row[x] = (d[x] + pred) & 0xFF
        out[y], prev = row, row
    return out


def png_deflate_size(img: np.ndarray, bpp: int) -> int:
    return len(png_deflate(img, bpp))


def test_png_reference_is_lossless():
    """The PNG-style sizes are those of real, invertible encodings: inflate and unfilter small images."""
    rng = np.random.default_rng(1)
    for img, bpp in [(rng.integers(0, 256, (9, 7, 3)).astype(np.uint8), 3),
                     (rng.integers(0, 4096, (6, 11)).astype(np.uint16), 2),
                     ((np.indices((12, 10)).sum(0) * 9 % 256).astype(np.uint8), 1)]:
        a = _rows(img)
        back = png_inflate(png_deflate(img, bpp), a.shape[0], a.shape[1], bpp)
        assert np.array_equal(back, a)


@pytest.mark.parametrize("name", ["phantom", "slide", "stain"])
def test_lossless_size_against_png_deflate(orc, synth, name):
    if name == "phantom":
        img, levels, bits, bpp = synth.phantom(synth.config_seed(2), 2048, 2048), 5, 12, 2
        ours = len(orc.encode_tile(img, levels, bits, [0] * (levels + 1)))
        bound = 0.85          # smooth 12-bit content: the wavelet codec is well ahead (0.74 measured)
    elif name == "slide":
        img, bpp = synth.slide(synth.config_seed(3), 8000, 12000, 1024, 512), 3
        ours = sum(len(orc.encode_tile(np.ascontiguousarray(img[y:y + 256, x:x + 256]), 8, 8, [0] * 9))
                   for y in range(0, 512, 256) for x in range(0, 1024, 256))
        bound = 1.05          # 256 x 256 tiles, each with its own headers and codes (about 1.00 measured)
    else:
        img, bpp = synth.stain(synth.config_seed(1)), 3
        ours = len(orc.encode_tile(img, 3, 8, [0] * 4))
        bound = 1.08          # N(0, 8^2) noise on smooth fields (1.03 measured)
    png = png_deflate_size(img, bpp)
    assert ours < img.nbytes
    assert ours / png < bound, (name, ours, png, ours / png)
