"""Helpers of the GPU parity tests: run the CUDA library through the C ABI
and compare its streams with the oracle's, block by block, with a message
that says where and how they differ."""
from __future__ import annotations

import struct

import numpy as np


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "CUDA device required"
    return torch


def to_device(img: np.ndarray):
    torch = torch_cuda()
    a = np.ascontiguousarray(img)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a).cuda()


def gpu_encode(codec, imgs, levels, bits, qsteps=None, origins=None, capacity=None, transforms=None):
    """Encode a list of images as one batch of tiles; returns (list of tile stream bytes, raw stream, offsets)."""
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    tiles, keep = [], []
    if origins is None:
        # independent images: spread them along x so that no two overlap at any level
        maxw = max(a.shape[1] for a in imgs)
        maxl = max(levels) if isinstance(levels, (list, tuple)) else levels
        S = 1
        while S < max(maxw, 2 ** maxl):
            S *= 2
        origins = [(i * S, 0) for i in range(len(imgs))]
    for i, img in enumerate(imgs):
        dt = to_device(img)
        keep.append(dt)
        L = levels[i] if isinstance(levels, (list, tuple)) else levels
        B = bits[i] if isinstance(bits, (list, tuple)) else bits
        q = qsteps[i] if qsteps and isinstance(qsteps[0], (list, tuple)) else tuple(qsteps or ())
        x0, y0 = origins[i]
        ct = transforms[i] if isinstance(transforms, (list, tuple)) else (transforms or 0)
        tiles.append(isx.tile_from_tensor(dt, L, B, q, x0, y0, transform=ct))
    if capacity is None:
        capacity = sum(a.nbytes for a in imgs) * 3 + 4096 * len(imgs)
    out = torch.zeros(capacity, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(len(imgs) + 1, dtype=torch.int64, device="cuda")
    codec.encode_tiles(tiles, out, offs)
    rc = codec.sync_status()
    assert rc == 0, f"device status {rc}"
    o = offs.cpu().numpy()
    raw = out[: int(o[-1])].cpu().numpy().tobytes()
    streams = [raw[o[i]:o[i + 1]] for i in range(len(imgs))]
    return streams, tiles, out, offs


def split_blocks(stream: bytes):
    nb = struct.unpack_from("<I", stream, 12)[0]
    ends = struct.unpack_from(f"<{nb}I", stream, 32)
    data = stream[32 + 4 * nb:]
    out, prev = [], 0
    for e in ends:
        out.append(data[prev:e])
        prev = e
    return stream[:32], out


def explain_mismatch(gpu: bytes, ref: bytes) -> str:
    if gpu == ref:
        return "identical"
    if len(gpu) < 32 or gpu[:32] != ref[:32]:
        return f"tile headers differ: gpu {gpu[:32].hex()} ref {ref[:32].hex()}"
    hg, bg = split_blocks(gpu)
    hr, br = split_blocks(ref)
    for i, (a, b) in enumerate(zip(bg, br)):
        if a != b:
            k = next((j for j in range(min(len(a), len(b))) if a[j] != b[j]), min(len(a), len(b)))
            return (f"block {i}: gpu {len(a)} B, ref {len(b)} B, first differing byte {k}: "
                    f"gpu {a[max(0, k - 4):k + 8].hex()} ref {b[max(0, k - 4):k + 8].hex()}; "
                    f"ref header {b[:12].hex()} gpu header {a[:12].hex()}")
    return f"block tables differ ({len(bg)} vs {len(br)} blocks), sizes {len(gpu)} vs {len(ref)}"


def gpu_decode_tile(codec, out_buf, offs, tiles, index, level=0, drop=0):
    """Decode tile `index` alone at `level` via a region decode of its own rectangle."""
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    t = tiles[index]
    zw, zh = isx.level_dim(t.width, level), isx.level_dim(t.height, level)
    rx, ry = t.x0 >> level, t.y0 >> level
    dt = torch.uint8 if t.bits <= 8 else torch.int16
    shape = (zh, zw, t.channels) if t.channels > 1 else (zh, zw)
    out = torch.zeros(shape, dtype=dt, device="cuda")
    codec.decode_region(out_buf, offs, tiles, level, (rx, ry, zw, zh), out, drop)
    rc = codec.sync_status()
    assert rc == 0, f"device status {rc}"
    a = out.cpu().numpy()
    return a.view(np.uint16) if t.bits > 8 else a
