"""Host-side behaviour of the library that needs no GPU: argument checks and
the working-memory sizing of the no-allocation encoder return before any
CUDA call, and without a usable device every entry fails loudly (an error
status, never a CPU fallback).  The product package never loads the
oracle, and the oracle shares no source with the CUDA library.

Tests that reach the library's CUDA calls are skipped where a GPU is
present: they pass descriptors whose pixel address is not a buffer."""
import ast
import ctypes
import os
import re

import pytest

from paper_2005_08713_gb300 import isx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FAKE_PIXELS = 0x1000   # never dereferenced: every call below returns on the host or at its first CUDA call


def _no_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: these descriptors must not reach a launch")


def _desc(**kw):
    t = isx.TileDescC()
    t.width, t.height, t.channels, t.bits, t.levels = 64, 48, 3, 8, 3
    t.pixels, t.row_pitch_bytes = FAKE_PIXELS, 64 * 3
    for k, v in kw.items():
        if k == "qstep_log2":
            for i, q in enumerate(v):
                t.qstep_log2[i] = q
        else:
            setattr(t, k, v)
    return t


def _static(t, d_out=None, cap=0):
    lib = isx.load()
    size = ctypes.c_size_t(0)
    err = ctypes.create_string_buffer(512)
    rc = lib.isx_encode_tile_static(ctypes.byref(t), d_out, cap, ctypes.byref(size), None, err, 512)
    return rc, err.value.decode(), size.value


@pytest.mark.parametrize("field,value,msg", [
    ("width", 0, "width/height"), ("width", 65536, "width/height"), ("height", -3, "width/height"),
    ("channels", 0, "channels"), ("channels", 17, "channels"), ("bits", 0, "bits"), ("bits", 17, "bits"),
    ("transform", 4, "transform"), ("transform", -1, "transform"), ("reserved", 1, "reserved"),
    ("levels", -1, "levels"), ("levels", 16, "levels"), ("x0", -1, "origin"), ("y0", -256, "origin"),
    ("pixels", 0, "pixels"), ("row_pitch_bytes", 64 * 3 - 1, "row pitch"),
])
def test_static_encode_rejects_bad_descriptors(field, value, msg):
    rc, err, _ = _static(_desc(**{field: value}))
    assert rc == isx.ISX_ERR_ARG and msg in err, (rc, err)


@pytest.mark.parametrize("channels", [1, 2])
@pytest.mark.parametrize("transform", [2, 3])
def test_colour_transform_needs_three_channels(channels, transform):
    rc, err, _ = _static(_desc(channels=channels, transform=transform, row_pitch_bytes=64 * channels))
    assert rc == isx.ISX_ERR_ARG and "3 or more channels" in err, (rc, err)


def test_static_encode_rejects_bad_quantiser_steps_and_buffers():
    rc, err, _ = _static(_desc(qstep_log2=[0, 0, 16, 0]))
    assert rc == isx.ISX_ERR_ARG and "qstep_log2" in err
    rc, err, _ = _static(_desc(), d_out=None, cap=4096)
    assert rc == isx.ISX_ERR_ARG and "bad arguments" in err
    rc, err, _ = _static(_desc(), d_out=0x1002, cap=4096)
    assert rc == isx.ISX_ERR_ARG and "aligned" in err
    # 16-bit storage doubles the minimum row pitch
    rc, err, _ = _static(_desc(channels=1, bits=12, row_pitch_bytes=64 * 2 - 1))
    assert rc == isx.ISX_ERR_ARG and "row pitch" in err


def test_static_encode_reads_no_step_past_the_ll_band():
    _no_gpu()
    rc, err, _ = _static(_desc(levels=1, qstep_log2=[0, 0, 200]))
    assert rc == isx.ISX_ERR_CUDA, (rc, err)


@pytest.mark.parametrize("w,h", [(512, 512), (511, 509), (1, 512), (512, 1), (257, 300)])
def test_static_scratch_holds_every_tile_up_to_512(w, h):
    """The documented bound: a tile of at most 512 x 512 pixels and 4
    channels fits the 16 MiB static scratch at any bit depth, colour
    transform and level count, so the sizing passes and the call proceeds to
    the device (which this machine lacks: a CUDA error, not ISX_ERR_OOM)."""
    _no_gpu()
    for c in (1, 2, 3, 4):
        for bits in (1, 8, 11, 12, 13, 16):
            for levels in range(16):
                t = _desc(width=w, height=h, channels=c, bits=bits, levels=levels,
                          transform=3 if c >= 3 and levels % 2 else 0,
                          row_pitch_bytes=w * c * (1 if bits <= 8 else 2))
                rc, err, _ = _static(t)
                assert rc == isx.ISX_ERR_CUDA, (w, h, c, bits, levels, rc, err)


def test_static_scratch_rejects_a_tile_too_large_before_any_cuda_call():
    t = _desc(width=4096, height=4096, channels=3, bits=8, levels=6, row_pitch_bytes=4096 * 3)
    rc, err, _ = _static(t)
    assert rc == isx.ISX_ERR_OOM
    m = re.search(r"needs (\d+) bytes .* holds (\d+)", err)
    assert m and int(m.group(1)) > int(m.group(2)) == 16 << 20, err


def test_context_creation_fails_loudly_without_a_gpu():
    _no_gpu()
    with pytest.raises(isx.IsxError):
        isx.Codec(0)


def test_missing_library_is_an_error_not_a_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(isx, "_lib", None)
    monkeypatch.setattr(isx, "LIB_PATH", str(tmp_path / "libisx_gb300.so"))
    with pytest.raises(OSError):
        isx.load(build_if_missing=False)


def _python_imports(path):
    tree = ast.parse(open(path).read())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            yield from (a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            yield node.module or ""
            yield from (a.name for a in node.names)


def test_product_package_never_loads_the_oracle():
    pkg = os.path.join(ROOT, "paper_2005_08713_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "__pycache__" in dirpath or "_build" in dirpath:
            continue
        for f in files:
            p = os.path.join(dirpath, f)
            if f.endswith(".py"):
                names = list(_python_imports(p))
                assert not any(n == "oracle" or n.startswith("oracle.") for n in names), p
                assert "liborc" not in open(p).read(), p
            elif f.endswith((".cu", ".cuh", ".h", ".c", ".cpp")):
                src = open(p).read()
                assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', src), p


def test_oracle_shares_no_source_with_the_cuda_library():
    src = open(os.path.join(ROOT, "oracle", "isx_oracle.cpp")).read()
    includes = re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', src)
    assert all("/" not in i and not i.startswith("isx") for i in includes), includes
    py = list(_python_imports(os.path.join(ROOT, "oracle", "__init__.py")))
    assert not any("paper_2005_08713_gb300" in n for n in py), py
