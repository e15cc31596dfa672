"""The C-ABI library builds for sm_103a and exports every entry point that
include/isx.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    with open(os.path.join(ROOT, "include", "isx.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(isx_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    from paper_2005_08713_gb300 import isx
    assert declared_entry_points() == sorted(isx.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    from paper_2005_08713_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_tile_descriptor_layout_matches_header():
    from paper_2005_08713_gb300 import isx
    # int32 x 7, uint8[16], pointer, int64, int32 x 2  ->  72 bytes with natural alignment
    assert ctypes.sizeof(isx.TileDescC) == 72
    assert isx.TileDescC.pixels.offset == 48 and isx.TileDescC.row_pitch_bytes.offset == 56
    assert isx.TileDescC.transform.offset == 64 and isx.TileDescC.reserved.offset == 68
    with open(os.path.join(ROOT, "include", "isx.h")) as f:
        src = f.read()
    for name, value in (("ISX_CT_DEFAULT", 0), ("ISX_CT_NONE", 1), ("ISX_CT_RCT", 2), ("ISX_CT_YCOCG_R", 3)):
        assert re.search(rf"#define {name} {value}\b", src), name
    assert (isx.CT_DEFAULT, isx.CT_NONE, isx.CT_RCT, isx.CT_YCOCG_R) == (0, 1, 2, 3)


def test_decode_job_array_layout_matches_header():
    from paper_2005_08713_gb300 import isx
    assert ctypes.sizeof(isx.DecodeJobC) == isx.JOB_DTYPE.itemsize == 40
    for name in ("tile", "rx", "ry", "rw", "rh", "d_out", "out_pitch_bytes"):
        assert getattr(isx.DecodeJobC, name).offset == isx.JOB_DTYPE.fields[name][1], name


def test_struct_layouts_match_the_compiled_header(tmp_path):
    """The C compiler's offsets and sizes of isx_tile_desc, isx_decode_job and isx_rect_copy (a small
    program built against include/isx.h) equal the binding's ctypes and numpy layouts."""
    import shutil
    import subprocess
    import pytest
    from paper_2005_08713_gb300 import isx
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {"isx_tile_desc": [n for n, _ in isx.TileDescC._fields_],
              "isx_decode_job": ["tile", "rx", "ry", "rw", "rh", "d_out", "out_pitch_bytes"],
              "isx_rect_copy": ["src", "src_pitch", "dst", "dst_pitch", "row_bytes", "rows"]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "isx.h"', "int main(void) {"]
    for st, names in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for n in names:
            lines.append(f'  printf("{st} {n} %zu\\n", offsetof({st}, {n}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        st, name, v = line.split()
        got[(st, name)] = int(v)
    assert got[("isx_tile_desc", "size")] == ctypes.sizeof(isx.TileDescC)
    for n in fields["isx_tile_desc"]:
        assert got[("isx_tile_desc", n)] == getattr(isx.TileDescC, n).offset, n
    assert got[("isx_decode_job", "size")] == ctypes.sizeof(isx.DecodeJobC) == isx.JOB_DTYPE.itemsize
    for n in fields["isx_decode_job"]:
        assert got[("isx_decode_job", n)] == getattr(isx.DecodeJobC, n).offset == isx.JOB_DTYPE.fields[n][1], n
    assert got[("isx_rect_copy", "size")] == isx.COPY_DTYPE.itemsize == 40
    for n in fields["isx_rect_copy"]:
        assert got[("isx_rect_copy", n)] == isx.COPY_DTYPE.fields[n][1], n


def test_status_names_match_the_header_enum():
    from paper_2005_08713_gb300 import isx
    with open(os.path.join(ROOT, "include", "isx.h")) as f:
        src = f.read()
    body = src[src.index("typedef enum {"):src.index("} isx_status;")]
    enum = {int(v): n for n, v in re.findall(r"\b(ISX_[A-Z_]+)\s*=\s*(\d+)", body)}
    assert enum == isx.STATUS_NAMES
