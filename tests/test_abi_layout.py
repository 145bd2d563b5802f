"""The structs of the C ABI and the ctypes binding agree field by field: a
small C program compiled against include/qwlsh.h prints every struct's size
and each field's offset, and the binding's ctypes structures must match."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "qw_index_params": ["m", "w", "c", "v", "l", "delta", "shadow_bf16", "bitmaps",
                        "host_bitmaps", "seed", "projection", "family"],
    "qw_query_params": ["batch", "profile", "path", "clusters", "order", "rerank", "start",
                        "graph", "bitmap_loads", "l2_mode", "l2_index_permille", "projection",
                        "rerank_rows", "tiles_per_warp", "probes"],
    "qw_profile": ["launches", "ms", "timed_launches", "queries", "rerank_candidates",
                   "rerank_fp32_rows", "start_levels_skipped", "start_fallbacks", "level_passes",
                   "bitmap_fallbacks", "bitmap_live_items", "bitmap_live_groups",
                   "bitmap_live_words", "l2_setaside_bytes", "l2_index_permille",
                   "bitmap_overflows"],
    "qw_index_info": ["n", "d", "m", "w", "c", "v", "l", "tile", "n_tiles", "span_max",
                      "n_fixups", "device_bytes", "bitmap_bytes", "host_bytes", "family"],
    "qw_tune_report": ["tried", "params", "ms", "best"],
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "qwlsh.h"', "int main(void) {"]
    for s, fields in STRUCTS.items():
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    return got


def test_structs_match_the_header(tmp_path):
    import paper_1907_11803_gb300 as qw
    got = _c_layout(tmp_path)
    for s, fields in STRUCTS.items():
        cls = getattr(qw, s)
        assert C.sizeof(cls) == got[(s, "size")], s
        names = [f[0] for f in cls._fields_]
        assert names == fields, (s, names)
        for f in fields:
            assert getattr(cls, f).offset == got[(s, f)], (s, f)
