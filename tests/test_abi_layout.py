"""Host-only: every structure the ctypes binding mirrors has the C header's size and field
offsets (a C program compiled against include/gx.h prints them)."""
import os
import shutil
import subprocess

import pytest

from paper_2512_12615_gb300 import gx as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MIRRORS = {
    "gx_map_spec": G.MapSpec,
    "gx_prog_opts": G.ProgOpts,
    "gx_launch": G.Launch,
    "gx_analysis": G.Analysis,
    "gx_run_stats": G.RunStats,
    "gx_server_opts": G.ServerOpts,
    "gx_completion": G.Completion,
    "gx_request": G.Request,
    "gx_simt_spec": G.SimtSpec,
    "gx_simt_report": G.SimtReport,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("cc") or shutil.which("gcc")
    if not cc:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "gx.h"', "int main(void) {"]
    for cname, py in MIRRORS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = line.split()
        out[(a, b)] = int(v)
    return out


@pytest.mark.parametrize("cname", sorted(MIRRORS))
def test_mirror_matches_header(c_layout, cname):
    py = MIRRORS[cname]
    import ctypes

    assert ctypes.sizeof(py) == c_layout[(cname, "size")], cname
    for fname, _ in py._fields_:
        assert getattr(py, fname).offset == c_layout[(cname, fname)], (cname, fname)
