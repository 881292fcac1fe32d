"""Host-only: the region tests of the checked interpreter (GX_PROG_CHECKED), compiled from
gx_layout.h for the host (tests/host/access_check.cpp): every edge of the stack and of
array, hash and ring-buffer regions, misalignment, empty and wrapping ranges."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_access_checks(tmp_path):
    import paper_2512_12615_gb300._build as B

    if not shutil.which("g++"):
        pytest.skip("no host compiler")
    exe = tmp_path / "access_check"
    cmd = ["g++", "-std=c++17", "-Wall", "-I" + B.CSRC, "-I" + B.INCLUDE, os.path.join(HERE, "host", "access_check.cpp"),
           "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
