"""The autotuner's on-disk cache (GX_TUNE_CACHE; csrc/tune_cache.h) on the host
(tests/host/tune_cache_check.cpp): FNV-1a against published vectors, the record round
trip, and malformed or refused records ignored.  The tuner's use of it needs a device."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tune_cache(tmp_path):
    import paper_2512_12615_gb300._build as B

    if not shutil.which("g++"):
        pytest.skip("no host compiler")
    exe = tmp_path / "tune_cache_check"
    cmd = ["g++", "-std=c++17", "-Wall", "-I" + B.CSRC, os.path.join(HERE, "host", "tune_cache_check.cpp"),
           "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    scratch = tmp_path / "cache"
    scratch.mkdir()
    r = subprocess.run([str(exe), str(scratch)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
