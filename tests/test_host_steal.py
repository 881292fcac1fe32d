"""The work-stealing walk of the persistent kernel on the host (tests/host/steal_check.cpp):
the shares cut the chunk table exactly; whatever a `should_try_steal` policy answers and
however blocks interleave (host threads claiming with atomic adds), every chunk runs once,
a policy that never steals leaves each block its own share, the per-block counters agree
and every walk ends within its claim bound; plus exact pins for blocks walked in turn.
No device is touched."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_steal_walk(tmp_path):
    import paper_2512_12615_gb300._build as B

    if not shutil.which("g++"):
        pytest.skip("no host compiler")
    exe = tmp_path / "steal_check"
    cmd = (["g++"] + [f for f in B.CXX_FLAGS if f != "-fPIC"] +
           [os.path.join(HERE, "host", "steal_check.cpp"), "-o", str(exe), "-pthread"])
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
