"""The batch planner's chunk cutting on the host (tests/host/plan_check.cpp): coverage of
every item's events, chunk bounds, largest-first order, program slots and the per-program
sharding choice carried on chunks.  Compiled against the engine's sources and library;
no device is touched."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_make_chunks(tmp_path):
    import paper_2512_12615_gb300._build as B

    if not shutil.which("g++") or not os.path.isdir(os.path.join(B.CUDA_HOME, "include")):
        pytest.skip("no host compiler or CUDA headers")
    B.build()
    exe = tmp_path / "plan_check"
    cmd = (["g++"] + [f for f in B.CXX_FLAGS if f != "-fPIC"] + [os.path.join(HERE, "host", "plan_check.cpp"),
           "-o", str(exe), "-L" + os.path.dirname(B.LIB), "-lgx", "-L" + os.path.join(B.CUDA_HOME, "lib64"),
           "-lcudart", "-lpthread", "-ldl", "-Wl,-rpath," + os.path.dirname(B.LIB),
           "-Wl,-rpath," + os.path.join(B.CUDA_HOME, "lib64")])
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
