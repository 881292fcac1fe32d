"""Host-only: the source tree stays small whatever the engine compiles.

Compiled programs are cached outside the package (GX_JIT_CACHE defaults to a per-user
folder), and the tree a GPU run copies must stay far below the copy limit of a remote run.
"""
import os

import pytest

import paper_2512_12615_gb300 as gx
from paper_2512_12615_gb300 import gx as binding
from workloads import programs as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2512_12615_gb300")
LIMIT_MIB = 200
# not part of what a run copies: history, and the folder results come back into
SKIP = {".git", "gpurun_out"}


def _tree_bytes(top):
    total = 0
    for d, dirs, files in os.walk(top):
        if d == top:
            dirs[:] = [x for x in dirs if x not in SKIP]
        for f in files:
            try:
                total += os.lstat(os.path.join(d, f)).st_size
            except OSError:
                pass
    return total


def _files(top):
    out = set()
    for d, _, files in os.walk(top):
        for f in files:
            out.add(os.path.relpath(os.path.join(d, f), top))
    return out


def test_default_jit_cache_is_outside_the_tree(monkeypatch):
    monkeypatch.delenv("XDG_CACHE_HOME", raising=False)
    path = os.path.realpath(binding.default_jit_cache())
    assert not path.startswith(os.path.realpath(ROOT) + os.sep)
    monkeypatch.setenv("XDG_CACHE_HOME", "/var/cache/someone")
    assert binding.default_jit_cache() == "/var/cache/someone/gx-jit"


def test_compiling_writes_nothing_into_the_package():
    gx.lib()
    before = _files(PKG)
    prog, specs, cs = P.counting()
    rc, log = gx.jit_check(prog, specs, cs, deterministic=True)
    if rc == gx.E_NODEV:
        pytest.skip("no runtime compiler on this host")
    assert rc == 0, log
    added = {f for f in _files(PKG) - before if "__pycache__" not in f}
    assert not added, f"compilation wrote into the package tree: {sorted(added)[:10]}"


def test_tree_is_small():
    mib = _tree_bytes(ROOT) / 2**20
    assert mib < LIMIT_MIB, f"the tree outside .git holds {mib:.0f} MiB (limit {LIMIT_MIB} MiB)"
