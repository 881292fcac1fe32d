"""The work-stealing walk of the persistent kernel on the host (tests/host/steal_check.cpp):
the shares cut the chunk table exactly; whatever a `should_try_steal` policy answers and
however blocks interleave (host threads claiming with atomic adds), every chunk runs once,
a policy that never steals leaves each block its own share, the per-block counters agree
and every walk ends within its claim bound; plus exact pins for blocks walked in turn.  The
walk of one block per chunk (cancel_walk) runs over a model of the launcher: a cancelled
block never starts and no block cancels again after a failed cancel.
The same check run over planted mistakes in a copy of the walk must fail.  No device is
touched."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _run_check(tmp_path, header_dir=None):
    import paper_2512_12615_gb300._build as B

    if not shutil.which("g++"):
        pytest.skip("no host compiler")
    exe = tmp_path / "steal_check"
    inc = ([f"-I{header_dir}"] if header_dir else []) + [f"-I{B.CSRC}"]
    cmd = (["g++"] + inc + [f for f in B.CXX_FLAGS if f != "-fPIC"] +
           [os.path.join(HERE, "host", "steal_check.cpp"), "-o", str(exe), "-pthread"])
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)


def test_steal_walk(tmp_path):
    r = _run_check(tmp_path)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr


# plausible mistakes in the walk, each of which breaks exactly-once, the share cut, the
# counters or the policy's power to stop a block
MUTANTS = {
    "owner runs one past its share": ("if (k >= size) break;\n        run(lo + k);\n        t[GX_STEAL_OWNED]++;",
                                      "if (k > size) break;\n        run(lo + k);\n        t[GX_STEAL_OWNED]++;"),
    "thief runs one past the share": ("if (k >= size) break;\n            run(lo + k);",
                                      "if (k > size) break;\n            run(lo + k);"),
    "stolen counted before the claim": ("t[GX_STEAL_GRANTED]++;\n            const uint32_t k = claim(v);",
                                        "t[GX_STEAL_GRANTED]++;\n            t[GX_STEAL_STOLEN]++;\n"
                                        "            const uint32_t k = claim(v);"),
    "share cut drops the remainder": ("return (uint32_t)((uint64_t)s * n / shares);",
                                      "return (uint32_t)(s * (n / shares));"),
    "a refusal only skips one share": ("if (!ask(v, l, t[GX_STEAL_OWNED] + t[GX_STEAL_STOLEN])) return;",
                                       "if (!ask(v, l, t[GX_STEAL_OWNED] + t[GX_STEAL_STOLEN])) break;"),
    "the owner never drains": ("    for (;;) {\n        const uint32_t k = claim(self);",
                               "    for (int once_ = 0; once_ < 1; once_++) {\n        const uint32_t k = claim(self);"),
    "restarts the search from the first share": ("o < shares; o = find(o))", "o < shares; o = find(0u))"),
    # one block per chunk (cancel_walk)
    "cancels again after a failed cancel": ("const uint32_t c = cancel();\n        if (c >= n) break;",
                                            "const uint32_t c = cancel();\n        if (c >= n) continue;"),
    "asks with nothing left": ("const uint32_t l = left();\n        if (l == 0) break;",
                               "const uint32_t l = left();"),
    "runs its own chunk again for a cancelled one": ("if (c >= n) break;\n        run(c);",
                                                      "if (c >= n) break;\n        run(self);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_steal_check_catches_mutant(tmp_path, name):
    import paper_2512_12615_gb300._build as B

    src = open(os.path.join(B.CSRC, "gx_steal.cuh")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    mdir = tmp_path / "mutant"
    mdir.mkdir()
    (mdir / "gx_steal.cuh").write_text(src.replace(old, new))
    r = _run_check(tmp_path, mdir)
    assert r.returncode != 0 and "FAIL" in r.stdout, (name, r.stdout[-2000:])
