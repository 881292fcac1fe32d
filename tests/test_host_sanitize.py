"""Memory safety and defined behaviour of the host code that reads untrusted bytecode.

The verifier and decoder (the engine's csrc/verifier.cpp, csrc/decode.cpp), the load-time
code generator (csrc/jit.cpp, source generation only) and the oracle (oracle/gx_oracle.c,
which claims to be safe on programs nobody verified) are built with AddressSanitizer and
UndefinedBehaviorSanitizer and run over a corpus: the fuzzers' program generators, the
workload programs and seeded mutants of all of them (bit flips, random words, duplicated
and dropped instructions).  A sanitizer report fails the test.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from tests.asmtext import assemble
from workloads import programs as P

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SAN = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]
ENV = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")


def corpus(seed=77):
    from tests import test_combinable_fuzz as C
    from tests import test_det_fuzz as D
    from tests import test_simt_verifier as S
    from tests import test_verifier_fuzz as V

    rng = np.random.default_rng(seed)
    out = []
    for build in (P.counting, P.page_heat, P.latency, P.warp_heat):
        out.append(build())
    out += list(P.batch_programs())
    out += [P.sched_policy(k) for k in ("fixed", "greedy", "latency_budget")]
    import json

    with open(os.path.join(HERE, "golden", "handworked.json")) as f:
        for case in json.load(f)["cases"]:  # hand-worked programs: every opcode family, faults included
            out.append((assemble(case["asm"]).prog(), case.get("maps", []), 8 * len(case["events"][0])))
    for gen, specs, cs, n in ((lambda: V.Gen(rng).program(), V.SPECS, V.CTX, 150),
                              (lambda: D.Gen(rng).program(), D.SPECS, 32, 100),
                              (lambda: C.CGen(rng).program(), D.SPECS, 32, 60),
                              (lambda: S.random_handler(rng), S.RANDOM_SPECS, 32, 100)):
        for _ in range(n):
            try:
                out.append((assemble(gen()).prog(), specs, cs))
            except Exception:  # an encoding the assembler refuses
                continue
    return out


def write_corpus(path, progs):
    with open(path, "wb") as f:
        f.write(b"GXCP" + struct.pack("<I", len(progs)))
        for insns, specs, cs in progs:
            insns = np.ascontiguousarray(insns, dtype=np.uint64)
            f.write(struct.pack("<4I", insns.size, len(specs), cs, 0))
            for s in specs:
                f.write(struct.pack("<6I", s["type"], s["key_size"], s["value_size"], s["max_entries"],
                                    s.get("flags", 0), 0))
            f.write(insns.tobytes())


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("no sanitizer runtime on this host: " + r.stderr[-300:])
    assert r.returncode == 0, r.stderr[-3000:]


@pytest.fixture(scope="module")
def corpus_file(tmp_path_factory):
    path = tmp_path_factory.mktemp("san") / "corpus.bin"
    write_corpus(path, corpus())
    return path


def test_verifier_and_decoder_under_sanitizers(corpus_file, tmp_path):
    if not shutil.which("g++"):
        pytest.skip("no host compiler")
    csrc = os.path.join(ROOT, "paper_2512_12615_gb300", "csrc")
    exe = tmp_path / "verify_sanitize"
    _compile(["g++", "-std=c++17"] + SAN + ["-I" + os.path.join(ROOT, "include"), "-I" + csrc,
              os.path.join(csrc, "verifier.cpp"), os.path.join(csrc, "decode.cpp"),
              os.path.join(HERE, "host", "verify_sanitize.cpp"), "-o", str(exe)])
    r = subprocess.run([str(exe), str(corpus_file), "8"], capture_output=True, text=True, timeout=600, env=ENV)
    assert r.returncode == 0 and r.stdout.startswith("OK"), (r.stdout[-2000:], r.stderr[-6000:])
    assert "runtime error" not in r.stderr, r.stderr[-6000:]
    counts = dict(kv.split("=") for kv in r.stdout.split()[1:])
    assert int(counts["accepted"]) > 800 and int(counts["simt_accepted"]) > 60, r.stdout


def test_oracle_under_sanitizers(corpus_file, tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("no host compiler")
    exe = tmp_path / "oracle_sanitize"
    _compile(["gcc", "-std=c11"] + SAN + [os.path.join(HERE, "host", "oracle_sanitize.c"), "-o", str(exe)])
    r = subprocess.run([str(exe), str(corpus_file), "8"], capture_output=True, text=True, timeout=600, env=ENV)
    assert r.returncode == 0 and r.stdout.startswith("OK"), (r.stdout[-2000:], r.stderr[-6000:])
    assert "runtime error" not in r.stderr, r.stderr[-6000:]


def test_code_generator_under_sanitizers(corpus_file, tmp_path):
    """Every accepted program as per-lane, multi-program, work-stealing and warp-level source
    (balanced braces and parentheses), in four parallel parts."""
    import paper_2512_12615_gb300._build as B

    if not shutil.which("g++"):
        pytest.skip("no host compiler")
    B.build()  # writes the embedded device headers the generator links against
    csrc = os.path.join(ROOT, "paper_2512_12615_gb300", "csrc")
    exe = tmp_path / "jit_sanitize"
    _compile(["g++", "-std=c++17"] + SAN + ["-O2", "-I" + os.path.join(ROOT, "include"), "-I" + csrc,
              "-I" + os.path.join(B.CUDA_HOME, "include"), os.path.join(csrc, "jit.cpp"),
              os.path.join(csrc, "verifier.cpp"), os.path.join(csrc, "decode.cpp"),
              os.path.join(B.BUILD, "gx_embed.cpp"), os.path.join(HERE, "host", "jit_sanitize.cpp"), "-o", str(exe),
              "-L" + os.path.join(B.CUDA_HOME, "lib64"), "-lcudart", "-ldl", "-lpthread",
              "-Wl,-rpath," + os.path.join(B.CUDA_HOME, "lib64")])
    procs = [subprocess.Popen([str(exe), str(corpus_file), "0", str(k), "4"], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=ENV) for k in range(4)]
    totals = {}
    for p in procs:
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0 and out.startswith("OK"), (out[-2000:], err[-6000:])
        assert "runtime error" not in err, err[-6000:]
        for kv in out.split()[1:]:
            k, v = kv.split("=")
            totals[k] = totals.get(k, 0) + int(v)
    assert totals["lane"] > 200 and totals["warp"] > 100 and totals["multi"] > 50 and totals["sched"] > 30, totals


def test_sanitized_oracle_catches_a_planted_bounds_bug(corpus_file, tmp_path):
    """The harness has teeth: in a copy of the oracle whose region check lets an access run
    past the end of its region, the same corpus makes AddressSanitizer report."""
    if not shutil.which("gcc"):
        pytest.skip("no host compiler")
    src = open(os.path.join(ROOT, "oracle", "gx_oracle.c")).read()
    old = "if (a >= b && size <= g->r[i].size && a - b <= g->r[i].size - size) {"
    assert src.count(old) == 1
    (tmp_path / "oracle").mkdir()
    (tmp_path / "tests" / "host").mkdir(parents=True)
    (tmp_path / "oracle" / "gx_oracle.c").write_text(src.replace(old, "if (a >= b && a - b <= g->r[i].size) {"))
    shutil.copy(os.path.join(HERE, "host", "oracle_sanitize.c"), tmp_path / "tests" / "host")
    exe = tmp_path / "oracle_mutant"
    _compile(["gcc", "-std=c11"] + SAN + [str(tmp_path / "tests" / "host" / "oracle_sanitize.c"), "-o", str(exe)])
    r = subprocess.run([str(exe), str(corpus_file), "8"], capture_output=True, text=True, timeout=600, env=ENV)
    assert r.returncode != 0 and "AddressSanitizer" in r.stderr, (r.stdout[-500:], r.stderr[-2000:])


def test_sanitized_verifier_catches_a_planted_bounds_bug(corpus_file, tmp_path):
    """The same for the verifier: in a copy that no longer refuses jumps past the last
    instruction, the corpus's mutants make AddressSanitizer report."""
    if not shutil.which("g++"):
        pytest.skip("no host compiler")
    csrc = os.path.join(ROOT, "paper_2512_12615_gb300", "csrc")
    src = open(os.path.join(csrc, "verifier.cpp")).read()
    old = 'if (tgt < 0 || tgt >= (s64)n) return fail(pc, "jump out of range");'
    assert src.count(old) == 1
    mutant = tmp_path / "verifier.cpp"
    mutant.write_text(src.replace(old, 'if (tgt < 0) return fail(pc, "jump out of range");'))
    exe = tmp_path / "verify_mutant"
    _compile(["g++", "-std=c++17"] + SAN + ["-I" + os.path.join(ROOT, "include"), "-I" + csrc, str(mutant),
              os.path.join(csrc, "decode.cpp"), os.path.join(HERE, "host", "verify_sanitize.cpp"), "-o", str(exe)])
    r = subprocess.run([str(exe), str(corpus_file), "8"], capture_output=True, text=True, timeout=600, env=ENV)
    assert r.returncode != 0 and "AddressSanitizer" in r.stderr, (r.stdout[-500:], r.stderr[-2000:])
