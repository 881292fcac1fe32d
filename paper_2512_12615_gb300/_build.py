"""Builds the engine library `_build/libgx.so` in-tree.

CUDA sources are compiled by nvcc for sm_103a only; host C++ by g++; all translation
units compile in parallel, and a stamp of the sources and flags skips work that is
already done.  No CMake, no Python extension machinery.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgx.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-I" + INCLUDE, "-I" + os.path.join(CUDA_HOME, "include")]

CU_SOURCES = ["interp.cu"]
CXX_SOURCES = ["verifier.cpp", "decode.cpp", "api.cpp", "batch.cpp", "jit.cpp"]
HEADERS = ["gx_layout.h", "gx_internal.h", "gx_kernels.h", "gx_runtime.h", "gx_device.cuh", "gx_jit.h", "gx_steal.cuh", "tune_cache.h",
           "gx_trace.h"]


def _stamp() -> str:
    h = hashlib.sha256()
    for f in CU_SOURCES + CXX_SOURCES + HEADERS:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    with open(os.path.join(INCLUDE, "gx.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + CXX_FLAGS).encode())
    return h.hexdigest()


def _obj_stamp(src: str, flags) -> str:
    h = hashlib.sha256()
    with open(os.path.join(CSRC, src), "rb") as fh:
        h.update(fh.read())
    for f in HEADERS:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(INCLUDE, "gx.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(flags).encode())
    return h.hexdigest()[:16]


def _compile(src: str, verbose: bool) -> str:
    is_cu = src.endswith(".cu")
    flags = NVCC_FLAGS if is_cu else CXX_FLAGS
    obj = os.path.join(BUILD, f"{src}.{_obj_stamp(src, flags)}.o")
    if os.path.exists(obj):
        return obj
    cmd = ([NVCC] + flags + (["-Xptxas", "-v"] if verbose else []) if is_cu else ["g++"] + flags)
    tmp = obj + f".tmp{os.getpid()}"
    cmd += ["-c", os.path.join(CSRC, src), "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stderr or r.stdout):
        sys.stderr.write(r.stdout + r.stderr)
    os.replace(tmp, obj)
    return obj


EMBED = [("gx_h", os.path.join(INCLUDE, "gx.h")), ("gx_layout_h", os.path.join(CSRC, "gx_layout.h")),
         ("gx_device_cuh", os.path.join(CSRC, "gx_device.cuh")), ("gx_steal_cuh", os.path.join(CSRC, "gx_steal.cuh"))]


def _write_embed() -> str:
    """The device headers as C strings, handed to NVRTC when programs are specialised."""
    out = os.path.join(BUILD, "gx_embed.cpp")
    parts = ["/* generated by _build.py: device headers for load-time compilation */\n"]
    for name, path in EMBED:
        with open(path) as fh:
            text = fh.read()
        assert ")GXEMBED\"" not in text
        parts.append(f'extern "C" const char gx_embed_{name}[] = R"GXEMBED({text})GXEMBED";\n')
    body = "".join(parts)
    if not os.path.exists(out) or open(out).read() != body:
        with open(out, "w") as fh:
            fh.write(body)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libgx.so if the sources changed; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp_file = os.path.join(BUILD, "libgx.stamp")
    stamp = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read().strip() == stamp:
                return LIB
    if shutil.which(NVCC) is None and not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    srcs = CU_SOURCES + CXX_SOURCES
    embed = _write_embed()
    with ThreadPoolExecutor(max_workers=len(srcs) + 1) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), srcs))
        embed_obj = os.path.join(BUILD, "gx_embed.o")
        r = subprocess.run(["g++", "-c", "-fPIC", "-O1", embed, "-o", embed_obj], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"embed compile failed\n{r.stderr}")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-shared", "-o", tmp] + objs + [embed_obj, "-L" + os.path.join(CUDA_HOME, "lib64"), "-lcudart",
                                                  "-lpthread", "-ldl", "-Wl,-rpath," + os.path.join(CUDA_HOME, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    _remove_stale_objects(set(objs))
    return LIB


def _remove_stale_objects(keep) -> None:
    """Objects of earlier source versions (their names carry a stamp) are not kept."""
    for name in os.listdir(BUILD):
        path = os.path.join(BUILD, name)
        if name.endswith(".o") and name != "gx_embed.o" and path not in keep:
            try:
                os.remove(path)
            except OSError:
                pass


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
