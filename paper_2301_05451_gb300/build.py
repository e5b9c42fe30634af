"""Builds the library: every .cu/.cpp under csrc/ compiled for sm_103a with
nvcc (in parallel) and linked into libtdq.so beside this file."""
from __future__ import annotations

import hashlib
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtdq.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-I" + OUT]
CUDA_LIB = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(NVCC))), "lib64")
# device headers compiled again at run time (specialised sweep programs)
JIT_HEADERS = [os.path.join(ROOT, "include", "tdq.h")] + [
    os.path.join(CSRC, f) for f in ("sweep_common.cuh", "engine.cuh", "k1_body.cuh", "k2_body.cuh")]


def _write_jit_headers():
    """jit_headers.inc: the run-time compiled headers as string literals."""
    names, bodies = [], []
    for path in JIT_HEADERS:
        text = open(path).read()
        if ")TDQJIT\"" in text:
            raise RuntimeError("raw-string delimiter found in " + path)
        names.append('"%s"' % os.path.basename(path))
        bodies.append('R"TDQJIT(' + text + ')TDQJIT"')
    out = ["// Generated by build.py from the device headers; not edited by hand.",
           "static const int kJitHeaderCount = %d;" % len(names),
           "static const char* const kJitHeaderNames[] = {%s};" % ", ".join(names),
           "static const char* const kJitHeaderSrc[] = {", ",\n".join(bodies), "};", ""]
    dst = os.path.join(OUT, "jit_headers.inc")
    data = "\n".join(out)
    if not os.path.exists(dst) or open(dst).read() != data:
        with open(dst, "w") as f:
            f.write(data)


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _digest():
    h = hashlib.sha256()
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in sorted(os.listdir(d)):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode())
                h.update(fh.read())
    # the flags without this checkout's absolute paths, so that the same sources
    # give the same digest on every machine
    h.update(" ".join(f.replace(ROOT, ".") for f in FLAGS).encode())
    return h.hexdigest()


# The files that determine the specialised whole-state kernel (its generated
# source, the headers compiled with it, and the host code that picks its launch
# shape); a measurement of that kernel stays valid while these are unchanged.
K2_KERNEL_FILES = ["include/tdq.h"] + ["paper_2301_05451_gb300/csrc/" + f for f in (
    "sweep.cu", "sweep_jit.cu", "sweep_jit.h", "sweep_common.cuh", "engine.cuh", "k2_body.cuh", "k1_body.cuh",
    "sweep_tiled.cuh", "tdq_internal.h")]
# The same for the tiled sweep's kernels: the whole-state set plus the host code
# that cuts the tile passes and picks their launch shape.
K1_KERNEL_FILES = K2_KERNEL_FILES + ["paper_2301_05451_gb300/csrc/sweep_tiled.cu"]


def files_digest(relpaths):
    """SHA-256 of the named files (paths relative to the repository root) and
    the compile flags, the same on every machine."""
    h = hashlib.sha256()
    for rel in sorted(relpaths):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(rel.encode())
            h.update(fh.read())
    h.update(" ".join(f.replace(ROOT, ".") for f in FLAGS).encode())
    return h.hexdigest()


def build(force=False, verbose=False):
    """Compile and link libtdq.so unless it is up to date; returns its path."""
    stamp = os.path.join(OUT, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    os.makedirs(OUT, exist_ok=True)
    _write_jit_headers()

    def compile_one(src):
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        cmd = [NVCC] + FLAGS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + [
        "-lcudart_static", "-L" + CUDA_LIB, "-lnvrtc", "-lnvJitLink", "-Xlinker", "-rpath=" + CUDA_LIB, "-ldl", "-lrt", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
