"""Build the CUDA library ``_build/libnetburn.so`` for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libnetburn.so")
SOURCES = ["burn.cu", "adjoint.cu", "noalloc.cu", "multi.cu", "expcheck.cu", "netload.cpp",
           "codegen.cpp"]
HEADERS = ["blob.h", "device.cuh", "integrator.cuh", "adjoint.cuh", "coop.cuh", "host.h",
           "expf64.cuh", "codegen.h"]
# headers the run-time compiler needs, embedded as text into the library
# (name as written in the #include directive, path)
EMBED = [("expf64.cuh", "csrc/expf64.cuh"), ("integrator.cuh", "csrc/integrator.cuh"),
         ("blob.h", "csrc/blob.h"), ("../../include/netburn.h", "../include/netburn.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(HERE, "..", "include", "netburn.h"))
    return [f for f in files if os.path.exists(f)]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def _write_embedded() -> str:
    """Write _build/nb_embedded.h: the run-time compiler's headers as raw
    string literals."""
    path = os.path.join(BUILD, "nb_embedded.h")
    lines = ["// written by build.py: headers of the run-time compiled kernel", "#pragma once"]
    names, srcs = [], []
    for name, rel in EMBED:
        with open(os.path.join(HERE, rel)) as f:
            text = f.read()
        if ")NBSRC" in text:
            raise RuntimeError(rel + " contains the raw-string delimiter")
        names.append('"%s"' % name)
        srcs.append('R"NBSRC(' + text + ')NBSRC"')
    lines.append("static const int kEmbedCount = %d;" % len(EMBED))
    lines.append("static const char* const kEmbedNames[] = {%s};" % ", ".join(names))
    lines.append("static const char* const kEmbedSources[] = {\n" + ",\n".join(srcs) + "};")
    text = "\n".join(lines) + "\n"
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as f:
            f.write(text)
    return path


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel, then link the shared
    library.  Returns the library path."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    _write_embedded()
    nvcc = os.environ.get("NVCC", "nvcc")
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(HERE, "..", "include"), "-I", BUILD]
    procs, objs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        cmd = [nvcc] + common + ["-c", path, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs +
                          ["-lcudart", "-ldl"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
