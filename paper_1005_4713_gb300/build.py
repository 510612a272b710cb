"""In-tree build of libspkmc.so for sm_103a (GB300) with nvcc.

Three translation units (the cycle kernel, the set-up and read-out kernels,
and the host runtime) are compiled in parallel and linked into
``paper_1005_4713_gb300/libspkmc.so``.  Device FP64 arithmetic is
compiled without fused multiply-add (``-fmad=false``) and host code with
``-ffp-contract=off``, so that the frequency lines are summed exactly as
written.
"""
from __future__ import annotations

import hashlib
import os
import platform
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libspkmc.so")
STAMP = LIB + ".sha256"  # hash of the sources, headers and flags the library was built from
SOURCES = ["spkmc_kernels.cu", "spkmc_setup_kernels.cu", "spkmc_api.cu"]
HEADERS = ["spkmc_internal.h", "spkmc_device.cuh", "spkmc_setup.h", os.path.join("..", "..", "include", "spkmc.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def source_hash() -> str:
    """SHA-256 of everything the library is built from: the translation
    units, the headers, the nvcc flags, the compiler path and the host
    architecture (a library built on another machine type never matches)."""
    h = hashlib.sha256()
    for name in SOURCES + HEADERS:
        path = os.path.normpath(os.path.join(CSRC, name))
        h.update(name.encode() + b"\0")
        with open(path, "rb") as f:
            h.update(f.read())
        h.update(b"\0")
    h.update(" ".join(ARCH + NVCC_FLAGS).replace(ROOT, "<root>").encode())
    h.update(nvcc().encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def _stale() -> bool:
    """A library is reused only when its stamp holds the hash of the current
    sources and flags (a library copied from elsewhere, or built from other
    sources, has none or another)."""
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    try:
        with open(STAMP) as f:
            return f.read().strip() != source_hash()
    except OSError:
        return True


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile libspkmc.so unless the one in place was built from exactly
    the current sources and flags."""
    if not force and not _stale():
        return LIB
    digest = source_hash()
    with tempfile.TemporaryDirectory(prefix="spkmc_build_") as tmp:
        procs = []
        objs = []
        for src in SOURCES:
            obj = os.path.join(tmp, src + ".o")
            cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
            objs.append(obj)
        errors = []
        for src, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                errors.append(f"{src}:\n{out.decode(errors='replace')}")
            elif verbose or ptxas_info:
                sys.stderr.write(out.decode(errors="replace"))
        if errors:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
        tmp_lib = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp_lib, *objs]
        subprocess.run(cmd, check=True)
        # the stamp goes first: a library in place without a matching stamp is rebuilt
        if os.path.exists(STAMP):
            os.remove(STAMP)
        os.replace(tmp_lib, LIB)
        tmp_stamp = STAMP + f".tmp{os.getpid()}"
        with open(tmp_stamp, "w") as f:
            f.write(digest + "\n")
        os.replace(tmp_stamp, STAMP)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
