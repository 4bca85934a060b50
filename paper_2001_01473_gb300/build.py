"""Build step: compiles the CUDA sources into the in-tree liban5d.so (sm_103a).

All translation units (csrc/*.cu plus small generated units that instantiate
the sweep kernels listed in kernels.py) are compiled by nvcc in parallel and
linked into paper_2001_01473_gb300/_build/liban5d.so.  Objects are cached by
a hash of their source, the headers and the flags, so a rebuild only
recompiles what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

from . import kernels

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
GEN = os.path.join(BUILD, "gen")
OBJ = os.path.join(BUILD, "obj-" + platform.machine())  # never reuse another host's objects
LIB = os.path.join(BUILD, "liban5d.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-O2", f"-I{INCLUDE}", f"-I{CSRC}"]
PER_UNIT = 3  # kernel instantiations per generated translation unit


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers_digest() -> str:
    h = hashlib.sha1()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".h", ".cuh")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    return h.hexdigest()


def _generate() -> list:
    os.makedirs(GEN, exist_ok=True)
    inst = list(kernels.instantiations())
    units = []
    for u in range(0, len(inst), PER_UNIT):
        chunk = inst[u:u + PER_UNIT]
        headers = sorted({h for h, _ in chunk})
        body = "\n".join(f"    {e}," for _, e in chunk)
        src = ("// generated by build.py from kernels.py -- do not edit\n"
               + "".join(f'#include "{h}"\n' for h in headers)
               + "namespace an5d {\nnamespace {\nconst KernelEntry k_entries[] = {\n" + body
               + "\n};\nconst Registrar k_reg(k_entries, sizeof(k_entries) / sizeof(k_entries[0]));\n"
               + "}  // namespace\n}  // namespace an5d\n")
        path = os.path.join(GEN, f"inst_{u // PER_UNIT:03d}.cu")
        old = open(path).read() if os.path.exists(path) else None
        if old != src:
            with open(path, "w") as f:
                f.write(src)
        units.append(path)
    for f in os.listdir(GEN):
        p = os.path.join(GEN, f)
        if p not in units:
            os.remove(p)
    return units


def _compile(src: str, hdr: str, verbose: bool) -> str:
    with open(src, "rb") as f:
        key = hashlib.sha1(f.read() + hdr.encode() + " ".join(NVCC_FLAGS).encode()).hexdigest()[:16]
    obj = os.path.join(OBJ, os.path.basename(src) + f".{key}.o")
    if os.path.exists(obj):
        return obj
    tmp = obj + f".tmp{os.getpid()}"
    cmd = [nvcc()] + NVCC_FLAGS + ["-c", src, "-o", tmp]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, obj)
    return obj


def build(jobs: int | None = None, verbose: bool = False) -> str:
    """Compile and link the library if anything changed; return its path."""
    os.makedirs(OBJ, exist_ok=True)
    srcs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    srcs += _generate()
    hdr = _headers_digest()
    jobs = jobs or os.cpu_count() or 4
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, hdr, verbose), srcs))
    link_key = hashlib.sha1("\n".join(objs).encode()).hexdigest()
    stamp = LIB + ".key"
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == link_key:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    if verbose:
        print(" ".join(cmd[:8]) + " ...", file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(link_key)
    # drop stale objects
    keep = set(objs)
    for f in os.listdir(OBJ):
        p = os.path.join(OBJ, f)
        if p not in keep and not f.endswith(".tmp"):
            try:
                os.remove(p)
            except OSError:
                pass
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
