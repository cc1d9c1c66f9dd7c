"""Build the native libraries (CUDA for sm_103a + C++ host runtime) in-tree.

``python -m paper_1112_0065_gb300._build`` or ``build()`` compiles every
``csrc/*.cu`` translation unit with nvcc in parallel and links
``_build/libdd.so`` (the product library); ``csrc/probe/*.cu`` become
``_build/libddprobe.so`` (measurement probes for the tests and the benchmark,
not part of the product).

An object is rebuilt when its key changes: a SHA-256 over the compiler
command, the machine architecture, the source text and the text of every
header under ``csrc/`` and ``include/``.  Modification times play no part, so
objects copied from another machine or left from older sources are never
linked.
"""
from __future__ import annotations

import glob
import hashlib
import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libdd.so")
PROBE_LIB = os.path.join(BUILD, "libddprobe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")] + ARCH


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _headers():
    pats = ("*.h", "*.cuh")
    found = []
    for d in (CSRC, os.path.join(CSRC, "probe"), os.path.join(ROOT, "include")):
        for p in pats:
            found += glob.glob(os.path.join(d, p))
    return sorted(found)


def _digest(parts) -> str:
    h = hashlib.sha256()
    for p in parts:
        h.update(p if isinstance(p, bytes) else str(p).encode())
        h.update(b"\0")
    return h.hexdigest()


def _read(path) -> bytes:
    with open(path, "rb") as fh:
        return fh.read()


def _key_ok(path: str, key: str) -> bool:
    try:
        return os.path.exists(path) and _read(path + ".key").decode() == key
    except OSError:
        return False


def _write_key(path: str, key: str) -> None:
    with open(path + ".key", "w") as fh:
        fh.write(key)


def _compile_all(groups, force: bool, verbose: bool):
    """groups: {lib_path: [sources]} -> {lib_path: [(obj, key)]}, compiling
    every object whose key changed (all in one thread pool)."""
    nvcc = _nvcc()
    hdr_key = _digest([os.path.relpath(h, ROOT).encode() + b"\0" + _read(h) for h in _headers()])
    objs, jobs = {}, []
    for lib, srcs in groups.items():
        tag = os.path.splitext(os.path.basename(lib))[0]
        objs[lib] = []
        for s in srcs:
            o = os.path.join(BUILD, f"{tag}_{os.path.basename(s)[:-3]}.o")
            cmd = [nvcc] + NVCC_FLAGS + ["-c", s, "-o", o + ".tmp"]
            key = _digest([" ".join(cmd[1:]), platform.machine(), _read(s), hdr_key])
            objs[lib].append((o, key))
            if force or not _key_ok(o, key):
                jobs.append((cmd, o, key))

    def compile_one(job):
        cmd, o, key = job
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(o)}:\n{r.stderr}")
        os.replace(o + ".tmp", o)
        _write_key(o, key)
        return r.stderr

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for msg in ex.map(compile_one, jobs):
                if verbose and msg:
                    print(msg)
    return objs


def _link(lib: str, objs, force: bool) -> None:
    key = _digest([platform.machine()] + [k for _, k in objs])
    if not force and _key_ok(lib, key):
        return
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in objs] + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stderr}")
    os.replace(tmp, lib)
    _write_key(lib, key)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libdd.so and libddprobe.so; returns libdd.so's path."""
    os.makedirs(BUILD, exist_ok=True)
    groups = {LIB: sorted(glob.glob(os.path.join(CSRC, "*.cu"))),
              PROBE_LIB: sorted(glob.glob(os.path.join(CSRC, "probe", "*.cu")))}
    objs = _compile_all(groups, force, verbose)
    for lib, ol in objs.items():
        _link(lib, ol, force)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
