"""Python side of oracle/cpu_sort.c: the oracle's stable sort run on every host
core, for timing a CPU baseline (test infrastructure, like the rest of
oracle/).  build() compiles the C file with gcc into oracle/libcpusort.so."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_sort.c")
LIB = os.path.join(HERE, "libcpusort.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for oracle/cpu_sort.c")
    tmp = LIB + ".tmp"
    subprocess.run([cc, "-O3", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, SRC], check=True)
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.pgs_cpu_stable_sort.restype = ctypes.c_int
        lib.pgs_cpu_stable_sort.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int]
        _lib = lib
    return _lib


def threads_available() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def stable_sort(keys: np.ndarray, vals: np.ndarray | None, dtype: str, threads: int | None = None):
    """Sorted copies of keys (uint32 / uint64 / float32 bits as uint32) and vals."""
    k = np.ascontiguousarray(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    T = threads or threads_available()
    rc = load().pgs_cpu_stable_sort(k.ctypes.data, v.ctypes.data if v is not None else None, len(k),
                                    8 if dtype == "u64" else 4, 1 if dtype == "f32" else 0, T)
    if rc != 0:
        raise MemoryError("pgs_cpu_stable_sort failed")
    return k, v


def cpu_model() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"
