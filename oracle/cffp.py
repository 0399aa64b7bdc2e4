"""The C version of the FP64 oracle FFP (oracle/ffp_ref.c), run on all host cores.

TEST INFRASTRUCTURE ONLY (see the package docstring): it computes what fp64.ffp() computes
(f64 storage, no row L2), as loops in C with OpenMP over rows, so that the oracle can be timed
on every host core as the CPU baseline. build() compiles it with gcc (no -march flags, so the
same source builds on x86 and Arm hosts); ffp() loads the library on first use.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ffp_ref.c")
LIB = os.path.join(HERE, "_build", "libffp_ref.so")
_lib = None


def build(force=False):
    """Compile libffp_ref.so (gcc -O2 -fopenmp); returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the C oracle")
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    r = subprocess.run([cc, "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"], capture_output=True,
                       text=True)
    if r.returncode != 0:
        raise RuntimeError(f"building the C oracle failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.oracle_ffp.restype = ctypes.c_int
        L.oracle_ffp.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        L.oracle_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def threads():
    """Threads the C oracle runs on by default (OpenMP's count: the host cores it may use)."""
    return int(_load().oracle_threads())


def ffp(row_ptr, col, X, tau, L, alpha=1.0, theta=0.1, eps=1e-3, ddof=1, nthreads=0):
    """fp64.ffp(row_ptr, col, X, tau, L, alpha, theta, eps, ddof) in C on `nthreads` threads
    (0: all). Returns Z~ (N x d, fp64)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    N = rp.size - 1
    if X.shape[0] != N:
        raise ValueError("X must have N rows")
    d = X.shape[1]
    out = np.empty((N, d), dtype=np.float64)
    st = _load().oracle_ffp(N, rp.ctypes.data, cl.ctypes.data if cl.size else None, X.ctypes.data, d, float(tau),
                            int(L), float(alpha), float(theta), float(eps), int(ddof), int(nthreads),
                            out.ctypes.data)
    if st != 0:
        raise RuntimeError(f"oracle_ffp failed ({st})")
    return out
