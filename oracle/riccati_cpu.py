"""Python access to riccati_cpu.cpp: the CP operator T (Eq.
(chambolle-pock-operator)) in plain FP64 C++ with the S1 projection by
Algorithms 1 and 2 as printed, OpenMP over the nodes of a stage.
Oracle (test infrastructure only): the tests, the CPU baseline of the
benchmark and full-size checks use it; the CUDA library never does.

Pins (tests/test_oracle_riccati_cpu.py): L, L*, prox_f (Algorithm 2 against
the KKT projection), prox_g* and T agree with the Python oracle to 1e-12 on
small trees, with 1 and several threads.

    python -m oracle.riccati_cpu --build     # compiles the shared library
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "riccati_cpu.cpp")
LIB = os.path.join(HERE, "_lib", "libriccati_cpu.so")


def build(force=False):
    """g++ -O2 -fopenmp; rebuilt when the source is newer than the library."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"g++ failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


_lib = None
_D = C.POINTER(C.c_double)


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.rc_create.restype = C.c_void_p
        _lib.rc_create.argtypes = [C.c_int32, C.POINTER(C.c_int32), _D, C.c_int32, C.c_int32] + [_D] * 10 + \
            [C.c_int32]
        _lib.rc_sizes.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        _lib.rc_set_threads.argtypes = [C.c_void_p, C.c_int32]
        _lib.rc_apply_L.argtypes = [C.c_void_p, _D, _D]
        _lib.rc_apply_Lt.argtypes = [C.c_void_p, _D, _D]
        _lib.rc_prox_f.argtypes = [C.c_void_p, _D, C.c_double, _D, _D]
        _lib.rc_prox_gconj.argtypes = [C.c_void_p, C.c_double, _D, _D]
        _lib.rc_T.argtypes = [C.c_void_p, _D, C.c_double, _D, _D, _D, _D]
        _lib.rc_free.argtypes = [C.c_void_p]
    return _lib


def _p(a):
    return a.ctypes.data_as(_D)


class RiccatiCPU:
    """T and its parts on the CPU for a workload dict (see the workload
    generators); parents must precede their children in the numbering.
    Algorithm 1 runs at construction with ``threads`` OpenMP threads."""

    def __init__(self, d, threads=1):
        if "Gx" in d or np.asarray(d["Q"]).ndim == 3:
            raise NotImplementedError("RiccatiCPU: box constraints and diagonal costs only")
        lib = _load()
        self._keep = {k: np.ascontiguousarray(d[k], dtype=np.float64)
                      for k in ("prob", "A", "B", "Q", "R", "QN", "a", "xmin", "xmax", "umin", "umax")}
        anc = np.ascontiguousarray(d["anc"], dtype=np.int32)
        k = self._keep
        self.h = lib.rc_create(len(anc), anc.ctypes.data_as(C.POINTER(C.c_int32)), _p(k["prob"]), int(d["nx"]),
                               int(d["nu"]), _p(k["A"]), _p(k["B"]), _p(k["Q"]), _p(k["R"]), _p(k["QN"]), _p(k["a"]),
                               _p(k["xmin"]), _p(k["xmax"]), _p(k["umin"]), _p(k["umax"]), int(threads))
        if not self.h:
            raise ValueError("riccati_cpu: parents must precede children and Rtilde must be positive definite")
        nz, ne = C.c_int64(), C.c_int64()
        lib.rc_sizes(self.h, C.byref(nz), C.byref(ne))
        self.n_z, self.n_eta = nz.value, ne.value
        self.x0 = np.ascontiguousarray(d["x0"], dtype=np.float64)

    def set_threads(self, threads):
        _lib.rc_set_threads(self.h, int(threads))

    def apply_L(self, z):
        z = np.ascontiguousarray(z, dtype=np.float64)
        out = np.empty(self.n_eta)
        _lib.rc_apply_L(self.h, _p(z), _p(out))
        return out

    def apply_Lt(self, eta):
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        out = np.empty(self.n_z)
        _lib.rc_apply_Lt(self.h, _p(eta), _p(out))
        return out

    def prox_f(self, z, alpha, x0=None):
        z = np.ascontiguousarray(z, dtype=np.float64)
        x0 = self.x0 if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        out = np.empty(self.n_z)
        _lib.rc_prox_f(self.h, _p(x0), float(alpha), _p(z), _p(out))
        return out

    def prox_gconj(self, eta, alpha):
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        out = np.empty(self.n_eta)
        _lib.rc_prox_gconj(self.h, float(alpha), _p(eta), _p(out))
        return out

    def T(self, z, eta, alpha, x0=None, out=None):
        z = np.ascontiguousarray(z, dtype=np.float64)
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        x0 = self.x0 if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        zo, eo = (np.empty(self.n_z), np.empty(self.n_eta)) if out is None else out
        _lib.rc_T(self.h, _p(x0), float(alpha), _p(z), _p(eta), _p(zo), _p(eo))
        return zo, eo

    def close(self):
        if getattr(self, "h", None):
            _lib.rc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


if __name__ == "__main__":
    if "--build" in sys.argv:
        print(build(force="--force" in sys.argv))
