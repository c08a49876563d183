"""Python binding of libspock (include/spock.h): argument marshalling only.

Every function named ``spock_*`` calls the C entry point of the same name.
Host-buffer calls take numpy arrays; ``*_dev`` calls take CUDA tensors
(torch is used only as the owner of device memory and streams).  The
library must be built (``paper_2212_01110_gb300.build.build()``); importing
this module without it raises ``ImportError`` -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libspock.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libspock.so is not built ({LIB_PATH}); run paper_2212_01110_gb300.build.build()")
_lib = C.CDLL(LIB_PATH)

SPOCK_OK = 0
SPOCK_MAX_ITER = 1
SPOCK_FP64 = 0
SPOCK_FP32 = 1
SPOCK_ERR_INVALID_ARG = -1
SPOCK_ERR_BAD_TREE = -2
SPOCK_ERR_NOT_POSDEF = -3
SPOCK_ERR_NUMERICAL = -4
SPOCK_ERR_CUDA = -5
SPOCK_ERR_OOM = -6
SPOCK_ERR_UNSUPPORTED = -7
ERRORS = {-1: "INVALID_ARG", -2: "BAD_TREE", -3: "NOT_POSDEF", -4: "NUMERICAL", -5: "CUDA", -6: "OOM",
          -7: "UNSUPPORTED"}
BRANCHES = {0: "K0", 1: "K1", 2: "K2", 3: "CAP"}


class SpockError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Settings(C.Structure):
    _fields_ = [("eps_abs", C.c_double), ("eps_rel", C.c_double), ("alpha", C.c_double),
                ("memory", C.c_int32), ("c0", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
                ("beta", C.c_double), ("sigma", C.c_double), ("lambda_", C.c_double),
                ("rho_coef", C.c_double), ("max_iter", C.c_int32), ("max_backtracks", C.c_int32),
                ("precision", C.c_int32), ("trace", C.POINTER(C.c_int32)), ("profile", C.c_int32),
                ("fp64_tail", C.c_int32), ("stall_window", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("n_T", C.c_int32),
                ("n_K0", C.c_int32), ("n_K1", C.c_int32), ("n_K2", C.c_int32), ("n_cap", C.c_int32),
                ("n_backtracks", C.c_int32), ("xi", C.c_double), ("xi0", C.c_double),
                ("alpha", C.c_double), ("solve_ms", C.c_double), ("n_launches", C.c_int32),
                ("n_timed", C.c_int32), ("t_group_ms", C.c_double * 7), ("fp64_iterations", C.c_int32),
                ("certified", C.c_int32), ("xi_fp32", C.c_double), ("n_L", C.c_int32)]

    GROUPS = ("prep", "bwd_chain", "bwd_stages", "fwd_stages", "fwd_chain", "dual", "stats")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "t_group_ms"}
        d["t_group_ms"] = dict(zip(self.GROUPS, list(self.t_group_ms)))
        return d


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)

_sig = {
    "spock_default_settings": ([C.POINTER(Settings)], C.c_int),
    "spock_tree_create": ([C.c_int32, _I32, _D, C.POINTER(_P)], C.c_int),
    "spock_tree_create_abs": ([C.c_int32, _I32, _D, C.POINTER(_P)], C.c_int),
    "spock_tree_info": ([_P, _I32, _I32, _I32], C.c_int),
    "spock_problem_create": ([_P, C.c_int32, C.c_int32] + [_D] * 10 + [C.c_int32, C.POINTER(_P)], C.c_int),
    "spock_problem_create_general": ([_P, C.c_int32, C.c_int32] + [_D] * 6 + [_P, C.c_int32] + [_D] * 4
                                     + [C.c_int32] + [_D] * 3 + [C.c_int32, C.POINTER(_P)], C.c_int),
    "spock_problem_info": ([_P, _I64, _I64, _D, _D], C.c_int),
    "spock_problem_clone": ([_P, C.POINTER(_P)], C.c_int),
    "spock_solve": ([_P, _D, C.POINTER(Settings), _D, _D, C.c_int32, C.POINTER(Info)], C.c_int),
    "spock_solve_dev": ([_P, _P, C.POINTER(Settings), _P, _P, C.c_int32, C.POINTER(Info), _P], C.c_int),
    "spock_cp_step": ([_P, _D, C.c_int32, C.c_double, C.c_int32, _D, _D, _D], C.c_int),
    "spock_cp_step_dev": ([_P, _P, C.c_int32, C.c_double, C.c_int32, _P, _P, _D, _P], C.c_int),
    "spock_apply_L_dev": ([_P, _P, _P, _P], C.c_int),
    "spock_apply_Lt_dev": ([_P, _P, _P, _P], C.c_int),
    "spock_prox_f_dev": ([_P, _P, C.c_double, _P, _P, _P], C.c_int),
    "spock_prox_f_noalloc_dev": ([_P, _P, C.c_double, _P, _P, _P], C.c_int),
    "spock_prox_gconj_dev": ([_P, C.c_double, _P, _P, _P], C.c_int),
    "spock_T_dev": ([_P, _P, C.c_double, _P, _P, _P, _P, _P], C.c_int),
    "spock_grad_dev": ([_P, _P, _P, C.c_int32, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "spock_grad": ([_P, _D, _D, C.c_int32, _D, _D, _D, _D, _D, _D], C.c_int),
    "spock_adjoint_dev": ([_P, _P, _P, _P, C.c_int32, C.c_double] + [_P] * 6 + [_I32, _D, _P], C.c_int),
    "spock_batch_create": ([C.c_int32, C.POINTER(_P), C.POINTER(_P)], C.c_int),
    "spock_batch_solve_dev": ([_P, C.POINTER(_P), C.POINTER(Settings), C.POINTER(_P), C.POINTER(_P), C.c_int32,
                               C.POINTER(Info)], C.c_int),
    "spock_batch_solve": ([_P, C.POINTER(_D), C.POINTER(Settings), C.POINTER(_D), C.POINTER(_D), C.c_int32,
                           C.POINTER(Info)], C.c_int),
    "spock_fp64_fma_rate": ([C.c_int32, _D, _P], C.c_int),
    "spock_free": ([_P], None),
    "spock_last_error": ([], C.c_char_p),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_sig)


def _check(rc, ok=(SPOCK_OK,)):
    if rc not in ok:
        raise SpockError(rc, _lib.spock_last_error().decode())
    return rc


def _dptr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _tptr(t, numel=None, dtype=None):
    """Device pointer of a contiguous CUDA tensor (checked)."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# thin wrappers with the C names
# ---------------------------------------------------------------------------

def spock_default_settings(**overrides):
    s = Settings()
    _check(_lib.spock_default_settings(C.byref(s)))
    for k, v in overrides.items():
        setattr(s, "lambda_" if k == "lambda" else k, v)
    return s


def spock_tree_create(anc, prob):
    anc = np.ascontiguousarray(anc, dtype=np.int32)
    prob, pp = _dptr(prob)
    h = _P()
    _check(_lib.spock_tree_create(len(anc), anc.ctypes.data_as(_I32), pp, C.byref(h)))
    return h


def spock_tree_create_abs(anc, pi):
    """Tree from absolute node probabilities pi^i."""
    anc = np.ascontiguousarray(anc, dtype=np.int32)
    pi, pp = _dptr(pi)
    h = _P()
    _check(_lib.spock_tree_create_abs(len(anc), anc.ctypes.data_as(_I32), pp, C.byref(h)))
    return h


SPOCK_DENSE_COST = 1


class Risk(C.Structure):
    """spock_risk: a coherent risk measure in conic form at one node."""
    _fields_ = [("ny", C.c_int32), ("n_nu", C.c_int32), ("kp", C.c_int32),
                ("b", _D), ("E", _D), ("F", _D)]


def _risk_array(risk):
    """ctypes array of spock_risk from a per-node list (None at leaves) of
    dicts b, E, F, kp; returns (array, arrays kept alive)."""
    arr = (Risk * len(risk))()
    keep = []
    for i, r in enumerate(risk):
        if r is None:
            continue
        b, pb = _dptr(r["b"])
        E, pE = _dptr(r["E"])
        F = np.asarray(r.get("F", np.zeros((b.size, 0))), float)
        nnu = F.shape[1] if F.ndim == 2 else 0
        Fa, pF = _dptr(F) if nnu > 0 else (None, None)
        arr[i] = Risk(b.size, nnu, int(r["kp"]), pb, pE, pF)
        keep += [b, E, Fa]
    return arr, keep


def spock_problem_create(tree, d):
    """Problem from a workload dict: the box form, or -- when the dict has
    constraint matrices "Gx" or conic risk measures "risk" --
    spock_problem_create_general (box constraints become Gamma = I).  Q, R,
    QN given as [n][nx][nx] arrays are dense (SPOCK_DENSE_COST)."""
    nx, nu = int(d["nx"]), int(d["nu"])
    dense = np.asarray(d["Q"]).ndim == 3
    flags = SPOCK_DENSE_COST if dense else 0
    h = _P()
    risk = d.get("risk")
    if "Gx" in d or risk is not None:
        if "Gx" not in d:   # box constraints as constraint rows
            n = len(d["anc"])
            Gx = np.zeros((n, nx + nu, nx))
            Gu = np.zeros((n, nx + nu, nu))
            Gx[:, :nx] = np.eye(nx)
            Gu[:, nx:] = np.eye(nu)
            d = dict(d, Gx=Gx, Gu=Gu, cmin=np.concatenate([d["xmin"], d["umin"]], 1),
                     cmax=np.concatenate([d["xmax"], d["umax"]], 1), GN=np.repeat(np.eye(nx)[None], n, 0),
                     cNmin=d["xmin"], cNmax=d["xmax"])
        nc, ncN = int(np.asarray(d["Gx"]).shape[1]), int(np.asarray(d["GN"]).shape[1])
        arrs = [_dptr(d[k]) for k in ("A", "B", "Q", "R", "QN", "a")]
        cons = [_dptr(d[k]) for k in ("Gx", "Gu", "cmin", "cmax")]
        term = [_dptr(d[k]) for k in ("GN", "cNmin", "cNmax")]
        rarr, keep = _risk_array(risk) if risk is not None else (None, [])
        _check(_lib.spock_problem_create_general(tree, nx, nu, *[p for _, p in arrs],
                                                 C.cast(rarr, _P) if rarr is not None else None, nc,
                                                 *[p for _, p in cons], ncN, *[p for _, p in term], flags,
                                                 C.byref(h)))
        del keep
        return h
    arrs = [_dptr(d[k]) for k in ("A", "B", "Q", "R", "QN", "a", "xmin", "xmax", "umin", "umax")]
    _check(_lib.spock_problem_create(tree, nx, nu, *[p for _, p in arrs], flags, C.byref(h)))
    return h


def spock_problem_clone(problem):
    """A problem sharing the data and factors of `problem` (device memory),
    with its own iterate and scratch buffers."""
    h = _P()
    _check(_lib.spock_problem_clone(problem, C.byref(h)))
    return h


def spock_problem_info(problem):
    nz, ne = C.c_int64(), C.c_int64()
    nl, fs = C.c_double(), C.c_double()
    _check(_lib.spock_problem_info(problem, C.byref(nz), C.byref(ne), C.byref(nl), C.byref(fs)))
    return nz.value, ne.value, nl.value, fs.value


def spock_solve(problem, x0, settings, z, eta, warm):
    """Host buffers (float64 numpy arrays, modified in place)."""
    info = Info()
    x0, px = _dptr(x0)
    assert z.dtype == np.float64 and eta.dtype == np.float64 and z.flags.c_contiguous and eta.flags.c_contiguous
    rc = _lib.spock_solve(problem, px, C.byref(settings) if settings is not None else None,
                          z.ctypes.data_as(_D), eta.ctypes.data_as(_D), int(warm), C.byref(info))
    _check(rc, (SPOCK_OK, SPOCK_MAX_ITER))
    return info


def spock_solve_dev(problem, x0, settings, z, eta, warm, stream=None):
    import torch
    info = Info()
    rc = _lib.spock_solve_dev(problem, _tptr(x0, dtype=torch.float64), C.byref(settings) if settings is not None else None,
                              _tptr(z, dtype=torch.float64), _tptr(eta, dtype=torch.float64), int(warm),
                              C.byref(info), _stream(stream))
    _check(rc, (SPOCK_OK, SPOCK_MAX_ITER))
    return info


def spock_cp_step(problem, x0, k, alpha, precision, z, eta):
    x0, px = _dptr(x0)
    xi = C.c_double()
    _check(_lib.spock_cp_step(problem, px, int(k), float(alpha), int(precision), z.ctypes.data_as(_D),
                              eta.ctypes.data_as(_D), C.byref(xi)))
    return xi.value


def spock_cp_step_dev(problem, x0, k, alpha, precision, z, eta, stream=None):
    import torch
    xi = C.c_double()
    _check(_lib.spock_cp_step_dev(problem, _tptr(x0, dtype=torch.float64), int(k), float(alpha), int(precision),
                                  _tptr(z, dtype=torch.float64), _tptr(eta, dtype=torch.float64), C.byref(xi),
                                  _stream(stream)))
    return xi.value


def spock_apply_L_dev(problem, z, eta_out, stream=None):
    _check(_lib.spock_apply_L_dev(problem, _tptr(z), _tptr(eta_out), _stream(stream)))


def spock_apply_Lt_dev(problem, eta, z_out, stream=None):
    _check(_lib.spock_apply_Lt_dev(problem, _tptr(eta), _tptr(z_out), _stream(stream)))


def spock_prox_f_dev(problem, x0, alpha, z, z_out, stream=None):
    _check(_lib.spock_prox_f_dev(problem, _tptr(x0), float(alpha), _tptr(z), _tptr(z_out), _stream(stream)))


def spock_prox_f_noalloc_dev(problem, x0, alpha, z, z_out, stream=None):
    """prox_{alpha f} with the library's fixed device scratch (no allocation);
    see include/spock.h for the size limit and the sharing rules."""
    _check(_lib.spock_prox_f_noalloc_dev(problem, _tptr(x0), float(alpha), _tptr(z), _tptr(z_out),
                                         _stream(stream)))


def spock_prox_gconj_dev(problem, alpha, eta, eta_out, stream=None):
    _check(_lib.spock_prox_gconj_dev(problem, float(alpha), _tptr(eta), _tptr(eta_out), _stream(stream)))


def spock_T_dev(problem, x0, alpha, z, eta, z_out, eta_out, stream=None):
    _check(_lib.spock_T_dev(problem, _tptr(x0), float(alpha), _tptr(z), _tptr(eta), _tptr(z_out), _tptr(eta_out),
                            _stream(stream)))


def spock_grad_dev(problem, z, eta, precision, g_x0=None, g_A=None, g_B=None, g_Q=None, g_R=None, g_QN=None,
                   stream=None):
    """Gradient of the optimal cost from a converged (z, eta); outputs are
    float64 CUDA tensors (or None) in the caller's node numbering."""
    import torch
    ptr = lambda t: None if t is None else _tptr(t, dtype=torch.float64)
    _check(_lib.spock_grad_dev(problem, _tptr(z, dtype=torch.float64), _tptr(eta, dtype=torch.float64),
                               int(precision), ptr(g_x0), ptr(g_A), ptr(g_B), ptr(g_Q), ptr(g_R), ptr(g_QN),
                               _stream(stream)))


def spock_adjoint_dev(problem, z, eta, g_z=None, max_iter=20000, tol=1e-10, g_x0=None, g_A=None, g_B=None,
                      g_Q=None, g_R=None, g_QN=None, stream=None):
    """Gradient of <g_z, z*> (default: the optimal cost) by the adjoint of the
    CP fixed point; device float64 tensors.  Returns (status, iterations,
    final relative change of the adjoint)."""
    import torch
    ptr = lambda t: None if t is None else _tptr(t, dtype=torch.float64)
    its, res = C.c_int32(), C.c_double()
    rc = _lib.spock_adjoint_dev(problem, _tptr(z, dtype=torch.float64), _tptr(eta, dtype=torch.float64), ptr(g_z),
                                int(max_iter), float(tol), ptr(g_x0), ptr(g_A), ptr(g_B), ptr(g_Q), ptr(g_R),
                                ptr(g_QN), C.byref(its), C.byref(res), _stream(stream))
    _check(rc, (SPOCK_OK, SPOCK_MAX_ITER))
    return rc, its.value, res.value


def spock_grad(problem, z, eta, precision, g_x0=None, g_A=None, g_B=None, g_Q=None, g_R=None, g_QN=None):
    """Host-buffer gradient: z, eta and the outputs are float64 numpy arrays
    (outputs written in place, any may be None)."""
    def hp(a):
        if a is None:
            return None
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data_as(_D)
    z = np.ascontiguousarray(z, dtype=np.float64)
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    _check(_lib.spock_grad(problem, hp(z), hp(eta), int(precision), hp(g_x0), hp(g_A), hp(g_B), hp(g_Q), hp(g_R),
                           hp(g_QN)))


def spock_batch_create(problems):
    """problems: list of problem handles (c_void_p)."""
    arr = (_P * len(problems))(*[p.value if isinstance(p, _P) else p for p in problems])
    h = _P()
    _check(_lib.spock_batch_create(len(problems), arr, C.byref(h)))
    return h


def spock_batch_solve_dev(batch, x0s, settings, zs, etas, warm):
    """x0s, zs, etas: lists of float64 CUDA tensors, one per instance.
    Returns the list of per-instance Info."""
    import torch
    n = len(x0s)
    ptrs = lambda ts: (_P * n)(*[_tptr(t, dtype=torch.float64).value for t in ts])
    infos = (Info * n)()
    rc = _lib.spock_batch_solve_dev(batch, ptrs(x0s), C.byref(settings) if settings is not None else None,
                                    ptrs(zs), ptrs(etas), int(warm), infos)
    _check(rc, (SPOCK_OK, SPOCK_MAX_ITER))
    return list(infos)


def spock_batch_solve(batch, x0s, settings, zs, etas, warm):
    """Host buffers: x0s, zs, etas are lists of float64 numpy arrays (zs and
    etas modified in place).  Returns the list of per-instance Info."""
    n = len(x0s)
    x0s = [np.ascontiguousarray(a, dtype=np.float64) for a in x0s]
    for a in list(zs) + list(etas):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    ptrs = lambda arrs: (_D * n)(*[a.ctypes.data_as(_D) for a in arrs])
    infos = (Info * n)()
    rc = _lib.spock_batch_solve(batch, ptrs(x0s), C.byref(settings) if settings is not None else None,
                                ptrs(zs), ptrs(etas), int(warm), infos)
    _check(rc, (SPOCK_OK, SPOCK_MAX_ITER))
    return list(infos)


def spock_fp64_fma_rate(iters=20000, stream=None):
    """Measured FP64 FMA throughput of the current device in TFLOP/s."""
    v = C.c_double()
    _check(_lib.spock_fp64_fma_rate(int(iters), C.byref(v), _stream(stream)))
    return v.value


def spock_free(handle):
    _lib.spock_free(handle)


def spock_last_error():
    return _lib.spock_last_error().decode()


# ---------------------------------------------------------------------------
# convenience owner of a tree + problem pair
# ---------------------------------------------------------------------------

class Problem:
    """Tree and problem handles built from a workload dict (see
    ``workloads``); frees both on close / garbage collection."""

    def __init__(self, d):
        self.handle = None
        self.tree = spock_tree_create(d["anc"], d["prob"])
        try:
            self.handle = spock_problem_create(self.tree, d)
        except Exception:
            # free the tree once: close() / __del__ must not free it again (the
            # address may already belong to another handle by then)
            spock_free(self.tree)
            self.tree = None
            raise
        self.nx, self.nu = int(d["nx"]), int(d["nu"])
        self.n_nodes = len(d["anc"])
        self.n_z, self.n_eta, self.norm_L, self.factor_seconds = spock_problem_info(self.handle)

    @property
    def n_v(self):
        return self.n_z + self.n_eta

    def clone(self):
        """A problem sharing this one's data and factors on the device, with its
        own iterate and scratch buffers (spock_problem_clone)."""
        return _Clone(self)

    def close(self):
        if getattr(self, "handle", None):
            spock_free(self.handle)
            self.handle = None
        if getattr(self, "tree", None):
            spock_free(self.tree)
            self.tree = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Clone:
    """Owner of a spock_problem_clone handle; same attributes as Problem."""

    def __init__(self, base):
        self.handle = spock_problem_clone(base.handle)
        self.tree = None
        self.nx, self.nu, self.n_nodes = base.nx, base.nu, base.n_nodes
        self.n_z, self.n_eta, self.norm_L, self.factor_seconds = spock_problem_info(self.handle)

    @property
    def n_v(self):
        return self.n_z + self.n_eta

    def close(self):
        if getattr(self, "handle", None):
            spock_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
