"""Thin ctypes binding of ``libncl_kkt.so`` (the C ABI of include/ncl_kkt.h).

Argument marshalling only: every step of factor / solve / adjoint runs in the
library's CUDA kernels.  Device arrays are torch CUDA tensors (FP64); pattern
arrays are numpy int32.  If the library cannot be built or loaded the
functions raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

STABILIZED, CONDENSED = 0, 1
PREC_FP64, PREC_FP32_IR = 0, 1
PIVOT_PERTURB, PIVOT_STOP = 0, 1

STATUS = ["NCL_OK", "NCL_ERR_INVALID_ARG", "NCL_ERR_PATTERN", "NCL_ERR_OOM", "NCL_ERR_CUDA",
          "NCL_ERR_STATE", "NCL_ERR_ZERO_PIVOT", "NCL_ERR_NUMERIC", "NCL_ERR_IR_NOT_CONVERGED",
          "NCL_ERR_TIMEOUT", "NCL_ERR_INERTIA"]
OK, ERR_IR_NOT_CONVERGED, ERR_ZERO_PIVOT, ERR_INERTIA = 0, 8, 6, 10


class Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("pivot_policy", ctypes.c_int32),
                ("pivot_eps", ctypes.c_double), ("ir_tol", ctypes.c_double),
                ("ir_max_iter", ctypes.c_int32), ("use_fgmres", ctypes.c_int32),
                ("use_tensor_cores", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("host_only", ctypes.c_int32), ("precision_fallback", ctypes.c_int32),
                ("max_device_bytes", ctypes.c_int64), ("wait_cycles", ctypes.c_int64),
                ("persistent_fronts", ctypes.c_int32), ("ir_switch", ctypes.c_double),
                ("subtree_sweeps", ctypes.c_int32), ("tc_min_pivots", ctypes.c_int32),
                ("autotune_path", ctypes.c_char_p)]


class FactorInfo(ctypes.Structure):
    _fields_ = [("n_pos", ctypes.c_int64), ("n_neg", ctypes.c_int64), ("n_zero", ctypes.c_int64),
                ("n_perturbed", ctypes.c_int64), ("nnz_L", ctypes.c_int64),
                ("flops", ctypes.c_double), ("ms", ctypes.c_float), ("fp64_fallback", ctypes.c_int32)]

    @property
    def inertia(self):
        return (self.n_pos, self.n_neg, self.n_zero)

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveInfo(ctypes.Structure):
    _fields_ = [("ir_iters", ctypes.c_int32), ("used_fgmres", ctypes.c_int32),
                ("backward_err", ctypes.c_double), ("ms", ctypes.c_float), ("fp64_fallback", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AnalysisInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int64), ("nnz_A", ctypes.c_int64), ("nnz_L", ctypes.c_int64),
                ("nnz_L_stored", ctypes.c_int64), ("update_entries", ctypes.c_int64),
                ("n_supernodes", ctypes.c_int64), ("n_levels", ctypes.c_int64),
                ("max_front", ctypes.c_int64), ("max_pivots", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("flops", ctypes.c_double),
                ("analyze_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NewtonPoint(ctypes.Structure):
    """Device pointers of a Newton point (ncl_kkt_newton_point)."""
    _fields_ = [(k, ctypes.c_void_p) for k in ("grad_phi", "x", "lower", "upper", "z_lower", "z_upper",
                                               "c", "y", "y_k", "r")]


class NclError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS[status] if 0 <= status < len(STATUS) else status}: {msg}")
        self.status = status


_lib = None
P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
D = ctypes.c_double

_SIGS = {
    "ncl_kkt_default_options": (None, [ctypes.POINTER(Options)]),
    "ncl_kkt_analyze": (I32, [I32, I32, I32, P, P, P, P, ctypes.POINTER(Options), ctypes.POINTER(P)]),
    "ncl_kkt_batch_analyze": (I32, [I32, I32, P, P, P, P, P, P, ctypes.POINTER(Options), ctypes.POINTER(P)]),
    "ncl_kkt_analyze_like": (I32, [P, ctypes.POINTER(Options), ctypes.POINTER(P)]),
    "ncl_kkt_factor": (I32, [P, P, P, P, D, D, P, ctypes.POINTER(FactorInfo)]),
    "ncl_kkt_batch_factor": (I32, [P, P, P, P, P, P, P, P]),
    "ncl_kkt_factor_regularize": (I32, [P, P, P, P, P, P, D, D, I32, P, P, P]),
    "ncl_kkt_factor_k1s": (I32, [P, P, P, P, P, P, P, P, P]),
    "ncl_kkt_k1s_slack_step": (I32, [P, I32, P, I64, P, I64, P, I64, P]),
    "ncl_kkt_k1s_rhs": (I32, [P, I32, P, I64, P, I64, P, I64, P]),
    "ncl_kkt_newton_rhs": (I32, [P, ctypes.POINTER(NewtonPoint), P, P, P]),
    "ncl_kkt_newton_recover": (I32, [P, ctypes.POINTER(NewtonPoint), P, P, P, P, P, P, P, P]),
    "ncl_kkt_solve": (I32, [P, I32, P, I64, P, I64, P, ctypes.POINTER(SolveInfo)]),
    "ncl_kkt_solve_noalloc": (I32, [P, I32, P, I64, P, I64, P, ctypes.POINTER(SolveInfo)]),
    "ncl_kkt_batch_factor_solve": (I32, [P, P, P, P, P, P, I32, P, I64, P, I64, P, P,
                                         ctypes.POINTER(SolveInfo)]),
    "ncl_kkt_adjoint": (I32, [P, I32, P, I64, P, I64, P, I64, P, P, P, P, P, ctypes.POINTER(SolveInfo)]),
    "ncl_kkt_get_analysis_info": (I32, [P, ctypes.POINTER(AnalysisInfo)]),
    "ncl_kkt_get_options": (I32, [P, ctypes.POINTER(Options)]),
    "ncl_kkt_get_permutation": (I32, [P, P]),
    "ncl_kkt_get_supernodes": (I32, [P, P, P, P]),
    "ncl_kkt_instance_count": (I32, [P]),
    "ncl_kkt_kernel_launches": (I64, []),
    "ncl_kkt_selftest_tensor_update": (I32, [I32, I32, I32, P, P, I32, I32, I32, I32, P, I32, P]),
    "ncl_kkt_selftest_wait_timeout": (I32, [P, I32, I64, P]),
    "ncl_kkt_profile": (I32, [P, I32]),
    "ncl_kkt_profile_report": (I32, [P, ctypes.c_char_p, I64]),
    "ncl_kkt_destroy": (None, [P]),
    "ncl_kkt_status_string": (ctypes.c_char_p, [I32]),
    "ncl_kkt_last_error": (ctypes.c_char_p, []),
}

EXPORTED = tuple(_SIGS)


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libncl_kkt.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libncl_kkt.so is not built")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st):
    if st != OK:
        raise NclError(st, _lib.ncl_kkt_last_error().decode())
    return st


def _ptr(t):
    """Device (or host numpy) pointer of a tensor/array, None for None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def default_options(**kw) -> Options:
    lib = load()
    o = Options()
    lib.ncl_kkt_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "prec" and isinstance(v, str):
            v = {"fp64": PREC_FP64, "fp32_ir": PREC_FP32_IR}[v]
        if k == "autotune_path":
            setattr(o, k, os.fsencode(v))
            continue
        setattr(o, k, int(v) if isinstance(getattr(o, k), int) else float(v))
    return o


def ncl_kkt_get_options(h) -> Options:
    o = Options()
    _check(load().ncl_kkt_get_options(h, ctypes.byref(o)))
    return o


# ---------------------------------------------------------------------------
# C-named functions (argument marshalling only)
# ---------------------------------------------------------------------------

def ncl_kkt_analyze(form, n, m, H_rowptr, H_colind, J_rowptr, J_colind, opt: Options | None = None):
    lib = load()
    arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in (H_rowptr, H_colind, J_rowptr, J_colind)]
    h = P()
    _check(lib.ncl_kkt_analyze(form, n, m, *(a.ctypes.data for a in arrs),
                               ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    return h


def ncl_kkt_batch_analyze(form, ns, ms, H_rowptrs, H_colinds, J_rowptrs, J_colinds, opt: Options | None = None):
    lib = load()
    count = len(ns)
    keep = []

    def ptrs(lst):
        arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in lst]
        keep.extend(arrs)
        return (P * count)(*[a.ctypes.data for a in arrs])
    n = np.ascontiguousarray(ns, dtype=np.int32)
    m = np.ascontiguousarray(ms, dtype=np.int32)
    pH, pHi, pJ, pJi = ptrs(H_rowptrs), ptrs(H_colinds), ptrs(J_rowptrs), ptrs(J_colinds)
    h = P()
    _check(lib.ncl_kkt_batch_analyze(count, form, n.ctypes.data, m.ctypes.data, ctypes.cast(pH, P),
                                     ctypes.cast(pHi, P), ctypes.cast(pJ, P), ctypes.cast(pJi, P),
                                     ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    return h


def ncl_kkt_analyze_like(src, opt: Options | None = None):
    out = P()
    _check(load().ncl_kkt_analyze_like(src, ctypes.byref(opt or default_options()), ctypes.byref(out)))
    return out


def ncl_kkt_factor(h, H_val, J_val, Sigma, delta, rho, stream=None) -> FactorInfo:
    info = FactorInfo()
    st = load().ncl_kkt_factor(h, _ptr(H_val), _ptr(J_val), _ptr(Sigma), float(delta), float(rho),
                               _stream_ptr(stream), ctypes.byref(info))
    if st not in (OK, ERR_ZERO_PIVOT):
        _check(st)
    info.status = st
    return info


def ncl_kkt_batch_factor(h, H_val, J_val, Sigma, delta, rho, stream=None):
    lib = load()
    count = lib.ncl_kkt_instance_count(h)
    infos = (FactorInfo * count)()
    dl = np.ascontiguousarray(delta, dtype=np.float64)
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    st = lib.ncl_kkt_batch_factor(h, _ptr(H_val), _ptr(J_val), _ptr(Sigma), dl.ctypes.data, rh.ctypes.data,
                                  _stream_ptr(stream), ctypes.cast(infos, P))
    if st not in (OK, ERR_ZERO_PIVOT):
        _check(st)
    return list(infos), st


def ncl_kkt_factor_regularize(h, H_val, J_val, Sigma, delta, rho, delta_first=1e-4, growth=10.0, max_tries=20,
                              stream=None, raise_on_inertia=True):
    """Inertia correction (Section 3.1): returns (infos, delta per instance,
    tries, status).  rho is the unregularised penalty; the matrix uses
    rho + delta.  With raise_on_inertia=False an NCL_ERR_INERTIA outcome is
    returned in the status instead of raised."""
    lib = load()
    count = lib.ncl_kkt_instance_count(h)
    infos = (FactorInfo * count)()
    dl = np.array(np.broadcast_to(np.asarray(delta, dtype=np.float64), (count,)))
    rh = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, dtype=np.float64), (count,)))
    tries = ctypes.c_int32(0)
    st = lib.ncl_kkt_factor_regularize(h, _ptr(H_val), _ptr(J_val), _ptr(Sigma), dl.ctypes.data, rh.ctypes.data,
                                       float(delta_first), float(growth), int(max_tries), _stream_ptr(stream),
                                       ctypes.cast(infos, P), ctypes.byref(tries))
    if st not in (OK, ERR_ZERO_PIVOT) and not (st == ERR_INERTIA and not raise_on_inertia):
        _check(st)
    return list(infos), dl, int(tries.value), st


def ncl_kkt_factor_k1s(h, H_val, J_val, Sigma, Sigma_s, delta, rho, stream=None):
    """Condensed factorisation with slacks (Eq. K1s); Sigma_s: device float64
    per constraint row, +inf for a row without slack.  Returns (infos, status)."""
    lib = load()
    count = lib.ncl_kkt_instance_count(h)
    infos = (FactorInfo * count)()
    dl = np.ascontiguousarray(np.broadcast_to(np.asarray(delta, dtype=np.float64), (count,)))
    rh = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, dtype=np.float64), (count,)))
    st = lib.ncl_kkt_factor_k1s(h, _ptr(H_val), _ptr(J_val), _ptr(Sigma), _ptr(Sigma_s), dl.ctypes.data,
                                rh.ctypes.data, _stream_ptr(stream), ctypes.cast(infos, P))
    if st not in (OK, ERR_ZERO_PIVOT):
        _check(st)
    return list(infos), st


def _newton_point(pt: dict) -> NewtonPoint:
    return NewtonPoint(*[_ptr(pt[k]) if pt.get(k) is not None else None for k, _ in NewtonPoint._fields_])


def ncl_kkt_newton_rhs(h, pt: dict, mu, B, stream=None):
    count = load().ncl_kkt_instance_count(h)
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(mu, dtype=np.float64), (count,)))
    np_ = _newton_point(pt)
    _check(load().ncl_kkt_newton_rhs(h, ctypes.byref(np_), m.ctypes.data, _ptr(B), _stream_ptr(stream)))


def ncl_kkt_newton_recover(h, pt: dict, mu, X, dx=None, dy=None, dr=None, dzl=None, dzu=None, stream=None):
    count = load().ncl_kkt_instance_count(h)
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(mu, dtype=np.float64), (count,)))
    np_ = _newton_point(pt)
    _check(load().ncl_kkt_newton_recover(h, ctypes.byref(np_), m.ctypes.data, _ptr(X), _ptr(dx), _ptr(dy),
                                         _ptr(dr), _ptr(dzl), _ptr(dzu), _stream_ptr(stream)))


def ncl_kkt_k1s_rhs(h, nrhs, RT, ldt, RS, ldr, OUT, ldo, stream=None):
    _check(load().ncl_kkt_k1s_rhs(h, nrhs, _ptr(RT), ldt, _ptr(RS), ldr, _ptr(OUT), ldo, _stream_ptr(stream)))


def ncl_kkt_k1s_slack_step(h, nrhs, DT, ldt, RS, ldr, DS, lds, stream=None):
    _check(load().ncl_kkt_k1s_slack_step(h, nrhs, _ptr(DT), ldt, _ptr(RS), ldr, _ptr(DS), lds,
                                         _stream_ptr(stream)))


def ncl_kkt_solve(h, nrhs, B, ldb, X, ldx, stream=None):
    info = SolveInfo()
    st = load().ncl_kkt_solve(h, nrhs, _ptr(B), ldb, _ptr(X), ldx, _stream_ptr(stream), ctypes.byref(info))
    if st not in (OK, ERR_IR_NOT_CONVERGED):
        _check(st)
    info.status = st
    return info


def ncl_kkt_solve_noalloc(h, nrhs, B, ldb, X, ldx, stream=None):
    """ncl_kkt_solve on the library's fixed static workspace (no device
    allocation in the call)."""
    info = SolveInfo()
    st = load().ncl_kkt_solve_noalloc(h, nrhs, _ptr(B), ldb, _ptr(X), ldx, _stream_ptr(stream), ctypes.byref(info))
    if st not in (OK, ERR_IR_NOT_CONVERGED):
        _check(st)
    info.status = st
    return info


def ncl_kkt_batch_factor_solve(h, H_val, J_val, Sigma, delta, rho, nrhs, B, ldb, X, ldx, stream=None):
    lib = load()
    count = lib.ncl_kkt_instance_count(h)
    infos = (FactorInfo * count)()
    sinfo = SolveInfo()
    dl = np.ascontiguousarray(delta, dtype=np.float64)
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    st = lib.ncl_kkt_batch_factor_solve(h, _ptr(H_val), _ptr(J_val), _ptr(Sigma), dl.ctypes.data,
                                        rh.ctypes.data, nrhs, _ptr(B), ldb, _ptr(X), ldx,
                                        _stream_ptr(stream), ctypes.cast(infos, P), ctypes.byref(sinfo))
    if st not in (OK, ERR_IR_NOT_CONVERGED, ERR_ZERO_PIVOT):
        _check(st)
    sinfo.status = st
    return list(infos), sinfo


def ncl_kkt_adjoint(h, nrhs, X, ldx, GX, ldgx, GB, ldgb, G_H, G_J, G_S, G_scal, stream=None):
    info = SolveInfo()
    st = load().ncl_kkt_adjoint(h, nrhs, _ptr(X), ldx, _ptr(GX), ldgx, _ptr(GB), ldgb, _ptr(G_H), _ptr(G_J),
                                _ptr(G_S), _ptr(G_scal), _stream_ptr(stream), ctypes.byref(info))
    if st not in (OK, ERR_IR_NOT_CONVERGED):
        _check(st)
    info.status = st
    return info


def ncl_kkt_get_analysis_info(h) -> AnalysisInfo:
    info = AnalysisInfo()
    _check(load().ncl_kkt_get_analysis_info(h, ctypes.byref(info)))
    return info


def ncl_kkt_get_permutation(h, dim) -> np.ndarray:
    perm = np.empty(dim, np.int32)
    _check(load().ncl_kkt_get_permutation(h, perm.ctypes.data))
    return perm


def ncl_kkt_get_supernodes(h, ns):
    col0 = np.empty(ns + 1, np.int32)
    parent = np.empty(ns, np.int32)
    nrow = np.empty(ns, np.int32)
    _check(load().ncl_kkt_get_supernodes(h, col0.ctypes.data, parent.ctypes.data, nrow.ctypes.data))
    return col0, parent, nrow


def ncl_kkt_selftest_tensor_update(L, d, K, row_a, row_b, M, N, C, stream=None):
    """C (M x ldc float32 CUDA) -= L[row_a:row_a+M, :K] diag(d) L[row_b:row_b+N, :K]^T, lower part,
    on the tensor-core kernel.  L: (rows, ld) float32 CUDA tensor."""
    rows, ld = L.shape
    _check(load().ncl_kkt_selftest_tensor_update(rows, ld, K, _ptr(L), _ptr(d), row_a, row_b, M, N, _ptr(C),
                                                 C.shape[1], _stream_ptr(stream)))


def ncl_kkt_selftest_wait_timeout(h, which, wait_cycles, stream=None) -> int:
    """Status of the self-test (NCL_ERR_TIMEOUT = 9 expected); other errors raise."""
    st = load().ncl_kkt_selftest_wait_timeout(h, int(which), int(wait_cycles), _stream_ptr(stream))
    if st not in (OK, 9):
        _check(st)
    return st


def ncl_kkt_kernel_launches() -> int:
    return int(load().ncl_kkt_kernel_launches())


def ncl_kkt_profile(h, enable: int):
    _check(load().ncl_kkt_profile(h, int(enable)))


def ncl_kkt_profile_report(h) -> dict:
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().ncl_kkt_profile_report(h, buf, len(buf)))
    return json.loads(buf.value.decode())


def ncl_kkt_destroy(h):
    if h:
        load().ncl_kkt_destroy(h)


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

class KKT:
    """One analysed pattern (or a batch of them) and its current factors.

    ``KKT(form, n, m, H_rowptr, H_colind, J_rowptr, J_colind, prec="fp32_ir")``
    or ``KKT.batch(form, [(n, m, Hp, Hi, Jp, Ji), ...])``.
    """

    def __init__(self, form, n, m, H_rowptr, H_colind, J_rowptr, J_colind, **opts):
        self._h = None
        self.opt = default_options(**opts)
        self._h = ncl_kkt_analyze(form, n, m, H_rowptr, H_colind, J_rowptr, J_colind, self.opt)
        self.form, self.count = form, 1
        self.nnz_H = int(np.asarray(H_rowptr)[-1]) if n > 0 else 0
        self.nnz_J = int(np.asarray(J_rowptr)[-1]) if m > 0 else 0
        self.n_var = int(n)
        self._post()

    @classmethod
    def batch(cls, form, patterns, **opts):
        self = cls.__new__(cls)
        self._h = None
        self.opt = default_options(**opts)
        ns = [p[0] for p in patterns]
        ms = [p[1] for p in patterns]
        self._h = ncl_kkt_batch_analyze(form, ns, ms, [p[2] for p in patterns], [p[3] for p in patterns],
                                        [p[4] for p in patterns], [p[5] for p in patterns], self.opt)
        self.form, self.count = form, len(patterns)
        self.nnz_H = sum(int(np.asarray(p[2])[-1]) if p[0] > 0 else 0 for p in patterns)
        self.nnz_J = sum(int(np.asarray(p[4])[-1]) if p[1] > 0 else 0 for p in patterns)
        self.n_var = sum(int(p[0]) for p in patterns)
        self._post()
        return self

    @classmethod
    def like(cls, other, **opts):
        """A handle with new options (e.g. prec="fp64") on the analysis of
        ``other`` (copied, not recomputed)."""
        self = cls.__new__(cls)
        self._h = None
        self.opt = default_options(**opts)
        self._h = ncl_kkt_analyze_like(other._h, self.opt)
        self.form, self.count = other.form, other.count
        self.nnz_H, self.nnz_J, self.n_var = other.nnz_H, other.nnz_J, other.n_var
        self._post()
        return self

    def _post(self):
        self.analysis = ncl_kkt_get_analysis_info(self._h)
        self.dim = int(self.analysis.dim)
        self.generation = 0     # incremented by every factor call

    @property
    def permutation(self) -> np.ndarray:
        return ncl_kkt_get_permutation(self._h, self.dim)

    def supernodes(self):
        return ncl_kkt_get_supernodes(self._h, int(self.analysis.n_supernodes))

    def factor(self, H_val, J_val, Sigma, delta, rho, stream=None):
        self.generation += 1
        if self.count == 1:
            return ncl_kkt_factor(self._h, H_val, J_val, Sigma, delta, rho, stream)
        return ncl_kkt_batch_factor(self._h, H_val, J_val, Sigma, delta, rho, stream)[0]

    def factor_regularized(self, H_val, J_val, Sigma, delta, rho, delta_first=1e-4, growth=10.0, max_tries=20,
                           stream=None, raise_on_inertia=True):
        """Inertia-corrected factorisation (Section 3.1); see
        ncl_kkt_factor_regularize.  Returns (infos, delta, tries, status)."""
        self.generation += 1
        return ncl_kkt_factor_regularize(self._h, H_val, J_val, Sigma, delta, rho, delta_first, growth, max_tries,
                                         stream, raise_on_inertia)

    def factor_k1s(self, H_val, J_val, Sigma, Sigma_s, delta, rho, stream=None):
        """Condensed factorisation with slacks (Eq. K1s); see ncl_kkt_factor_k1s."""
        self.generation += 1
        infos, _ = ncl_kkt_factor_k1s(self._h, H_val, J_val, Sigma, Sigma_s, delta, rho, stream)
        return infos[0] if self.count == 1 else infos

    def newton_rhs(self, pt: dict, mu, stream=None):
        """Right-hand side of Eq. K2r / K1 at the Newton point ``pt`` (dict of
        float64 CUDA tensors: grad_phi, x, lower, upper, z_lower, z_upper, c,
        y, y_k, r)."""
        import torch
        B = torch.empty(self.dim, dtype=torch.float64, device=pt["x"].device)
        ncl_kkt_newton_rhs(self._h, pt, mu, B, stream)
        return B

    def newton_recover(self, pt: dict, mu, X, stream=None):
        """The Newton direction (dx, dy, dr, dz_lower, dz_upper) from the
        solution X of the system newton_rhs set up."""
        import torch
        dev = pt["x"].device
        n, m = int(pt["x"].numel()), int(pt["c"].numel()) if pt.get("c") is not None else 0
        out = {k: torch.empty(sz, dtype=torch.float64, device=dev)
               for k, sz in (("dx", n), ("dy", m), ("dr", m), ("dz_lower", n), ("dz_upper", n))}
        ncl_kkt_newton_recover(self._h, pt, mu, X.contiguous(), out["dx"], out["dy"], out["dr"], out["dz_lower"],
                               out["dz_upper"], stream)
        return out

    def k1s_rhs(self, RT, RS, stream=None):
        """r_t + rho J_I^T (Sigma_s + rho I)^{-1} r_s for the current K1s
        factorisation; RT (dim,) or (dim, nrhs), RS (m,) or (m, nrhs)."""
        import torch
        one = RT.dim() == 1
        Tc = RT.reshape(self.dim, -1).t().contiguous()
        nrhs = Tc.shape[0]
        ncon = RS.shape[0]
        Rc = RS.reshape(ncon, -1).t().contiguous()
        Oc = torch.empty_like(Tc)
        ncl_kkt_k1s_rhs(self._h, nrhs, Tc, self.dim, Rc, max(ncon, 1), Oc, self.dim, stream)
        return Oc.t()[:, 0] if one else Oc.t()

    def slack_step(self, DT, RS, stream=None):
        """Delta s of Eq. K1s from Delta t (dim,) or (dim, nrhs) and r_s (m,) or
        (m, nrhs), float64 CUDA tensors."""
        import torch
        one = DT.dim() == 1
        Tc = DT.reshape(self.dim, -1).t().contiguous()
        nrhs = Tc.shape[0]
        ncon = RS.shape[0]
        Rc = RS.reshape(ncon, -1).t().contiguous()
        Dc = torch.empty_like(Rc)
        ncl_kkt_k1s_slack_step(self._h, nrhs, Tc, self.dim, Rc, max(ncon, 1), Dc, max(ncon, 1), stream)
        return Dc.t()[:, 0] if one else Dc.t()

    def solve(self, B, X=None, stream=None):
        """B: (dim,) or (dim, nrhs) float64 CUDA tensor.  Returns (X, info)."""
        import torch
        one = B.dim() == 1
        Bc = B.reshape(self.dim, -1).t().contiguous()       # (nrhs, dim) = column-major (dim, nrhs)
        nrhs = Bc.shape[0]
        Xc = torch.empty_like(Bc)
        info = ncl_kkt_solve(self._h, nrhs, Bc, self.dim, Xc, self.dim, stream)
        Xo = Xc.t()
        if X is not None:
            X.copy_(Xo.reshape(X.shape))
            Xo = X
        return (Xo[:, 0] if one else Xo), info

    def adjoint(self, X, GX, stream=None, want=("b", "H", "J", "Sigma", "scal"), nnz_H=None, nnz_J=None,
                n_var=None):
        """Gradients of l(X) given GX = dl/dX (same shape as X)."""
        import torch
        nnz_H = self.nnz_H if nnz_H is None else nnz_H
        nnz_J = self.nnz_J if nnz_J is None else nnz_J
        n_var = self.n_var if n_var is None else n_var
        one = X.dim() == 1
        Xc = X.reshape(self.dim, -1).t().contiguous()
        GXc = GX.reshape(self.dim, -1).t().contiguous()
        nrhs = Xc.shape[0]
        dev = X.device
        f64 = torch.float64
        GB = torch.empty_like(Xc) if "b" in want else None
        G_H = torch.empty(nnz_H, dtype=f64, device=dev) if ("H" in want and nnz_H is not None) else None
        G_J = torch.empty(nnz_J, dtype=f64, device=dev) if ("J" in want and nnz_J is not None) else None
        G_S = torch.empty(n_var, dtype=f64, device=dev) if ("Sigma" in want and n_var is not None) else None
        G_sc = torch.empty(2 * self.count, dtype=f64, device=dev) if "scal" in want else None
        info = ncl_kkt_adjoint(self._h, nrhs, Xc, self.dim, GXc, self.dim, GB, self.dim, G_H, G_J, G_S, G_sc,
                               stream)
        out = {"info": info}
        if GB is not None:
            out["b"] = GB.t()[:, 0] if one else GB.t()
        out["H"], out["J"], out["Sigma"], out["scal"] = G_H, G_J, G_S, G_sc
        return out

    def close(self):
        if getattr(self, "_h", None):
            ncl_kkt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
