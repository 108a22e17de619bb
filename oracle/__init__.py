"""CPU oracle for the mixed-precision one-sided Jacobi SVD (arXiv 2209.04626).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg are the only users. It shares no code with the GPU library (it is plain
C in ``mpjsvd_oracle.c``, loaded with ctypes) and never imports it.

All arrays are numpy float64, column-major (Fortran order), as the C code expects.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class Params(ctypes.Structure):
    _fields_ = [("tol_alg", ctypes.c_double), ("tol_orth", ctypes.c_double),
                ("tol_cond_coef", ctypes.c_double), ("trailing_frac", ctypes.c_double),
                ("tol", ctypes.c_double), ("maxsweep", ctypes.c_int), ("mode", ctypes.c_int),
                ("precond", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("branch", ctypes.c_int), ("sweeps_low", ctypes.c_int),
                ("sweeps_work", ctypes.c_int), ("rot_low", ctypes.c_longlong),
                ("rot_work", ctypes.c_longlong), ("cond_r", ctypes.c_double),
                ("orth", ctypes.c_double), ("switch_off", ctypes.c_double),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


MODE = {"auto": 0, "mixed": 1, "plain": 2}
PRECOND = {"rt": 0, "r": 1}
BRANCH = {0: "mixed", 1: "skip_cond", 2: "skip_trailing", 3: "skip_orth", 4: "plain"}

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_default_params.argtypes = [ctypes.POINTER(Params)]
        L.orc_house.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_geqrf.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp]
        L.orc_geqp3.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _ip, _dp]
        L.orc_apply_q.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                  ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.orc_apply_q.restype = None
        L.orc_jacobi.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_double, ctypes.c_int, _ip,
                                 ctypes.POINTER(ctypes.c_longlong)]
        L.orc_jacobi_f32.argtypes = [ctypes.c_int, ctypes.c_int, _fp, ctypes.c_int, ctypes.c_float,
                                     ctypes.c_int, _ip, ctypes.POINTER(ctypes.c_longlong)]
        L.orc_rot_tangent.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_rot_tangent.restype = ctypes.c_double
        L.orc_svd.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp,
                              ctypes.POINTER(Params), ctypes.POINTER(Stats)]
        L.orc_svd_backward.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp,
                                       _dp, ctypes.c_double, _ip]
        _lib = L
    return _lib


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a, kind=_dp):
    return a.ctypes.data_as(kind) if a is not None else None


def default_params(**kw):
    p = Params()
    lib().orc_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "mode" and isinstance(v, str):
            v = MODE[v]
        if k == "precond" and isinstance(v, str):
            v = PRECOND[v]
        setattr(p, k, v)
    return p


def house(x):
    """Householder reflector of x: returns (beta_and_vtail, tau)."""
    x = np.array(x, dtype=np.float64)
    tau = ctypes.c_double()
    lib().orc_house(len(x), _ptr(x), ctypes.byref(tau))
    return x, tau.value


def geqrf(A):
    A = _f64(A).copy(order="F")
    m, n = A.shape
    tau = np.zeros(max(1, min(m, n)))
    rc = lib().orc_geqrf(m, n, _ptr(A), max(1, m), _ptr(tau))
    assert rc == 0
    return A, tau[:min(m, n)]


def geqp3(A):
    A = _f64(A).copy(order="F")
    m, n = A.shape
    tau = np.zeros(max(1, min(m, n)))
    jpvt = np.zeros(max(1, n), dtype=np.int32)
    rc = lib().orc_geqp3(m, n, _ptr(A), max(1, m), _ptr(jpvt, _ip), _ptr(tau))
    assert rc == 0
    return A, jpvt[:n], tau[:min(m, n)]


def apply_q(QR, tau, C, trans=False):
    """Q C (or Q^T C) for Q stored as reflectors below the diagonal of QR."""
    QR = _f64(QR)
    C = _f64(C).copy(order="F")
    m, nc = C.shape
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    lib().orc_apply_q(int(trans), m, nc, len(tau), _ptr(QR), QR.shape[0], _ptr(tau), _ptr(C),
                      m)
    return C


def rot_tangent(alpha, beta, gamma):
    return lib().orc_rot_tangent(alpha, beta, gamma)


def jacobi(X, V=None, tol=None, maxsweep=30):
    """Alg. 1 (binary64) on a copy of X; returns (X_inf, V, sweeps, rotations, rc)."""
    X = _f64(X).copy(order="F")
    m, n = X.shape
    if V is not None:
        V = _f64(V).copy(order="F")
    tol = np.sqrt(m) * 2.0 ** -53 if tol is None else tol
    sw = ctypes.c_int()
    rot = ctypes.c_longlong()
    rc = lib().orc_jacobi(m, n, _ptr(X), m, _ptr(V), V.shape[0] if V is not None else 1,
                          V.shape[0] if V is not None else 0, tol, maxsweep, ctypes.byref(sw),
                          ctypes.byref(rot))
    return X, V, sw.value, rot.value, rc


def jacobi_f32(X, tol=None, maxsweep=30):
    """Alg. 1 in binary32 without V; returns (X_inf, sweeps, rotations, rc)."""
    X = np.asfortranarray(np.asarray(X, dtype=np.float32)).copy(order="F")
    m, n = X.shape
    tol = np.sqrt(m) * 2.0 ** -24 if tol is None else tol
    sw = ctypes.c_int()
    rot = ctypes.c_longlong()
    rc = lib().orc_jacobi_f32(m, n, _ptr(X, _fp), m, tol, maxsweep, ctypes.byref(sw),
                              ctypes.byref(rot))
    return X, sw.value, rot.value, rc


def svd(A, mode="auto", **kw):
    """Algorithm 4 (mode 'auto'), forced low-precision stage ('mixed') or Algorithm 2
    ('plain'). Returns (U, S, V, stats_dict)."""
    A = _f64(A)
    m, n = A.shape
    U = np.zeros((m, n), order="F")
    S = np.zeros(n)
    V = np.zeros((n, n), order="F")
    p = default_params(mode=mode, **kw)
    st = Stats()
    lib().orc_svd(m, n, _ptr(A), max(1, m), _ptr(U), _ptr(S), _ptr(V), ctypes.byref(p),
                  ctypes.byref(st))
    d = st.as_dict()
    d["branch_name"] = BRANCH.get(d["branch"], "?")
    return U, S, V, d


def svd_backward(U, S, V, gU=None, gS=None, gV=None, gap_tol=1e-3):
    """Adjoint of the thin SVD; returns (gA, n_flagged)."""
    U = _f64(U)
    V = _f64(V)
    S = np.ascontiguousarray(S, dtype=np.float64)
    m, n = U.shape
    gU = _f64(gU) if gU is not None else None
    gV = _f64(gV) if gV is not None else None
    gS = np.ascontiguousarray(gS, dtype=np.float64) if gS is not None else None
    gA = np.zeros((m, n), order="F")
    nf = ctypes.c_int()
    rc = lib().orc_svd_backward(m, n, _ptr(U), _ptr(S), _ptr(V), _ptr(gU), _ptr(gS), _ptr(gV),
                                _ptr(gA), gap_tol, ctypes.byref(nf))
    assert rc == 0
    return gA, nf.value
