"""CPU oracle for the mixed-precision one-sided Jacobi SVD (arXiv 2209.04626).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg are the only users. It shares no code with the GPU library (it is plain
C in ``mpjsvd_oracle.c``, loaded with ctypes) and never imports it.

Two builds of the same C source: the binary64 oracle (the method's working precision;
default) and, with ``ext=True``, a long double build (x86-64: 64-bit significand,
aarch64: IEEE binary128) used as an extended-precision reference to attribute rounding
error. Arrays are numpy column-major (Fortran order): float64, or longdouble for ext.
"""
import ctypes

import numpy as np

from . import build as _build

MODE = {"auto": 0, "mixed": 1, "plain": 2}
PRECOND = {"rt": 0, "r": 1, "l": 2, "auto": 3}
BRANCH = {0: "mixed", 1: "skip_cond", 2: "skip_trailing", 3: "skip_orth", 4: "plain"}

_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)


class _Variant:
    def __init__(self, path, creal, npreal):
        self.creal = creal
        self.np = npreal
        rp = ctypes.POINTER(creal)
        self.rp = rp

        class Params(ctypes.Structure):
            _fields_ = [("tol_alg", creal), ("tol_orth", creal), ("tol_cond_coef", creal),
                        ("trailing_frac", creal), ("tol", creal), ("maxsweep", ctypes.c_int),
                        ("mode", ctypes.c_int), ("precond", ctypes.c_int), ("qrcp", ctypes.c_int),
                        ("switch_method", ctypes.c_int), ("v_by_qr", ctypes.c_int), ("stop", ctypes.c_int),
                        ("y_tol", creal)]

        class Stats(ctypes.Structure):
            _fields_ = [("branch", ctypes.c_int), ("sweeps_low", ctypes.c_int),
                        ("sweeps_work", ctypes.c_int), ("rot_low", ctypes.c_longlong),
                        ("rot_work", ctypes.c_longlong), ("cond_r", creal), ("orth", creal),
                        ("switch_off", creal), ("status", ctypes.c_int), ("precond", ctypes.c_int),
                        ("sweeps_v", ctypes.c_int), ("y2_cols", ctypes.c_int)]

            def as_dict(self):
                d = {name: getattr(self, name) for name, _ in self._fields_}
                for k in ("cond_r", "orth", "switch_off"):
                    d[k] = float(d[k])
                return d

        self.Params, self.Stats = Params, Stats
        L = ctypes.CDLL(path)
        L.orc_default_params.argtypes = [ctypes.POINTER(Params)]
        L.orc_house.argtypes = [ctypes.c_int, rp, rp]
        L.orc_geqrf.argtypes = [ctypes.c_int, ctypes.c_int, rp, ctypes.c_int, rp]
        L.orc_geqp3.argtypes = [ctypes.c_int, ctypes.c_int, rp, ctypes.c_int, _ip, rp]
        L.orc_geqp3_mixed.argtypes = [ctypes.c_int, ctypes.c_int, rp, ctypes.c_int, _ip, rp]
        L.orc_qrcp_pivots_f32.argtypes = [ctypes.c_int, ctypes.c_int, rp, ctypes.c_int, _ip]
        L.orc_apply_q.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, rp,
                                  ctypes.c_int, rp, rp, ctypes.c_int]
        L.orc_apply_q.restype = None
        L.orc_jacobi.argtypes = [ctypes.c_int, ctypes.c_int, rp, ctypes.c_int, rp, ctypes.c_int,
                                 ctypes.c_int, creal, ctypes.c_int, ctypes.c_int, _ip,
                                 ctypes.POINTER(ctypes.c_longlong)]
        L.orc_jacobi_derijk.argtypes = [ctypes.c_int, ctypes.c_int, rp, ctypes.c_int, rp, ctypes.c_int,
                                        ctypes.c_int, creal, ctypes.c_int, ctypes.c_int, _ip, _ip,
                                        ctypes.POINTER(ctypes.c_longlong)]
        L.orc_jacobi_f32.argtypes = [ctypes.c_int, ctypes.c_int, _fp, ctypes.c_int, _fp, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int, _ip,
                                     ctypes.POINTER(ctypes.c_longlong)]
        L.orc_rot_tangent.argtypes = [creal, creal, creal]
        L.orc_rot_tangent.restype = creal
        L.orc_svd.argtypes = [ctypes.c_int, ctypes.c_int, rp, ctypes.c_int, rp, rp, rp,
                              ctypes.POINTER(Params), ctypes.POINTER(Stats)]
        L.orc_svd_backward.argtypes = [ctypes.c_int, ctypes.c_int, rp, rp, rp, rp, rp, rp, rp,
                                       creal, _ip]
        self.L = L

    def arr(self, a):
        return np.asfortranarray(np.asarray(a, dtype=self.np))

    def ptr(self, a):
        return a.ctypes.data_as(self.rp) if a is not None else None


_variants = {}


def _v(ext=False):
    key = bool(ext)
    if key not in _variants:
        _build.build()
        if key:
            _variants[key] = _Variant(_build.OUT_EXT, ctypes.c_longdouble, np.longdouble)
        else:
            _variants[key] = _Variant(_build.OUT, ctypes.c_double, np.float64)
    return _variants[key]


def lib(ext=False):
    return _v(ext).L


def unit_roundoff(ext=False):
    return float(np.finfo(np.longdouble).eps) / 2 if ext else 2.0 ** -53


def default_params(ext=False, **kw):
    v = _v(ext)
    p = v.Params()
    v.L.orc_default_params(ctypes.byref(p))
    for k, val in kw.items():
        if k == "mode" and isinstance(val, str):
            val = MODE[val]
        if k == "precond" and isinstance(val, str):
            val = PRECOND[val]
        setattr(p, k, val)
    return p


def house(x, ext=False):
    """Householder reflector of x: returns (beta_and_vtail, tau)."""
    v = _v(ext)
    x = np.array(x, dtype=v.np)
    tau = v.creal()
    v.L.orc_house(len(x), v.ptr(x), ctypes.byref(tau))
    return x, tau.value


def geqrf(A, ext=False):
    v = _v(ext)
    A = v.arr(A).copy(order="F")
    m, n = A.shape
    tau = np.zeros(max(1, min(m, n)), dtype=v.np)
    rc = v.L.orc_geqrf(m, n, v.ptr(A), max(1, m), v.ptr(tau))
    assert rc == 0
    return A, tau[:min(m, n)]


def geqp3(A, ext=False):
    v = _v(ext)
    A = v.arr(A).copy(order="F")
    m, n = A.shape
    tau = np.zeros(max(1, min(m, n)), dtype=v.np)
    jpvt = np.zeros(max(1, n), dtype=np.int32)
    rc = v.L.orc_geqp3(m, n, v.ptr(A), max(1, m), jpvt.ctypes.data_as(_ip), v.ptr(tau))
    assert rc == 0
    return A, jpvt[:n], tau[:min(m, n)]


def geqp3_mixed(A, ext=False):
    """Alg. 5: binary32 pivot search on lower(A), then the QR of A P in working precision.
    Returns (QR of A P in geqrf layout, jpvt, tau)."""
    v = _v(ext)
    A = v.arr(A).copy(order="F")
    m, n = A.shape
    tau = np.zeros(max(1, min(m, n)), dtype=v.np)
    jpvt = np.zeros(max(1, n), dtype=np.int32)
    rc = v.L.orc_geqp3_mixed(m, n, v.ptr(A), max(1, m), jpvt.ctypes.data_as(_ip), v.ptr(tau))
    assert rc == 0
    return A, jpvt[:n], tau[:min(m, n)]


def qrcp_pivots_f32(A, ext=False):
    """The binary32 column permutation of Alg. 5 (step 2) for A."""
    v = _v(ext)
    A = v.arr(A).copy(order="F")
    m, n = A.shape
    jpvt = np.zeros(max(1, n), dtype=np.int32)
    rc = v.L.orc_qrcp_pivots_f32(m, n, v.ptr(A), max(1, m), jpvt.ctypes.data_as(_ip))
    assert rc == 0
    return jpvt[:n]


def apply_q(QR, tau, C, trans=False, ext=False):
    """Q C (or Q^T C) for Q stored as reflectors below the diagonal of QR."""
    v = _v(ext)
    QR = v.arr(QR)
    C = v.arr(C).copy(order="F")
    m, nc = C.shape
    tau = np.ascontiguousarray(tau, dtype=v.np)
    v.L.orc_apply_q(int(trans), m, nc, len(tau), v.ptr(QR), QR.shape[0], v.ptr(tau), v.ptr(C), m)
    return C


def rot_tangent(alpha, beta, gamma, ext=False):
    return _v(ext).L.orc_rot_tangent(alpha, beta, gamma)


def jacobi(X, V=None, tol=None, maxsweep=30, ext=False, stop=0):
    """Alg. 1 in the working precision on a copy of X; returns (X_inf, V, sweeps, rotations, rc).
    stop: 0 also ends after a negligible sweep (the paper's experiments), 1 only after a sweep
    without rotations (Alg. 1 as printed)."""
    v = _v(ext)
    X = v.arr(X).copy(order="F")
    m, n = X.shape
    if V is not None:
        V = v.arr(V).copy(order="F")
    tol = np.sqrt(m) * unit_roundoff(ext) if tol is None else tol
    sw = ctypes.c_int()
    rot = ctypes.c_longlong()
    rc = v.L.orc_jacobi(m, n, v.ptr(X), m, v.ptr(V), V.shape[0] if V is not None else 1,
                        V.shape[0] if V is not None else 0, tol, maxsweep, stop, ctypes.byref(sw),
                        ctypes.byref(rot))
    return X, V, sw.value, rot.value, rc


def jacobi_derijk(X, V=None, tol=None, maxsweep=30, ext=False, stop=0):
    """Alg. 1 with de Rijk's pivoting (Section 2.1) in the working precision on a copy of X;
    returns (X_inf, V, perm, sweeps, rotations, rc), perm[j] = the input column in position j."""
    v = _v(ext)
    X = v.arr(X).copy(order="F")
    m, n = X.shape
    if V is not None:
        V = v.arr(V).copy(order="F")
    tol = np.sqrt(m) * unit_roundoff(ext) if tol is None else tol
    perm = np.zeros(n, dtype=np.int32)
    sw = ctypes.c_int()
    rot = ctypes.c_longlong()
    rc = v.L.orc_jacobi_derijk(m, n, v.ptr(X), m, v.ptr(V), V.shape[0] if V is not None else 1,
                               V.shape[0] if V is not None else 0, tol, maxsweep, stop,
                               perm.ctypes.data_as(_ip), ctypes.byref(sw), ctypes.byref(rot))
    return X, V, perm, sw.value, rot.value, rc


def jacobi_f32(X, tol=None, maxsweep=30, stop=0):
    """Alg. 1 in binary32 without V; returns (X_inf, sweeps, rotations, rc)."""
    L = lib(False)
    X = np.asfortranarray(np.asarray(X, dtype=np.float32)).copy(order="F")
    m, n = X.shape
    tol = np.sqrt(m) * 2.0 ** -24 if tol is None else tol
    sw = ctypes.c_int()
    rot = ctypes.c_longlong()
    rc = L.orc_jacobi_f32(m, n, X.ctypes.data_as(_fp), m, None, 1, 0, tol, maxsweep, stop,
                          ctypes.byref(sw), ctypes.byref(rot))
    return X, sw.value, rot.value, rc


def svd(A, mode="auto", ext=False, **kw):
    """Algorithm 4 (mode 'auto'), forced low-precision stage ('mixed') or Algorithm 2
    ('plain'). Returns (U, S, V, stats_dict); ext=True runs the long double build."""
    v = _v(ext)
    A = v.arr(A)
    m, n = A.shape
    U = np.zeros((m, n), order="F", dtype=v.np)
    S = np.zeros(n, dtype=v.np)
    V = np.zeros((n, n), order="F", dtype=v.np)
    p = default_params(ext=ext, mode=mode, **kw)
    st = v.Stats()
    v.L.orc_svd(m, n, v.ptr(A), max(1, m), v.ptr(U), v.ptr(S), v.ptr(V), ctypes.byref(p),
                ctypes.byref(st))
    d = st.as_dict()
    d["branch_name"] = BRANCH.get(d["branch"], "?")
    return U, S, V, d


def svd_backward(U, S, V, gU=None, gS=None, gV=None, gap_tol=1e-3, ext=False):
    """Adjoint of the thin SVD; returns (gA, n_flagged)."""
    v = _v(ext)
    U = v.arr(U)
    V = v.arr(V)
    S = np.ascontiguousarray(S, dtype=v.np)
    m, n = U.shape
    gU = v.arr(gU) if gU is not None else None
    gV = v.arr(gV) if gV is not None else None
    gS = np.ascontiguousarray(gS, dtype=v.np) if gS is not None else None
    gA = np.zeros((m, n), order="F", dtype=v.np)
    nf = ctypes.c_int()
    rc = v.L.orc_svd_backward(m, n, v.ptr(U), v.ptr(S), v.ptr(V), v.ptr(gU), v.ptr(gS),
                              v.ptr(gV), v.ptr(gA), gap_tol, ctypes.byref(nf))
    assert rc == 0
    return gA, nf.value
