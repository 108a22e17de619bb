"""Thin Python binding of libmpjsvd (include/mpjsvd.h).

Argument marshalling only: every step of the SVD runs in the library's CUDA kernels.
PyTorch provides device memory and the stream. The functions named ``mpjsvd_*`` mirror
the C entry points one to one; ``svd`` / ``svd_batched`` / ``SVDFunction`` are
conveniences built on them.

Layout: the library works on column-major FP64 matrices. A column-major m x n matrix is
held here as a torch tensor of shape (m, n) with strides (1, m) (``colmajor`` makes one).
"""
import ctypes
import os
import warnings

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmpjsvd.so")

MODE = {"auto": 0, "mixed": 1, "plain": 2}
PRECOND = {"rt": 0, "r": 1, "l": 2, "auto": 3}
QRCP = {"mixed": 0, "f64": 1}
STOP = {"xgesvj": 0, "alg1": 1}
LOWK = {"auto": 0, "tc": 1, "reg": 2}
SWITCH = {"u": 0, "v": 1}
GEMMK = {"auto": 0, "tc": 1, "f64": 2}
WORKK = {"auto": 0, "cluster": 1, "cta": 2}
QRU = {"auto": 0, "tc": 1, "f64": 2}
BRANCH = {0: "mixed", 1: "skip_cond", 2: "skip_trailing", 3: "skip_orth", 4: "plain", -1: "?"}
STATUS_NOT_CONVERGED, STATUS_NONFINITE, STATUS_TIMEOUT, STATUS_ZERO_SIGMA = 1, 2, 4, 8

EXPORTS = ["mpjsvd_default_params", "mpjsvd_create", "mpjsvd_set_stream", "mpjsvd_set_params",
           "mpjsvd_svd", "mpjsvd_svd_batched", "mpjsvd_svd_backward", "mpjsvd_get_stats",
           "mpjsvd_destroy", "mpjsvd_last_error", "mpjsvd_svd_noalloc", "mpjsvd_geqrf",
           "mpjsvd_apply_q", "mpjsvd_geqp3", "mpjsvd_selftest_timeout",
           "mpjsvd_svd_backward_batched", "mpjsvd_measure_fp64_peak", "mpjsvd_tc_block_f32",
           "mpjsvd_svd_batched_dev", "mpjsvd_get_batched_tuning", "mpjsvd_dgemm_tc"]


class Params(ctypes.Structure):
    _fields_ = [("tol_alg", ctypes.c_double), ("tol_orth", ctypes.c_double),
                ("tol_cond_coef", ctypes.c_double), ("trailing_frac", ctypes.c_double),
                ("maxsweep", ctypes.c_int), ("block_w", ctypes.c_int), ("mode", ctypes.c_int),
                ("precond", ctypes.c_int), ("qr_first", ctypes.c_int), ("timing", ctypes.c_int),
                ("qrcp", ctypes.c_int), ("stop", ctypes.c_int), ("wait_limit_ms", ctypes.c_int),
                ("low_kernel", ctypes.c_int), ("v_by_qr", ctypes.c_int),
                ("switch_method", ctypes.c_int), ("gemm_kernel", ctypes.c_int), ("y_tol", ctypes.c_double),
                ("work_kernel", ctypes.c_int), ("work_cluster", ctypes.c_int), ("qr_update", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("branch", ctypes.c_int), ("sweeps_low", ctypes.c_int),
                ("sweeps_work", ctypes.c_int), ("rot_low", ctypes.c_longlong),
                ("rot_work", ctypes.c_longlong), ("cond_r", ctypes.c_double),
                ("orth", ctypes.c_double), ("block_w_low", ctypes.c_int),
                ("block_w_work", ctypes.c_int), ("ms_qr", ctypes.c_float),
                ("ms_branch", ctypes.c_float), ("ms_low", ctypes.c_float),
                ("ms_switch", ctypes.c_float), ("ms_work", ctypes.c_float),
                ("ms_final", ctypes.c_float), ("launches", ctypes.c_int), ("qrcp", ctypes.c_int),
                ("precond", ctypes.c_int), ("sweeps_v", ctypes.c_int), ("rot_v", ctypes.c_longlong),
                ("y2_cols", ctypes.c_int), ("n_flagged", ctypes.c_int), ("work_cluster", ctypes.c_int),
                ("rot_sweep_low", ctypes.c_longlong * 16), ("rot_sweep_work", ctypes.c_longlong * 16),
                ("cos_sweep_low", ctypes.c_float * 16), ("cos_sweep_work", ctypes.c_float * 16)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        for name in ("rot_sweep_low", "rot_sweep_work", "cos_sweep_low", "cos_sweep_work"):
            d[name] = list(d[name])
        d["branch_name"] = BRANCH.get(d["branch"], "?")
        return d


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


def load_library(path=LIB_PATH):
    """Load libmpjsvd.so. Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmpjsvd.so not found at %s: run __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)" % path)
    L = ctypes.CDLL(path)
    L.mpjsvd_default_params.argtypes = [ctypes.POINTER(Params)]
    L.mpjsvd_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(Params), _vp]
    L.mpjsvd_set_stream.argtypes = [_vp, _vp]
    L.mpjsvd_set_params.argtypes = [_vp, ctypes.POINTER(Params)]
    L.mpjsvd_svd.argtypes = [_vp, _i, _i, _vp, _i, _vp, _vp, _vp, _d]
    L.mpjsvd_svd_batched.argtypes = [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _d, _vp]
    L.mpjsvd_svd_backward.argtypes = [_vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _d,
                                      ctypes.POINTER(_i)]
    L.mpjsvd_get_stats.argtypes = [_vp, ctypes.POINTER(Stats)]
    L.mpjsvd_destroy.argtypes = [_vp]
    L.mpjsvd_last_error.restype = ctypes.c_char_p
    L.mpjsvd_svd_noalloc.argtypes = [_i, _i, _vp, _i, _vp, _vp, _vp, _d, _vp, _vp]
    L.mpjsvd_geqrf.argtypes = [_vp, _i, _i, _vp, _i, _vp]
    L.mpjsvd_apply_q.argtypes = [_vp, _i, _i, _i, _vp, _i, _vp, _vp, _i]
    L.mpjsvd_geqp3.argtypes = [_vp, _i, _i, _vp, _i, _vp, _vp]
    L.mpjsvd_selftest_timeout.argtypes = [_vp]
    L.mpjsvd_measure_fp64_peak.argtypes = [_vp, ctypes.POINTER(_d)]
    L.mpjsvd_tc_block_f32.argtypes = [_vp, _i, _vp, _i, _vp, _vp]
    L.mpjsvd_svd_batched_dev.argtypes = [_vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _d, _vp]
    L.mpjsvd_get_batched_tuning.argtypes = [_vp, _vp, _vp, _vp]
    L.mpjsvd_dgemm_tc.argtypes = [_vp, _i, _i, _i, _vp, _i, _i, _vp, _i, _vp, _i]
    L.mpjsvd_svd_backward_batched.argtypes = [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                              _vp, _d, _vp]
    _lib = L
    return L


# ---------------------------------------------------------------- C entry points, 1:1

def _check(rc, what):
    if rc != 0:
        raise RuntimeError("%s failed with %d (%s)" % (what, rc,
                                                        load_library().mpjsvd_last_error().decode()))


def mpjsvd_default_params(**overrides):
    p = Params()
    load_library().mpjsvd_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "mode" and isinstance(v, str):
            v = MODE[v]
        if k == "precond" and isinstance(v, str):
            v = PRECOND[v]
        if k == "qrcp" and isinstance(v, str):
            v = QRCP[v]
        if k == "stop" and isinstance(v, str):
            v = STOP[v]
        if k == "low_kernel" and isinstance(v, str):
            v = LOWK[v]
        if k == "switch_method" and isinstance(v, str):
            v = SWITCH[v]
        if k == "gemm_kernel" and isinstance(v, str):
            v = GEMMK[v]
        if k == "work_kernel" and isinstance(v, str):
            v = WORKK[v]
        if k == "qr_update" and isinstance(v, str):
            v = QRU[v]
        setattr(p, k, v)
    return p


def mpjsvd_create(params=None, stream=None):
    h = _vp()
    s = _vp(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    _check(load_library().mpjsvd_create(ctypes.byref(h), ctypes.byref(params) if params else None, s),
           "mpjsvd_create")
    return h


def mpjsvd_set_stream(h, stream):
    _check(load_library().mpjsvd_set_stream(h, _vp(stream)), "mpjsvd_set_stream")


def mpjsvd_set_params(h, params):
    _check(load_library().mpjsvd_set_params(h, ctypes.byref(params)), "mpjsvd_set_params")


def mpjsvd_svd(h, m, n, A_ptr, lda, U_ptr, S_ptr, V_ptr, tol=0.0):
    return load_library().mpjsvd_svd(h, m, n, _vp(A_ptr), lda, _vp(U_ptr), _vp(S_ptr), _vp(V_ptr), tol)


def mpjsvd_svd_batched(h, batch, m_host, n_host, lda_host, A_ptrs, U_ptrs, S_ptrs, V_ptrs, tol, info_ptr):
    return load_library().mpjsvd_svd_batched(h, batch, _vp(m_host), _vp(n_host), _vp(lda_host),
                                             _vp(A_ptrs), _vp(U_ptrs), _vp(S_ptrs), _vp(V_ptrs), tol,
                                             _vp(info_ptr))


def mpjsvd_svd_backward(h, m, n, U_ptr, S_ptr, V_ptr, gU_ptr, gS_ptr, gV_ptr, gA_ptr, gap_tol=1e-3):
    nf = _i(0)
    rc = load_library().mpjsvd_svd_backward(h, m, n, _vp(U_ptr), _vp(S_ptr), _vp(V_ptr),
                                            _vp(gU_ptr), _vp(gS_ptr), _vp(gV_ptr), _vp(gA_ptr),
                                            gap_tol, ctypes.byref(nf))
    return rc, nf.value


def mpjsvd_svd_backward_batched(h, batch, m_host, n_host, U_ptrs, S_ptrs, V_ptrs, gU_ptrs,
                                gS_ptrs, gV_ptrs, gA_ptrs, gap_tol, flags_ptr):
    return load_library().mpjsvd_svd_backward_batched(
        h, batch, _vp(m_host), _vp(n_host), _vp(U_ptrs), _vp(S_ptrs), _vp(V_ptrs), _vp(gU_ptrs),
        _vp(gS_ptrs), _vp(gV_ptrs), _vp(gA_ptrs), gap_tol, _vp(flags_ptr))


def mpjsvd_svd_batched_dev(h, batch, max_m, max_n, m_ptr, n_ptr, lda_ptr, A_ptrs, U_ptrs, S_ptrs,
                           V_ptrs, tol, info_ptr):
    return load_library().mpjsvd_svd_batched_dev(h, batch, max_m, max_n, _vp(m_ptr), _vp(n_ptr),
                                                 _vp(lda_ptr), _vp(A_ptrs), _vp(U_ptrs), _vp(S_ptrs),
                                                 _vp(V_ptrs), tol, _vp(info_ptr))


def mpjsvd_get_batched_tuning(h):
    """Per size class of n (<= 32, 64, 128, 256, 512): (w_low, w_work, sample ms), 0 if untuned."""
    wl, ww, ms = (ctypes.c_int * 5)(), (ctypes.c_int * 5)(), (ctypes.c_float * 5)()
    _check(load_library().mpjsvd_get_batched_tuning(h, wl, ww, ms), "mpjsvd_get_batched_tuning")
    return [(wl[i], ww[i], ms[i]) for i in range(5)]


def mpjsvd_dgemm_tc(h, M, N, K, A_ptr, lda, transA, B_ptr, ldb, C_ptr, ldc):
    return load_library().mpjsvd_dgemm_tc(h, M, N, K, _vp(A_ptr), lda, transA, _vp(B_ptr), ldb,
                                          _vp(C_ptr), ldc)


def mpjsvd_get_stats(h):
    st = Stats()
    _check(load_library().mpjsvd_get_stats(h, ctypes.byref(st)), "mpjsvd_get_stats")
    return st.as_dict()


def mpjsvd_destroy(h):
    if h:
        load_library().mpjsvd_destroy(h)


def mpjsvd_last_error():
    return load_library().mpjsvd_last_error().decode()


def mpjsvd_svd_noalloc(m, n, A_ptr, lda, U_ptr, S_ptr, V_ptr, tol=0.0, status_ptr=None,
                       stream=None):
    """Allocation-free SVD for m <= 512, n <= 256 (static device scratch, no handle).
    status_ptr: device int (or None) that receives the call's status bits."""
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    return load_library().mpjsvd_svd_noalloc(m, n, _vp(A_ptr), lda, _vp(U_ptr), _vp(S_ptr),
                                             _vp(V_ptr), tol, _vp(status_ptr), _vp(s))


def mpjsvd_measure_fp64_peak(stream=None):
    """FP64 FMA throughput of the current GPU in TFLOP/s (the FP64 roofline denominator)."""
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    v = _d(0.0)
    _check(load_library().mpjsvd_measure_fp64_peak(_vp(s), ctypes.byref(v)), "mpjsvd_measure_fp64_peak")
    return v.value


def mpjsvd_tc_block_f32(h, m, Z_ptr, ldz, G_ptr, W_ptr):
    return load_library().mpjsvd_tc_block_f32(h, m, _vp(Z_ptr), ldz, _vp(G_ptr), _vp(W_ptr))


def mpjsvd_selftest_timeout(h):
    return load_library().mpjsvd_selftest_timeout(h)


def mpjsvd_geqrf(h, m, n, A_ptr, lda, tau_ptr):
    return load_library().mpjsvd_geqrf(h, m, n, _vp(A_ptr), lda, _vp(tau_ptr))


def mpjsvd_geqp3(h, m, n, A_ptr, lda, jpvt_ptr, tau_ptr):
    return load_library().mpjsvd_geqp3(h, m, n, _vp(A_ptr), lda, _vp(jpvt_ptr), _vp(tau_ptr))


def mpjsvd_apply_q(h, m, ncols, k, A_ptr, lda, tau_ptr, C_ptr, ldc):
    return load_library().mpjsvd_apply_q(h, m, ncols, k, _vp(A_ptr), lda, _vp(tau_ptr), _vp(C_ptr), ldc)


# ---------------------------------------------------------------- conveniences

def colmajor(x, device=None):
    """A (m, n) float64 tensor with column-major strides (1, m), holding x's values."""
    x = torch.as_tensor(x, dtype=torch.float64)
    m, n = x.shape
    out = torch.empty((n, m), dtype=torch.float64, device=device or x.device).t()
    out.copy_(x)
    return out


def empty_colmajor(m, n, device):
    return torch.empty((n, m), dtype=torch.float64, device=device).t()


def _is_colmajor(x):
    return x.dim() == 2 and x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0])


class Handle:
    """Owns an mpjsvd handle bound to the current CUDA device and stream."""

    def __init__(self, **params):
        self.params = mpjsvd_default_params(**params)
        self.h = mpjsvd_create(self.params)

    def set(self, **params):
        for k, v in params.items():
            if k == "mode" and isinstance(v, str):
                v = MODE[v]
            if k == "precond" and isinstance(v, str):
                v = PRECOND[v]
            if k == "qrcp" and isinstance(v, str):
                v = QRCP[v]
            if k == "stop" and isinstance(v, str):
                v = STOP[v]
            if k == "low_kernel" and isinstance(v, str):
                v = LOWK[v]
            if k == "switch_method" and isinstance(v, str):
                v = SWITCH[v]
            if k == "gemm_kernel" and isinstance(v, str):
                v = GEMMK[v]
            if k == "work_kernel" and isinstance(v, str):
                v = WORKK[v]
            if k == "qr_update" and isinstance(v, str):
                v = QRU[v]
            setattr(self.params, k, v)
        mpjsvd_set_params(self.h, self.params)

    def svd(self, A, tol=0.0, out=None):
        """Thin SVD of a CUDA float64 column-major (m, n) tensor. Returns (U, S, V)."""
        if not (A.is_cuda and A.dtype == torch.float64):
            raise TypeError("A must be a CUDA float64 tensor")
        if not _is_colmajor(A):
            A = colmajor(A, A.device)
        m, n = A.shape
        if out is None:
            U = empty_colmajor(m, n, A.device)
            S = torch.empty(n, dtype=torch.float64, device=A.device)
            V = empty_colmajor(n, n, A.device)
        else:
            U, S, V = out
        mpjsvd_set_stream(self.h, torch.cuda.current_stream(A.device).cuda_stream)
        rc = mpjsvd_svd(self.h, m, n, A.data_ptr(), A.stride(1), U.data_ptr(), S.data_ptr(),
                        V.data_ptr(), tol)
        _check(rc, "mpjsvd_svd")
        return U, S, V

    def svd_batched(self, mats, tol=0.0):
        """Thin SVDs of a list of CUDA float64 (m_i, n_i) tensors in one persistent launch.
        Returns (list of U, list of S, list of V, info tensor)."""
        import numpy as np
        dev = mats[0].device
        mats = [A if _is_colmajor(A) else colmajor(A, dev) for A in mats]
        b = len(mats)
        m = np.array([A.shape[0] for A in mats], dtype=np.int32)
        n = np.array([A.shape[1] for A in mats], dtype=np.int32)
        lda = np.array([A.stride(1) for A in mats], dtype=np.int32)
        Us = [empty_colmajor(int(mi), int(ni), dev) for mi, ni in zip(m, n)]
        Ss = [torch.empty(int(ni), dtype=torch.float64, device=dev) for ni in n]
        Vs = [empty_colmajor(int(ni), int(ni), dev) for ni in n]
        ptr = lambda ts: torch.tensor([t.data_ptr() for t in ts], dtype=torch.int64, device=dev)
        pA, pU, pS, pV = ptr(mats), ptr(Us), ptr(Ss), ptr(Vs)
        info = torch.zeros(b, dtype=torch.int32, device=dev)
        mpjsvd_set_stream(self.h, torch.cuda.current_stream(dev).cuda_stream)
        rc = mpjsvd_svd_batched(self.h, b, m.ctypes.data, n.ctypes.data, lda.ctypes.data,
                                pA.data_ptr(), pU.data_ptr(), pS.data_ptr(), pV.data_ptr(), tol,
                                info.data_ptr())
        _check(rc, "mpjsvd_svd_batched")
        self._keep = (pA, pU, pS, pV)  # pointer arrays live until the next call
        return Us, Ss, Vs, info

    def stats(self):
        return mpjsvd_get_stats(self.h)

    def geqrf(self, A):
        """Householder QR of a CUDA float64 (m, n) tensor: returns (QR in geqrf layout, tau)."""
        A = colmajor(A, A.device)  # a fresh column-major copy (factorized in place)
        m, n = A.shape
        tau = torch.empty(n, dtype=torch.float64, device=A.device)
        mpjsvd_set_stream(self.h, torch.cuda.current_stream(A.device).cuda_stream)
        _check(mpjsvd_geqrf(self.h, m, n, A.data_ptr(), A.stride(1), tau.data_ptr()), "mpjsvd_geqrf")
        return A, tau

    def geqp3(self, A):
        """The preconditioner's RRQR of a CUDA float64 (m, n) tensor (Alg. 5 unless params.qrcp
        says binary64): returns (QR of A P in pivot order, jpvt, tau)."""
        A = colmajor(A, A.device)  # a fresh column-major copy (factorized in place)
        m, n = A.shape
        jpvt = torch.empty(n, dtype=torch.int32, device=A.device)
        tau = torch.empty(n, dtype=torch.float64, device=A.device)
        mpjsvd_set_stream(self.h, torch.cuda.current_stream(A.device).cuda_stream)
        _check(mpjsvd_geqp3(self.h, m, n, A.data_ptr(), A.stride(1), jpvt.data_ptr(), tau.data_ptr()),
               "mpjsvd_geqp3")
        return A, jpvt, tau

    def apply_q(self, QR, tau, C):
        """Q C for Q from geqrf (QR: (m, k) reflectors, tau: k); returns a new tensor."""
        C = colmajor(C, C.device)  # a fresh column-major copy (overwritten)
        m, nc = C.shape
        k = tau.shape[0]
        mpjsvd_set_stream(self.h, torch.cuda.current_stream(C.device).cuda_stream)
        _check(mpjsvd_apply_q(self.h, m, nc, k, QR.data_ptr(), QR.stride(1), tau.data_ptr(),
                              C.data_ptr(), C.stride(1)), "mpjsvd_apply_q")
        return C

    def backward(self, U, S, V, gU=None, gS=None, gV=None, gap_tol=1e-3):
        m, n = U.shape
        gA = empty_colmajor(m, n, U.device)
        cm = lambda t: (colmajor(t, U.device) if t.dim() == 2 and not _is_colmajor(t) else t)
        gU = cm(gU) if gU is not None else None
        gV = cm(gV) if gV is not None else None
        gS = gS.contiguous() if gS is not None else None
        mpjsvd_set_stream(self.h, torch.cuda.current_stream(U.device).cuda_stream)
        rc, nf = mpjsvd_svd_backward(self.h, m, n, U.data_ptr(), S.data_ptr(), V.data_ptr(),
                                     gU.data_ptr() if gU is not None else None,
                                     gS.data_ptr() if gS is not None else None,
                                     gV.data_ptr() if gV is not None else None,
                                     gA.data_ptr(), gap_tol)
        _check(rc, "mpjsvd_svd_backward")
        self.last_n_flagged = nf
        return gA, nf

    def backward_batched(self, Us, Ss, Vs, gUs=None, gSs=None, gVs=None, gap_tol=1e-3):
        """Adjoints of a batch of thin SVDs in one launch. Each g* is a list (entries may be
        None) or None. Returns (list of gA, device int tensor of per-matrix flag counts)."""
        import numpy as np
        dev = Us[0].device
        b = len(Us)
        m = np.array([U.shape[0] for U in Us], dtype=np.int32)
        n = np.array([U.shape[1] for U in Us], dtype=np.int32)
        cm = lambda t: (colmajor(t, dev) if t.dim() == 2 and not _is_colmajor(t) else t)
        Us = [cm(U) for U in Us]
        Vs = [cm(V) for V in Vs]
        gAs = [empty_colmajor(int(mi), int(ni), dev) for mi, ni in zip(m, n)]

        def ptrs(ts):
            if ts is None:
                return None
            ts = [None if t is None else (cm(t) if t.dim() == 2 else t.contiguous()) for t in ts]
            keep.append(ts)
            return torch.tensor([0 if t is None else t.data_ptr() for t in ts], dtype=torch.int64,
                                device=dev)

        keep = []
        pU, pS, pV, pA = ptrs(Us), ptrs(Ss), ptrs(Vs), ptrs(gAs)
        pgU, pgS, pgV = ptrs(gUs), ptrs(gSs), ptrs(gVs)
        flags = torch.zeros(b, dtype=torch.int32, device=dev)
        mpjsvd_set_stream(self.h, torch.cuda.current_stream(dev).cuda_stream)
        rc = mpjsvd_svd_backward_batched(
            self.h, b, m.ctypes.data, n.ctypes.data, pU.data_ptr(), pS.data_ptr(), pV.data_ptr(),
            pgU.data_ptr() if pgU is not None else None, pgS.data_ptr() if pgS is not None else None,
            pgV.data_ptr() if pgV is not None else None, pA.data_ptr(), gap_tol, flags.data_ptr())
        _check(rc, "mpjsvd_svd_backward_batched")
        self._keep_bwd = (keep, pU, pS, pV, pA, pgU, pgS, pgV)  # alive until the next call
        return gAs, flags

    def close(self):
        if self.h:
            mpjsvd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default = {}


def default_handle(device=None):
    dev = torch.cuda.current_device() if device is None else device
    if dev not in _default:
        with torch.cuda.device(dev):
            _default[dev] = Handle()
    return _default[dev]


def svd(A, mode="auto", tol=0.0, **params):
    """Thin SVD through the library. A CPU input is copied to the current GPU and the
    factors are copied back (end-to-end use); a CUDA input stays on the device. A CUDA input
    that requires grad goes through SVDFunction (the library's hand-written adjoint)."""
    if A.is_cuda and A.requires_grad and torch.is_grad_enabled():
        return SVDFunction.apply(A, mode)
    host = not A.is_cuda
    dev = torch.device("cuda", torch.cuda.current_device())
    Ad = colmajor(A.to(torch.float64), dev) if host else A
    h = default_handle(Ad.device.index)
    h.set(mode=mode, **params)
    U, S, V = h.svd(Ad, tol=tol)
    if host:
        return U.cpu(), S.cpu(), V.cpu()
    return U, S, V


def last_backward_flags(device=None):
    """Near-degenerate count of the last adjoint computed on the default handle of `device`
    (pairs with |s_i - s_j| <= gap_tol max(s_i, s_j) plus s_i <= 2^-53 s_0), or None."""
    h = _default.get(torch.cuda.current_device() if device is None else device)
    return getattr(h, "last_n_flagged", None) if h is not None else None


class SVDFunction(torch.autograd.Function):
    """A -> (U, S, V) with the library's forward and hand-written adjoint. Near-degenerate
    singular values are never clamped: the backward warns with their count, which stays
    readable afterwards through last_backward_flags() and the handle's stats (n_flagged)."""

    @staticmethod
    def forward(ctx, A, mode="auto"):
        h = default_handle(A.device.index)
        h.set(mode=mode)
        U, S, V = h.svd(A.detach())
        ctx.save_for_backward(U, S, V)
        return U, S, V

    @staticmethod
    def backward(ctx, gU, gS, gV):
        U, S, V = ctx.saved_tensors
        h = default_handle(U.device.index)
        gA, nf = h.backward(U, S, V, gU, gS, gV)
        if nf:
            warnings.warn("mpjsvd adjoint: %d near-degenerate singular value pair(s) or tiny "
                          "singular value(s); the 1/(s_j^2 - s_i^2) terms are large" % nf,
                          RuntimeWarning, stacklevel=2)
        return gA, None
