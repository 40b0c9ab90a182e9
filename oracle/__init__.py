"""Oracle for tall-skinny QR — TEST INFRASTRUCTURE, NOT PRODUCT CODE.

A plain, slow FP64 CPU Householder QR / least-squares restatement (``tsqr_oracle.c``)
and its ctypes binding. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. It shares no code with the
CUDA library and never imports it.

Every function takes and returns NumPy arrays. Matrices are column-major
(Fortran-ordered) float64; the binding copies inputs into that layout itself.

Definitions followed (see the C file's header for the detail):
  * Householder QR, H = I - tau v v^T, essentially unique with diag(R) > 0 (paper §2.2).
  * TSQR reaches the same R and thin Q by an associative reduction (paper §2.3), so
    the oracle is the plain QR of the whole matrix.
  * Q^T b, Q b and the thin Q (paper §4, Table 2 and Property 1).
  * Least squares through QR, and two refinements around an FP32 QR for the
    mixed-precision path (no counterpart in the paper): Bjorck's augmented system and
    Bjorck's corrected semi-normal equations (the one the library runs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsqr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no FMA contraction, OpenMP over columns)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        sig = {
            "oracle_geqr2": (None, [_i64, _i64, _dp, _i64, _dp]),
            "oracle_apply_qt": (None, [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]),
            "oracle_apply_q": (None, [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]),
            "oracle_form_q": (None, [_i64, _i64, _dp, _i64, _dp, _dp, _i64]),
            "oracle_extract_r": (None, [_i64, _dp, _i64, _dp, _i64]),
            "oracle_sign_normalise_r": (None, [_i64, _dp, _i64, _dp]),
            "oracle_scale_rows": (None, [_i64, _dp, _i64, _dp, _i64]),
            "oracle_scale_cols": (None, [_i64, _i64, _dp, _dp, _i64]),
            "oracle_trsv_upper": (ctypes.c_int, [_i64, _dp, _i64, _dp]),
            "oracle_trsv_upper_t": (ctypes.c_int, [_i64, _dp, _i64, _dp]),
            "oracle_lstsq": (ctypes.c_int, [_i64, _i64, _dp, _i64, _i64, _dp, _i64, _dp, _i64]),
            "oracle_backward_error": (ctypes.c_double, [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]),
            "oracle_orth_error": (ctypes.c_double, [_i64, _i64, _dp, _i64]),
            "oracle_geqr2_f32": (None, [_i64, _i64, _fp, _i64, _fp]),
            "oracle_lstsq_refine_mixed": (ctypes.c_int, [_i64, _i64, _dp, _i64, _dp, _i32,
                                                         ctypes.c_double, _dp, _dp, _dp]),
            "oracle_lstsq_refine_x_only": (ctypes.c_int, [_i64, _i64, _dp, _i64, _dp, _i32, _dp, _dp]),
            "oracle_lstsq_refine_csne": (ctypes.c_int, [_i64, _i64, _dp, _i64, _dp, _i32, ctypes.c_double,
                                                        _dp, _dp]),
            "oracle_apply_qt_f32": (None, [_i64, _i64, _fp, _i64, _fp, _fp]),
            "oracle_r_mixed": (None, [_i64, _i64, _dp, _i64, _i64, _dp, _i64]),
            "oracle_apply_q_f32": (None, [_i64, _i64, _fp, _i64, _fp, _fp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    """A Fortran-ordered float64 copy (the oracle never writes into caller arrays)."""
    return np.array(a, dtype=np.float64, order="F", copy=True)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def set_threads(n: int) -> None:
    """OpenMP thread count for the column loops (results do not depend on it)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
    except OSError:
        pass


def householder(A):
    """Householder QR in place: returns (VR, tau) — R in the upper triangle of VR,
    the reflector tails below it (v_0 = 1 implicit)."""
    lib = _load()
    VR = _f64(A)
    m, n = VR.shape
    if m < n:
        raise ValueError("oracle.householder needs m >= n")
    tau = np.zeros(n)
    lib.oracle_geqr2(m, n, _p(VR), m, _p(tau))
    return VR, tau


def apply_qt(VR, tau, B):
    """Q^T B for the reflectors (VR, tau) of an m-by-n factorization."""
    lib = _load()
    VR = _f64(VR)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    Bv = _f64(B)
    vec = Bv.ndim == 1
    if vec:
        Bv = Bv.reshape(-1, 1, order="F")
    m, n = VR.shape
    lib.oracle_apply_qt(m, n, _p(VR), m, _p(tau), Bv.shape[1], _p(Bv), m)
    return Bv[:, 0] if vec else Bv


def apply_q(VR, tau, B):
    """Q B for the reflectors (VR, tau)."""
    lib = _load()
    VR = _f64(VR)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    Bv = _f64(B)
    vec = Bv.ndim == 1
    if vec:
        Bv = Bv.reshape(-1, 1, order="F")
    m, n = VR.shape
    lib.oracle_apply_q(m, n, _p(VR), m, _p(tau), Bv.shape[1], _p(Bv), m)
    return Bv[:, 0] if vec else Bv


def form_q(VR, tau):
    """The thin Q = Q [I_n; 0] for the reflectors (VR, tau) (no sign normalisation)."""
    lib = _load()
    VR = _f64(VR)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    m, n = VR.shape
    Q = np.zeros((m, n), order="F")
    lib.oracle_form_q(m, n, _p(VR), m, _p(tau), _p(Q), m)
    return Q


def qr(A, normalise: bool = True):
    """Thin QR of A (m >= n): returns (Q m-by-n, R n-by-n, d). With ``normalise`` the
    signs are fixed so that diag(R) >= 0 (R <- D R, Q <- Q D, sign(0) = +1); d holds
    the signs applied (all ones when ``normalise`` is False)."""
    lib = _load()
    VR, tau = householder(A)
    m, n = VR.shape
    Q = np.zeros((m, n), order="F")
    lib.oracle_form_q(m, n, _p(VR), m, _p(tau), _p(Q), m)
    R = np.zeros((n, n), order="F")
    lib.oracle_extract_r(n, _p(VR), m, _p(R), n)
    d = np.ones(n)
    if normalise:
        lib.oracle_sign_normalise_r(n, _p(R), n, _p(d))
        lib.oracle_scale_cols(m, n, _p(d), _p(Q), m)
    return Q, R, d


def r_factor(A):
    """R of A with diag(R) >= 0 (no Q formed)."""
    lib = _load()
    VR, _ = householder(A)
    n = VR.shape[1]
    R = np.zeros((n, n), order="F")
    lib.oracle_extract_r(n, _p(VR), VR.shape[0], _p(R), n)
    d = np.ones(n)
    lib.oracle_sign_normalise_r(n, _p(R), n, _p(d))
    return R


def qt_b(A, B):
    """The unique part of Q^T B: rows 0..n-1 of Q^T B with the sign convention
    diag(R) >= 0, and the column norms of the remaining m-n rows (which equal
    ||B - Q Q^T B|| column by column)."""
    lib = _load()
    VR, tau = householder(A)
    m, n = VR.shape
    C = apply_qt(VR, tau, B)
    vec = C.ndim == 1
    C2 = C.reshape(m, -1, order="F").copy(order="F")
    R = np.zeros((n, n), order="F")
    lib.oracle_extract_r(n, _p(VR), m, _p(R), n)
    d = np.ones(n)
    lib.oracle_sign_normalise_r(n, _p(R), n, _p(d))
    lib.oracle_scale_rows(n, _p(d), C2.shape[1], _p(C2), m)
    top = C2[:n].copy()
    tail = np.sqrt(np.sum(C2[n:] ** 2, axis=0))
    return (top[:, 0], tail[0]) if vec else (top, tail)


def lstsq(A, B):
    """min ||A x - b|| for each column of B (FP64 Householder, back substitution)."""
    lib = _load()
    Aw = _f64(A)
    Bw = _f64(B)
    vec = Bw.ndim == 1
    if vec:
        Bw = Bw.reshape(-1, 1, order="F")
    m, n = Aw.shape
    k = Bw.shape[1]
    X = np.zeros((n, k), order="F")
    rc = lib.oracle_lstsq(m, n, _p(Aw), m, k, _p(Bw), m, _p(X), n)
    if rc != 0:
        raise np.linalg.LinAlgError("oracle.lstsq: R has a zero diagonal entry")
    return X[:, 0] if vec else X


def trsv_upper(R, c):
    """x with R x = c for upper-triangular R (back substitution)."""
    lib = _load()
    R = _f64(R)
    x = np.array(c, dtype=np.float64, copy=True)
    if lib.oracle_trsv_upper(R.shape[0], _p(R), R.shape[0], _p(x)):
        raise np.linalg.LinAlgError("singular R")
    return x


def trsv_upper_t(R, g):
    """x with R^T x = g for upper-triangular R (forward substitution)."""
    lib = _load()
    R = _f64(R)
    x = np.array(g, dtype=np.float64, copy=True)
    if lib.oracle_trsv_upper_t(R.shape[0], _p(R), R.shape[0], _p(x)):
        raise np.linalg.LinAlgError("singular R")
    return x


def lstsq_refine_mixed(A, b, max_steps: int = 10, tol: float = 1e-14):
    """Bjorck augmented-system refinement around an FP32 Householder QR.
    Returns (x, r, hist) where hist[s] = ||dx||/||x|| after correction s."""
    lib = _load()
    Aw = _f64(A)
    m, n = Aw.shape
    bw = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n)
    r = np.zeros(m)
    hist = np.zeros(max(max_steps, 1))
    steps = lib.oracle_lstsq_refine_mixed(m, n, _p(Aw), m, _p(bw), max_steps, tol, _p(x), _p(r), _p(hist))
    if steps < 0:
        raise np.linalg.LinAlgError("singular R in the FP32 factorization")
    return x, r, hist[:steps]


def r_mixed(A, h: int = 128):
    """R (diag >= 0) of the mixed-precision TSQR: FP32 Householder QR of every h-row leaf,
    FP64 Householder QR of the stacked leaf triangles."""
    lib = _load()
    Aw = _f64(A)
    m, n = Aw.shape
    R = np.zeros((n, n), order="F")
    lib.oracle_r_mixed(m, n, _p(Aw), m, max(h, n), _p(R), n)
    d = np.ones(n)
    lib.oracle_sign_normalise_r(n, _p(R), n, _p(d))
    return R


def lstsq_refine_csne(A, b, max_steps: int = 10, tol: float = 1e-10):
    """Corrected semi-normal equations iterated from x = 0 around the R of the
    mixed-precision TSQR (FP32 leaves of 128 rows, FP64 combine; Bjorck 1987), with the
    library's stopping rule.
    Returns (x, hist) where hist[s] = ||dx||/||x|| after step s."""
    lib = _load()
    Aw = _f64(A)
    m, n = Aw.shape
    bw = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n)
    hist = np.zeros(max(max_steps, 1))
    steps = lib.oracle_lstsq_refine_csne(m, n, _p(Aw), m, _p(bw), max_steps, tol, _p(x), _p(hist))
    if steps < 0:
        raise np.linalg.LinAlgError("singular R in the FP32 factorization")
    return x, hist[:steps]


def lstsq_refine_x_only(A, b, max_steps: int = 10):
    """Negative control: x-only refinement around the same FP32 QR."""
    lib = _load()
    Aw = _f64(A)
    m, n = Aw.shape
    bw = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n)
    hist = np.zeros(max(max_steps, 1))
    steps = lib.oracle_lstsq_refine_x_only(m, n, _p(Aw), m, _p(bw), max_steps, _p(x), _p(hist))
    if steps < 0:
        raise np.linalg.LinAlgError("singular R in the FP32 factorization")
    return x, hist[:steps]


def backward_error(A, Q, R) -> float:
    """||A - Q R||_F / ||A||_F (compensated sums)."""
    lib = _load()
    A = _f64(A)
    Q = _f64(Q)
    R = _f64(R)
    m, n = A.shape
    return lib.oracle_backward_error(m, n, _p(A), m, _p(Q), m, _p(R), n)


def orth_error(Q) -> float:
    """||Q^T Q - I||_F (compensated sums)."""
    lib = _load()
    Q = _f64(Q)
    m, n = Q.shape
    return lib.oracle_orth_error(m, n, _p(Q), m)


def geqr2_f32(A):
    """FP32 Householder QR in place: returns (VR float32, tau float32)."""
    lib = _load()
    VR = np.array(A, dtype=np.float32, order="F", copy=True)
    m, n = VR.shape
    tau = np.zeros(n, dtype=np.float32)
    lib.oracle_geqr2_f32(m, n, VR.ctypes.data_as(_fp), m, tau.ctypes.data_as(_fp))
    return VR, tau


def apply_qt_f32(VR, tau, b):
    """Q^T b in FP32 for the reflectors (VR, tau) of geqr2_f32 (one vector b)."""
    lib = _load()
    VR = np.array(VR, dtype=np.float32, order="F", copy=True)
    tau = np.ascontiguousarray(tau, dtype=np.float32)
    w = np.array(b, dtype=np.float32, copy=True)
    m, n = VR.shape
    lib.oracle_apply_qt_f32(m, n, VR.ctypes.data_as(_fp), m, tau.ctypes.data_as(_fp), w.ctypes.data_as(_fp))
    return w


def apply_q_f32(VR, tau, b):
    """Q b in FP32 for the reflectors (VR, tau) of geqr2_f32 (one vector b)."""
    lib = _load()
    VR = np.array(VR, dtype=np.float32, order="F", copy=True)
    tau = np.ascontiguousarray(tau, dtype=np.float32)
    w = np.array(b, dtype=np.float32, copy=True)
    m, n = VR.shape
    lib.oracle_apply_q_f32(m, n, VR.ctypes.data_as(_fp), m, tau.ctypes.data_as(_fp), w.ctypes.data_as(_fp))
    return w


def normalised_r_from(VR) -> np.ndarray:
    """Upper triangle of a factored array with rows scaled so diag >= 0."""
    n = VR.shape[1]
    R = np.triu(np.asarray(VR, dtype=np.float64)[:n, :n])
    s = np.where(np.diag(R) < 0, -1.0, 1.0)
    return R * s[:, None]
