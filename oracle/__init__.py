"""CPU oracle for randomized XR-preconditioned CholeskyQR (FP64).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It shares no code with the CUDA
path; the product never falls back to it.

The arithmetic lives in ``rxr_oracle.c`` (plain C, compiled with
-ffp-contract=off); this module compiles it on demand with gcc and wraps it
with ctypes; a second build with -fopenmp runs the independent row blocks and
rows on all host cores with the same bits (the benchmark's multi-core CPU
baseline; ``rxr_cholqr(..., parallel=True)``).  All matrices are float64 and
column-major (Fortran order).  The
randomized SVD of Section 5.1 (``rsvd``) is composed here from the C
factorisation and library steps (sparse/dense products, LAPACK's SVD).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rxr_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "librxr_oracle.so")
# the same source built with -fopenmp: the multi-core CPU baseline (identical bits)
_LIB_OMP = os.path.join(_LIB_DIR, "librxr_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

OK, SKETCH_SINGULAR, CHOL_BREAKDOWN, NONFINITE = 0, 1, 2, 3
VARIANT_LU, VARIANT_QR, VARIANT_NONE = 0, 1, 2
SKETCH_ROWS = 16  # flag OR-ed into VARIANT_LU / VARIANT_QR: row extraction (Section 2.3)


def _compile(out: str, extra: list[str], force: bool) -> str:
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", *extra,
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/librxr_oracle.so (gcc, -O2,
    single-threaded) and librxr_oracle_omp.so (the same source with -fopenmp)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    _compile(_LIB_OMP, ["-fopenmp"], force)
    return _compile(_LIB, [], force)


def _load(parallel: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if parallel else _lib) is None:
            build()
            lib = ctypes.CDLL(_LIB_OMP if parallel else _LIB)
            P = ctypes.POINTER
            d, i64, u64, u32, i = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
            vp = ctypes.c_void_p
            lib.rxo_philox4x32_10.argtypes = [vp, vp, vp]
            lib.rxo_logf.argtypes = [ctypes.c_float]
            lib.rxo_logf.restype = ctypes.c_float
            lib.rxo_sincos2pi.argtypes = [u32, vp, vp]
            lib.rxo_normal4.argtypes = [u64, u64, u32, u32, vp]
            lib.rxo_omega_z.argtypes = [u64, i64, i64, i64, vp]
            lib.rxo_sketch.argtypes = [vp, i64, i64, i64, i64, u64, vp, i64]
            lib.rxo_sketch_quantised.argtypes = [vp, i64, i64, i64, i64, u64, vp, i64]
            lib.rxo_sketch_shard.argtypes = [vp, i64, i64, i64, i64, u64, i64, vp, i64]
            lib.rxo_row_indices.argtypes = [u64, i64, i64, vp]
            lib.rxo_sketch_rows.argtypes = [vp, i64, i64, i64, i64, u64, vp, i64]
            lib.rxo_geqr_r.argtypes = [vp, i64, i64, i64, vp, i64]
            lib.rxo_getrf_u.argtypes = [vp, i64, i64, i64, vp, i64, vp]
            lib.rxo_sign_normalise.argtypes = [vp, i64, i64]
            lib.rxo_check_factor.argtypes = [vp, i64, i64]
            lib.rxo_check_factor.restype = i
            lib.rxo_trsm_right_upper.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64]
            lib.rxo_gram.argtypes = [vp, i64, i64, i64, vp, i64]
            lib.rxo_potrf_u.argtypes = [vp, i64, i64, vp, i64]
            lib.rxo_potrf_u.restype = i
            lib.rxo_trmm_upper.argtypes = [vp, i64, vp, i64, i64, vp, i64]
            lib.rxo_rxr_cholqr.argtypes = [vp, i64, i64, i64, i, i64, u64, i, vp, i64, vp, i64,
                                           vp, vp, vp, vp, vp, vp, vp]
            lib.rxo_rxr_cholqr.restype = i
            lib.rxo_householder_qr.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64]
            lib.rxo_scholqr.argtypes = [vp, i64, i64, i64, d, i, vp, i64, vp, i64, vp]
            lib.rxo_scholqr.restype = i
            lib.rxo_lstsq.argtypes = [vp, i64, i64, i64, vp, i64, i64, i, i64, u64, vp, i64]
            lib.rxo_lstsq.restype = i
            lib.rxo_orth_error.argtypes = [vp, i64, i64, i64]
            lib.rxo_orth_error.restype = d
            lib.rxo_resid_error.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64]
            lib.rxo_resid_error.restype = d
            lib.rxo_dot2.argtypes = [vp, vp, i64]
            lib.rxo_dot2.restype = d
            lib.rxo_threads.restype = i
            if parallel:
                _lib_omp = lib
            else:
                _lib = lib
    return _lib_omp if parallel else _lib


def threads(parallel: bool = True) -> int:
    """Host threads the oracle's loops use: the OpenMP build's count
    (OMP_NUM_THREADS, else every core) or 1 for the serial build."""
    return int(_load(parallel).rxo_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ld(a: np.ndarray) -> int:
    assert a.flags["F_CONTIGUOUS"]
    return max(1, a.shape[0])


# ---------------------------------------------------------------- generator
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    _load().rxo_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def logf(u: float) -> np.float32:
    return np.float32(_load().rxo_logf(ctypes.c_float(u)))


def sincos2pi(nint: int):
    s = np.zeros(1, np.float32)
    c = np.zeros(1, np.float32)
    _load().rxo_sincos2pi(int(nint), _p(s), _p(c))
    return s[0], c[0]


def normal4(seed: int, i: int, k: int, stream: int = 0) -> np.ndarray:
    z = np.zeros(4, np.float32)
    _load().rxo_normal4(seed, i, k, stream, _p(z))
    return z


def omega_z(seed: int, s: int, i0: int, rows: int) -> np.ndarray:
    """z values (float32) of Omega's columns i0..i0+rows-1: shape (rows, s)."""
    z = np.zeros((rows, s), np.float32)
    _load().rxo_omega_z(seed, s, i0, rows, _p(z))
    return z


def omega(seed: int, s: int, m: int) -> np.ndarray:
    """The s x m sketch matrix Omega = z / sqrt(s) in float64 (small m only)."""
    z = omega_z(seed, s, 0, m)
    return np.asfortranarray((1.0 / np.sqrt(float(s))) * z.T.astype(np.float64))


# ---------------------------------------------------------------- steps
def sketch(A: np.ndarray, s: int, seed: int, row0: int = 0) -> np.ndarray:
    """Y = Omega A; with row0, A holds rows row0 .. row0 + m - 1 of a larger
    matrix and Omega's columns follow those global rows (a row shard's share)."""
    A = _f64(A)
    m, n = A.shape
    Y = np.zeros((s, n), order="F")
    if row0:
        _load().rxo_sketch_shard(_p(A), m, n, _ld(A), s, seed, int(row0), _p(Y), s)
    else:
        _load().rxo_sketch(_p(A), m, n, _ld(A), s, seed, _p(Y), s)
    return Y


def sketch_quantised(A: np.ndarray, s: int, seed: int) -> np.ndarray:
    """Y' = Omega' A with Omega' = rint(4096 z) / 4096 / sqrt(s): the sketch matrix
    of the split-precision path (the same draws on the 2^-12 grid)."""
    A = _f64(A)
    m, n = A.shape
    Y = np.zeros((s, n), order="F")
    _load().rxo_sketch_quantised(_p(A), m, n, _ld(A), s, seed, _p(Y), s)
    return Y


def row_indices(seed: int, l: int, m: int) -> np.ndarray:
    """Row extraction (Section 2.3, Theorem 3.2): l rows of m drawn independently
    with probability 1/m each (with replacement), in draw order."""
    idx = np.zeros(l, np.int64)
    _load().rxo_row_indices(seed, l, m, _p(idx))
    return idx


def sketch_rows(A: np.ndarray, l: int, seed: int) -> np.ndarray:
    """A_1 = PA: row k is row row_indices(seed, l, m)[k] of A."""
    A = _f64(A)
    m, n = A.shape
    Y = np.zeros((l, n), order="F")
    _load().rxo_sketch_rows(_p(A), m, n, _ld(A), l, seed, _p(Y), l)
    return Y


def omega_quantised(seed: int, s: int, m: int) -> np.ndarray:
    z = omega_z(seed, s, 0, m).astype(np.float64)
    return np.asfortranarray((1.0 / np.sqrt(float(s))) * (np.rint(z * 4096.0) / 4096.0).T)


def geqr_r(W: np.ndarray) -> np.ndarray:
    W = _f64(W).copy(order="F")
    l, n = W.shape
    R = np.zeros((n, n), order="F")
    _load().rxo_geqr_r(_p(W), l, n, _ld(W), _p(R), n)
    return R


def getrf_u(W: np.ndarray):
    W = _f64(W).copy(order="F")
    l, n = W.shape
    U = np.zeros((n, n), order="F")
    piv = np.zeros(n, np.int64)
    _load().rxo_getrf_u(_p(W), l, n, _ld(W), _p(U), n, _p(piv))
    L = np.tril(W[:, :n], -1)
    L[np.arange(n), np.arange(n)] = 1.0
    return U, L, piv


def sign_normalise(R: np.ndarray) -> np.ndarray:
    R = _f64(R).copy(order="F")
    _load().rxo_sign_normalise(_p(R), R.shape[0], _ld(R))
    return R


def check_factor(R: np.ndarray) -> int:
    R = _f64(R)
    return int(_load().rxo_check_factor(_p(R), R.shape[0], _ld(R)))


def trsm_right_upper(A: np.ndarray, R: np.ndarray) -> np.ndarray:
    A = _f64(A)
    R = _f64(R)
    m, n = A.shape
    X = np.zeros((m, n), order="F")
    _load().rxo_trsm_right_upper(_p(A), m, n, _ld(A), _p(R), _ld(R), _p(X), max(1, m))
    return X


def gram(X: np.ndarray) -> np.ndarray:
    X = _f64(X)
    m, n = X.shape
    G = np.zeros((n, n), order="F")
    _load().rxo_gram(_p(X), m, n, _ld(X), _p(G), n)
    return G


def potrf_u(G: np.ndarray):
    """Upper Cholesky factor; returns (R, info) with info = breakdown column+1 or 0."""
    G = _f64(G)
    n = G.shape[0]
    R = np.zeros((n, n), order="F")
    info = _load().rxo_potrf_u(_p(G), n, _ld(G), _p(R), n)
    return R, int(info)


def trmm_upper(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    A = _f64(A)
    B = _f64(B)
    n = A.shape[0]
    C = np.zeros((n, n), order="F")
    _load().rxo_trmm_upper(_p(A), _ld(A), _p(B), _ld(B), n, _p(C), n)
    return C


class Result:
    """Outputs and intermediates of one oracle factorisation."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def rxr_cholqr(A: np.ndarray, variant: int = VARIANT_QR, s: int | None = None, seed: int = 0,
               passes: int = 2, parallel: bool = False) -> Result:
    """rLU-/rQR-CholeskyQR (Algorithms 4/5) with `passes` CholeskyQR passes.
    parallel: run the OpenMP build of the same code (the same bits)."""
    A = _f64(A)
    m, n = A.shape
    s = 2 * n if s is None else int(s)
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    Y = np.zeros((s, n), order="F")
    mats = [np.zeros((n, n), order="F") for _ in range(5)]
    info = np.zeros(2, np.int32)
    st = _load(parallel).rxo_rxr_cholqr(_p(A), m, n, _ld(A), variant, s, seed, passes, _p(Q), max(1, m), _p(R), n,
                                _p(Y), *[_p(x) for x in mats], _p(info))
    return Result(status=int(st), Q=Q, R=R, Y=Y, Rs=mats[0], G1=mats[1], R1=mats[2], G2=mats[3], R2=mats[4],
                  info=(int(info[0]), int(info[1])))


def scholqr(A: np.ndarray, shift: float, passes: int = 3) -> Result:
    """Shifted CholeskyQR3 (Section 2.1): R_1 = chol(A^T A + shift I), Q_1 = A R_1^{-1},
    then passes - 1 CholeskyQR steps; the shift is absolute."""
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    info = np.zeros(2, np.int32)
    st = _load().rxo_scholqr(_p(A), m, n, _ld(A), float(shift), int(passes), _p(Q), max(1, m), _p(R), n, _p(info))
    return Result(status=int(st), Q=Q, R=R, info=(int(info[0]), int(info[1])))


def lstsq(A: np.ndarray, b: np.ndarray, variant: int = VARIANT_QR, s: int | None = None, seed: int = 0):
    """min ||A x - b|| by Section 5.2's solver preconditioned by the sketch's R
    factor; b is m or m x k.  Returns (x, status)."""
    A = _f64(A)
    m, n = A.shape
    s = 2 * n if s is None else int(s)
    b2 = _f64(b.reshape(m, -1))
    k = b2.shape[1]
    x = np.zeros((n, k), order="F")
    st = _load().rxo_lstsq(_p(A), m, n, _ld(A), _p(b2), k, max(1, m), variant, s, seed, _p(x), n)
    return (x[:, 0] if b.ndim == 1 else x), int(st)


def householder_qr(A: np.ndarray):
    """Thin QR A = QR with diag(R) >= 0 by Householder reflections."""
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    _load().rxo_householder_qr(_p(A), m, n, _ld(A), _p(Q), max(1, m), _p(R), n)
    return Q, R


def orth_error(Q: np.ndarray) -> float:
    Q = _f64(Q)
    return float(_load().rxo_orth_error(_p(Q), Q.shape[0], Q.shape[1], _ld(Q)))


def resid_error(A: np.ndarray, Q: np.ndarray, R: np.ndarray) -> float:
    A, Q, R = _f64(A), _f64(Q), _f64(R)
    return float(_load().rxo_resid_error(_p(A), A.shape[0], A.shape[1], _ld(A), _p(Q), _ld(Q), _p(R), _ld(R)))


def dot2(x, y) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(_load().rxo_dot2(_p(x), _p(y), x.size))


def rsvd(A, X: np.ndarray, K: int, variant: int = VARIANT_QR, s: int | None = None, seed: int = 0,
         passes: int = 2, orth: str = "rxr") -> Result:
    """Randomized SVD with power iteration (Algorithm 7, Section 5.1) of an
    m x n matrix A (a scipy.sparse matrix or an ndarray) from the n x k
    starting block X:

        Y = orth(A X); K times: Y = orth(A^T Y), Y = orth(A Y);
        B = Y^T A (k x n) = U_B diag(S) V^T by LAPACK's SVD; U = Y U_B.

    orth="rxr": the j-th orthonormalisation (j = 0, 1, ...) is the Q factor of
    rxr_cholqr(., variant, s (default 2k), seed + j, passes), the replacement
    Section 5.1 makes; orth="householder": the Householder QR's Q.  A failed
    factorisation stops the iteration and its status is returned."""
    X = _f64(X)
    k = X.shape[1]
    s = 2 * k if s is None else int(s)
    calls = 0

    def orth_(Y):
        nonlocal calls
        Y = _f64(Y)
        if orth == "householder":
            return householder_qr(Y)[0], 0
        r = rxr_cholqr(Y, variant, s, seed + calls, passes)
        calls += 1
        return r.Q, r.status

    Y, st = orth_(A @ X)
    for _ in range(int(K)):
        if st:
            break
        Y, st = orth_(A.T @ Y)
        if st:
            break
        Y, st = orth_(A @ Y)
    if st:
        return Result(status=st, U=None, S=None, V=None, Q=None, calls=calls)
    B = np.asarray(A.T @ Y).T  # Y^T A
    Ub, S, Vt = np.linalg.svd(B, full_matrices=False)
    return Result(status=0, U=np.asfortranarray(Y @ Ub), S=S, V=np.asfortranarray(Vt.T), Q=Y, calls=calls)
