"""Thin ctypes binding of librxr (include/rxr.h): argument marshalling only.

Every step of the factorisation runs in the CUDA kernels of librxr.so; there is
no CPU fallback.  Importing works without a GPU, but every call raises
``RxrError`` if the library is missing or returns an error.

Device matrices are torch CUDA tensors in column-major layout: shape (m, n)
with stride (1, ld), ld >= m (``colmajor`` makes one).  Host matrices for the
``*_host`` entry point are Fortran-ordered float64 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librxr.so")

LU, QR, NONE, SHIFTED = 0, 1, 2, 3
SKETCH_ROWS = 16  # OR-ed into LU / QR: the sketch by row extraction
FP64, SPLIT_BF16, SPLIT_PRECOND = 0, 1, 3
(OK, SKETCH_SINGULAR, CHOL_BREAKDOWN, NONFINITE, CUDA_ERROR, TIMEOUT, NOMEM, UNSUPPORTED, BAD_SPARSE,
 NO_CONVERGENCE) = range(10)
HOOK_STALL, HOOK_JACOBI_SWEEPS, HOOK_BATCH_CTAS = 1, 2, 3  # rxr_set_test_hook
KERNEL_SKETCH, KERNEL_PRECOND_GRAM, KERNEL_PASS_GRAM, KERNEL_APPLY = range(4)

_VARIANTS = {"lu": LU, "qr": QR, "none": NONE, "shifted": SHIFTED, "lu-rows": LU | SKETCH_ROWS,
             "qr-rows": QR | SKETCH_ROWS, LU: LU, QR: QR, NONE: NONE, SHIFTED: SHIFTED,
             LU | SKETCH_ROWS: LU | SKETCH_ROWS, QR | SKETCH_ROWS: QR | SKETCH_ROWS}
_PRECS = {"fp64": FP64, "split": SPLIT_BF16, "split_bf16": SPLIT_BF16, "split_precond": SPLIT_PRECOND,
          FP64: FP64, SPLIT_BF16: SPLIT_BF16, SPLIT_PRECOND: SPLIT_PRECOND}


class RxrError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        msg = status_string(code) if _lib is not None else f"status {code}"
        super().__init__(f"{what}: {msg} (code {code})" if what else f"{msg} (code {code})")


_lib = None


def load() -> ctypes.CDLL:
    """Load librxr.so (built by paper_2111_11148_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RxrError(CUDA_ERROR, f"librxr.so not built at {LIB_PATH}; run paper_2111_11148_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, u64, i, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "rxr_create": ([P(vp), i], i),
        "rxr_destroy": ([vp], i),
        "rxr_workspace_bytes": ([i64, i64, i64, i, P(ctypes.c_size_t)], i),
        "rxr_set_workspace": ([vp, vp, ctypes.c_size_t], i),
        "rxr_cholqr": ([vp, vp, i64, i64, i64, i, i64, u64, i, vp, i64, vp, i64, i, vp], i),
        "rxr_cholqr_async": ([vp, vp, i64, i64, i64, i, i64, u64, i, vp, i64, vp, i64, i, vp, vp], i),
        "rxr_cholqr_host": ([vp, vp, i64, i64, i64, i, i64, u64, i, vp, i64, vp, i64, i, vp], i),
        "rxr_cholqr_batched": ([vp, i, vp, vp, vp, vp, i, vp, vp, i, vp, vp, vp, vp, i, vp, vp], i),
        "rxr_last_info": ([vp, P(i), P(i)], i),
        "rxr_status_string": ([i], ctypes.c_char_p),
        "rxr_omega": ([u64, i64, i64, i64, vp, vp], i),
        "rxr_sketch": ([vp, vp, i64, i64, i64, i64, u64, vp, i64, i, vp], i),
        "rxr_sketch_rows": ([vp, vp, i64, i64, i64, i64, u64, vp, i64, vp], i),
        "rxr_xr_factor": ([vp, vp, i64, i64, i64, i, vp, i64, vp], i),
        "rxr_precond_gram": ([vp, vp, i64, i64, i64, vp, i64, vp, i64, vp, i64, i, vp], i),
        "rxr_cholesky": ([vp, vp, i64, i64, vp, i64, vp], i),
        "rxr_apply_rinv": ([vp, vp, i64, i64, i64, vp, i64, i, vp], i),
        "rxr_lstsq": ([vp, vp, i64, i64, i64, vp, i64, i64, i, i64, u64, vp, i64, i, vp], i),
        "rxr_gram": ([vp, vp, i64, i64, i64, vp, i64, i, vp], i),
        "rxr_orth_error": ([vp, vp, i64, i64, i64, P(d), vp], i),
        "rxr_resid_error": ([vp, vp, i64, i64, i64, vp, i64, vp, i64, P(d), vp], i),
        "rxr_fp64_peak": ([P(d), vp], i),
        "rxr_last_kernel_ms": ([vp, i, P(ctypes.c_float)], i),
        "rxr_set_kernel_timing": ([vp, i], i),
        "rxr_sketch_noalloc": ([vp, i64, i64, i64, i64, u64, vp, i64, vp], i),
        "rxr_set_test_hook": ([vp, i, i], i),
        "rxr_sketch_part": ([vp, vp, i64, i64, i64, i64, u64, i64, vp, i64, i, vp], i),
        "rxr_batch_create": ([vp, i, vp, vp, vp, vp, i, vp, vp, i, vp, vp, vp, vp, i, vp, P(vp)], i),
        "rxr_batch_run": ([vp, vp], i),
        "rxr_batch_destroy": ([vp], i),
        "rxr_sum_parts": ([vp, vp, i, i64, vp, vp], i),
        "rxr_trmm_upper": ([vp, vp, i64, vp, i64, i64, vp, i64, vp], i),
        "rxr_rsvd": ([vp, i64, i64, vp, vp, vp, vp, vp, vp, i64, vp, i64, i64, i, i, i64, u64, i, i, vp, i64, vp, vp,
                      i64, vp], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return [n for n in ("rxr_create", "rxr_destroy", "rxr_workspace_bytes", "rxr_set_workspace", "rxr_cholqr",
                        "rxr_cholqr_async", "rxr_cholqr_host", "rxr_cholqr_batched", "rxr_last_info",
                        "rxr_status_string", "rxr_omega", "rxr_sketch", "rxr_sketch_rows", "rxr_xr_factor",
                        "rxr_precond_gram",
                        "rxr_cholesky", "rxr_apply_rinv", "rxr_lstsq", "rxr_gram", "rxr_orth_error", "rxr_resid_error", "rxr_fp64_peak",
                        "rxr_last_kernel_ms", "rxr_set_kernel_timing", "rxr_sketch_noalloc", "rxr_rsvd",
                        "rxr_set_test_hook", "rxr_sketch_part", "rxr_sum_parts", "rxr_trmm_upper",
                        "rxr_batch_create", "rxr_batch_run", "rxr_batch_destroy")]


def status_string(code: int) -> str:
    return load().rxr_status_string(int(code)).decode()


def _check(code: int, what: str):
    if code != 0:
        raise RxrError(code, what)


# ------------------------------------------------------------------ tensors
def colmajor(t, ld: Optional[int] = None):
    """Column-major copy of a 2-D torch tensor (stride (1, ld))."""
    import torch

    m, n = t.shape
    ld = m if ld is None else int(ld)
    buf = torch.empty((n, ld), dtype=t.dtype, device=t.device)
    out = buf.t()[:m]
    out.copy_(t)
    return out


def empty_colmajor(m: int, n: int, device="cuda", dtype=None, ld: Optional[int] = None):
    import torch

    ld = m if ld is None else int(ld)
    return torch.empty((n, ld), dtype=dtype or torch.float64, device=device).t()[:m]


def _ld(t) -> int:
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    m, n = t.shape
    if n == 1:
        return max(int(t.stride(1)) if t.stride(1) >= m else m, m)
    if t.stride(0) != 1 or t.stride(1) < m:
        raise ValueError("tensor must be column-major (stride (1, ld) with ld >= rows)")
    return int(t.stride(1))


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class BatchPlan:
    """A prepared batch (rxr_batch_plan): Qs, Rs and the device status array
    `status` (count x 4 int32) are owned here; run() enqueues one factorisation
    of every problem on the stream, with no host synchronisation."""

    def __init__(self, handle, As, variant, s, seeds, passes, prec):
        import torch

        self.handle = handle  # keeps the handle alive
        self.As = list(As)
        cnt = len(self.As)
        self.Qs = [empty_colmajor(a.shape[0], a.shape[1], device=a.device) for a in self.As]
        self.Rs = [empty_colmajor(a.shape[1], a.shape[1], device=a.device) for a in self.As]
        s = [2 * a.shape[1] for a in self.As] if s is None else list(s)
        seeds = list(range(cnt)) if seeds is None else list(seeds)
        self.status = torch.zeros((cnt, 4), dtype=torch.int32, device=self.As[0].device)
        arr = lambda T, v: (T * cnt)(*v)
        vp = ctypes.c_void_p
        self._p = ctypes.c_void_p()
        _check(load().rxr_batch_create(
            handle._h, cnt, arr(vp, [a.data_ptr() for a in self.As]), arr(ctypes.c_int64, [a.shape[0] for a in self.As]),
            arr(ctypes.c_int64, [a.shape[1] for a in self.As]), arr(ctypes.c_int64, [_ld(a) for a in self.As]),
            _VARIANTS[variant], arr(ctypes.c_int64, s), arr(ctypes.c_uint64, seeds), int(passes),
            arr(vp, [q.data_ptr() for q in self.Qs]), arr(ctypes.c_int64, [_ld(q) for q in self.Qs]),
            arr(vp, [r.data_ptr() for r in self.Rs]), arr(ctypes.c_int64, [_ld(r) for r in self.Rs]), _PRECS[prec],
            _ptr(self.status), ctypes.byref(self._p)), "rxr_batch_create")

    def run(self, stream=None):
        _check(load().rxr_batch_run(self._p, _stream(stream)), "rxr_batch_run")

    def close(self):
        if self._p:
            load().rxr_batch_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Handle:
    """An rxr_handle bound to one CUDA device."""

    def __init__(self, device: int = 0):
        lib = load()
        self._h = ctypes.c_void_p()
        _check(lib.rxr_create(ctypes.byref(self._h), int(device)), "rxr_create")
        self.device = int(device)

    def close(self):
        if self._h:
            load().rxr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def set_workspace(self, buf=None):
        """rxr_set_workspace: hand the handle caller-owned device memory (a CUDA
        tensor, kept alive by the handle) or return to self-managed workspace
        (None)."""
        self._ws = buf
        ptr = None if buf is None else _ptr(buf)
        nbytes = 0 if buf is None else buf.numel() * buf.element_size()
        _check(load().rxr_set_workspace(self._h, ptr, nbytes), "rxr_set_workspace")

    def set_test_hook(self, hook: int, value: int):
        """rxr_set_test_hook: HOOK_STALL (a bounded device wait runs out) or
        HOOK_JACOBI_SWEEPS (cap on the randomized SVD's Jacobi sweeps)."""
        _check(load().rxr_set_test_hook(self._h, int(hook), int(value)), "rxr_set_test_hook")

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- main calls
    def cholqr(self, A, variant="qr", s: Optional[int] = None, seed: int = 0, passes: int = 2, prec="fp64",
               Q=None, R=None, want_r: bool = True, stream=None, raise_on_error: bool = True):
        """Q, R = rLU/rQR-CholeskyQR(A).  Returns (Q, R, status)."""
        import torch

        m, n = A.shape
        s = 2 * n if s is None else int(s)
        if Q is None:
            Q = empty_colmajor(m, n, device=A.device)
        if R is None and want_r:
            R = empty_colmajor(n, n, device=A.device)
        code = load().rxr_cholqr(self._h, _ptr(A), m, n, _ld(A), _VARIANTS[variant], s, seed & (2**64 - 1),
                                 int(passes), _ptr(Q), _ld(Q), _ptr(R) if R is not None else None,
                                 _ld(R) if R is not None else n, _PRECS[prec], _stream(stream))
        if raise_on_error and code != 0:
            raise RxrError(code, "rxr_cholqr")
        return Q, R, code

    def cholqr_async(self, A, Q, R, status, variant="qr", s=None, seed=0, passes=2, prec="fp64", stream=None):
        m, n = A.shape
        s = 2 * n if s is None else int(s)
        code = load().rxr_cholqr_async(self._h, _ptr(A), m, n, _ld(A), _VARIANTS[variant], s, seed, int(passes),
                                       _ptr(Q), _ld(Q), _ptr(R) if R is not None else None,
                                       _ld(R) if R is not None else n, _PRECS[prec], _stream(stream), _ptr(status))
        _check(code, "rxr_cholqr_async")

    def cholqr_host(self, A: np.ndarray, variant="qr", s=None, seed=0, passes=2, prec="fp64", Q=None, R=None,
                    stream=None):
        """Host-buffer form: numpy (Fortran-order float64) in, numpy out."""
        m, n = A.shape
        if not A.flags["F_CONTIGUOUS"] or A.dtype != np.float64:
            raise ValueError("A must be a Fortran-ordered float64 array")
        s = 2 * n if s is None else int(s)
        Q = np.empty((m, n), order="F") if Q is None else Q
        R = np.empty((n, n), order="F") if R is None else R
        code = load().rxr_cholqr_host(self._h, A.ctypes.data_as(ctypes.c_void_p), m, n, m, _VARIANTS[variant], s,
                                      seed, int(passes), Q.ctypes.data_as(ctypes.c_void_p), m,
                                      R.ctypes.data_as(ctypes.c_void_p), n, _PRECS[prec], _stream(stream))
        _check(code, "rxr_cholqr_host")
        return Q, R

    def cholqr_batched(self, As: Sequence, variant="qr", s: Optional[Sequence[int]] = None,
                       seeds: Optional[Sequence[int]] = None, passes=2, prec="fp64", stream=None):
        """Factorise a list of column-major CUDA tensors; returns (Qs, Rs, statuses)."""
        import torch

        cnt = len(As)
        Qs = [empty_colmajor(a.shape[0], a.shape[1], device=a.device) for a in As]
        Rs = [empty_colmajor(a.shape[1], a.shape[1], device=a.device) for a in As]
        s = [2 * a.shape[1] for a in As] if s is None else list(s)
        seeds = list(range(cnt)) if seeds is None else list(seeds)
        arr = lambda T, v: (T * cnt)(*v)
        vp = ctypes.c_void_p
        st = torch.zeros(4 * cnt, dtype=torch.int32, device=As[0].device if cnt else "cuda")
        code = load().rxr_cholqr_batched(
            self._h, cnt, arr(vp, [a.data_ptr() for a in As]), arr(ctypes.c_int64, [a.shape[0] for a in As]),
            arr(ctypes.c_int64, [a.shape[1] for a in As]), arr(ctypes.c_int64, [_ld(a) for a in As]),
            _VARIANTS[variant], arr(ctypes.c_int64, s), arr(ctypes.c_uint64, seeds), int(passes),
            arr(vp, [q.data_ptr() for q in Qs]), arr(ctypes.c_int64, [_ld(q) for q in Qs]),
            arr(vp, [r.data_ptr() for r in Rs]), arr(ctypes.c_int64, [_ld(r) for r in Rs]), _PRECS[prec],
            _stream(stream), _ptr(st))
        if code < 0 or code == UNSUPPORTED:  # nothing was factorised
            raise RxrError(code, "rxr_cholqr_batched")
        return Qs, Rs, st.view(cnt, 4).cpu().numpy()

    # ---------------------------------------------------------------- row shards
    def sketch_part(self, A, s: int, seed: int = 0, row0: int = 0, prec="fp64", stream=None):
        """Partial sketch of a row shard whose first row is global row row0."""
        m, n = A.shape
        Y = empty_colmajor(s, n, device=A.device)
        _check(load().rxr_sketch_part(self._h, _ptr(A), m, n, _ld(A), s, seed & (2**64 - 1), int(row0), _ptr(Y),
                                      _ld(Y), _PRECS[prec], _stream(stream)), "rxr_sketch_part")
        return Y

    def sum_parts(self, parts, out=None, stream=None):
        """Sum of the blocks parts[0], parts[1], ... (a contiguous CUDA tensor of
        shape (count, ...)) in that order; returns a tensor of shape parts.shape[1:]."""
        import torch

        parts = parts.contiguous()
        count = parts.shape[0]
        if out is None:
            out = torch.empty(parts.shape[1:], dtype=torch.float64, device=parts.device)
        _check(load().rxr_sum_parts(self._h, _ptr(parts), int(count), parts[0].numel(), _ptr(out),
                                    _stream(stream)), "rxr_sum_parts")
        return out

    def trmm_upper(self, A, B, stream=None):
        """A B for upper-triangular column-major A, B (n x n)."""
        n = A.shape[0]
        C = empty_colmajor(n, n, device=A.device)
        _check(load().rxr_trmm_upper(self._h, _ptr(A), _ld(A), _ptr(B), _ld(B), n, _ptr(C), _ld(C),
                                     _stream(stream)), "rxr_trmm_upper")
        return C

    def batch_plan(self, As: Sequence, variant="qr", s: Optional[Sequence[int]] = None,
                   seeds: Optional[Sequence[int]] = None, passes=2, prec="fp64") -> "BatchPlan":
        """rxr_batch_create for the column-major CUDA tensors As (outputs
        allocated here); run it with BatchPlan.run."""
        return BatchPlan(self, As, variant, s, seeds, passes, prec)

    # ---------------------------------------------------------------- stages
    def sketch(self, A, s: int, seed: int = 0, prec="fp64", stream=None):
        m, n = A.shape
        Y = empty_colmajor(s, n, device=A.device)
        _check(load().rxr_sketch(self._h, _ptr(A), m, n, _ld(A), s, seed, _ptr(Y), _ld(Y), _PRECS[prec],
                                 _stream(stream)), "rxr_sketch")
        return Y

    def sketch_rows(self, A, s: int, seed: int = 0, stream=None):
        """Row-extraction sketch: s rows of A drawn uniformly with replacement."""
        m, n = A.shape
        Y = empty_colmajor(s, n, device=A.device)
        _check(load().rxr_sketch_rows(self._h, _ptr(A), m, n, _ld(A), s, seed, _ptr(Y), _ld(Y), _stream(stream)),
               "rxr_sketch_rows")
        return Y

    def xr_factor(self, Y, variant="qr", stream=None, raise_on_error=True):
        s, n = Y.shape
        Rs = empty_colmajor(n, n, device=Y.device)
        code = load().rxr_xr_factor(self._h, _ptr(Y), s, n, _ld(Y), _VARIANTS[variant], _ptr(Rs), _ld(Rs),
                                    _stream(stream))
        if raise_on_error:
            _check(code, "rxr_xr_factor")
        return Rs, code

    def precond_gram(self, A, R, X=None, write_x=True, prec="fp64", stream=None):
        m, n = A.shape
        if X is None and write_x:
            X = empty_colmajor(m, n, device=A.device)
        G = empty_colmajor(n, n, device=A.device)
        _check(load().rxr_precond_gram(self._h, _ptr(A), m, n, _ld(A), _ptr(R), _ld(R),
                                       _ptr(X) if X is not None else None, _ld(X) if X is not None else m,
                                       _ptr(G), _ld(G), _PRECS[prec], _stream(stream)), "rxr_precond_gram")
        return X, G

    def gram(self, X, prec="fp64", stream=None):
        m, n = X.shape
        G = empty_colmajor(n, n, device=X.device)
        _check(load().rxr_gram(self._h, _ptr(X), m, n, _ld(X), _ptr(G), _ld(G), _PRECS[prec], _stream(stream)),
               "rxr_gram")
        return G

    def cholesky(self, G, stream=None, raise_on_error=True):
        n = G.shape[0]
        R = empty_colmajor(n, n, device=G.device)
        code = load().rxr_cholesky(self._h, _ptr(G), n, _ld(G), _ptr(R), _ld(R), _stream(stream))
        if raise_on_error:
            _check(code, "rxr_cholesky")
        return R, code

    def lstsq(self, A, b, variant="qr", s=None, seed=0, prec="fp64", stream=None, raise_on_error=True):
        """x = argmin ||A x - b|| (Section 5.2's preconditioned normal equations);
        b is m or m x k (column-major CUDA tensors).  Returns (x, status)."""
        m, n = A.shape
        s = 2 * n if s is None else int(s)
        b2 = b.reshape(m, 1) if b.dim() == 1 else b
        k = b2.shape[1]
        x = empty_colmajor(n, k, device=A.device)
        code = load().rxr_lstsq(self._h, _ptr(A), m, n, _ld(A), _ptr(b2), k, _ld(b2) if k > 1 or b.dim() == 2 else m,
                                _VARIANTS[variant], s, seed, _ptr(x), _ld(x), _PRECS[prec], _stream(stream))
        if raise_on_error:
            _check(code, "rxr_lstsq")
        return (x[:, 0] if b.dim() == 1 else x), code

    def rsvd(self, A: "DeviceCsr", X, iters: int, variant="qr", s: Optional[int] = None, seed: int = 0,
             passes: int = 2, prec="fp64", U=None, S=None, V=None, stream=None, raise_on_error: bool = True):
        """Randomized SVD with power iteration (Algorithm 7) of the sparse A from
        the n x k starting block X (column-major CUDA tensor), each
        orthonormalisation by CholeskyQR.  Returns (U, S, V, status) with
        Y Y^T A = U diag(S) V^T."""
        import torch

        n, k = X.shape
        if n != A.n:
            raise ValueError("X must have A.n rows")
        s = 2 * k if s is None else int(s)
        U = empty_colmajor(A.m, k, device=X.device) if U is None else U
        V = empty_colmajor(A.n, k, device=X.device) if V is None else V
        S = torch.empty(k, dtype=torch.float64, device=X.device) if S is None else S
        code = load().rxr_rsvd(self._h, A.m, A.n, _ptr(A.indptr), _ptr(A.indices), _ptr(A.data), _ptr(A.t_indptr),
                               _ptr(A.t_indices), _ptr(A.t_data), A.nnz, _ptr(X), _ld(X), k, int(iters),
                               _VARIANTS[variant], s, seed & (2**64 - 1), int(passes), _PRECS[prec], _ptr(U), _ld(U),
                               _ptr(S), _ptr(V), _ld(V), _stream(stream))
        if raise_on_error and code != 0:
            raise RxrError(code, "rxr_rsvd")
        return U, S, V, code

    def apply_rinv(self, X, R, prec="fp64", stream=None):
        """X <- X R^{-1} in place (the Q of a CholeskyQR pass); returns X."""
        m, n = X.shape
        _check(load().rxr_apply_rinv(self._h, _ptr(X), m, n, _ld(X), _ptr(R), _ld(R), _PRECS[prec],
                                     _stream(stream)), "rxr_apply_rinv")
        return X

    def orth_error(self, Q, stream=None) -> float:
        m, n = Q.shape
        out = ctypes.c_double()
        _check(load().rxr_orth_error(self._h, _ptr(Q), m, n, _ld(Q), ctypes.byref(out), _stream(stream)),
               "rxr_orth_error")
        return out.value

    def resid_error(self, A, Q, R, stream=None) -> float:
        m, n = A.shape
        out = ctypes.c_double()
        _check(load().rxr_resid_error(self._h, _ptr(A), m, n, _ld(A), _ptr(Q), _ld(Q), _ptr(R), _ld(R),
                                      ctypes.byref(out), _stream(stream)), "rxr_resid_error")
        return out.value

    def last_info(self):
        p, c = ctypes.c_int(), ctypes.c_int()
        load().rxr_last_info(self._h, ctypes.byref(p), ctypes.byref(c))
        return p.value, c.value

    def set_kernel_timing(self, on: bool = True):
        load().rxr_set_kernel_timing(self._h, 1 if on else 0)

    def last_kernel_ms(self, kernel: int) -> float:
        v = ctypes.c_float()
        load().rxr_last_kernel_ms(self._h, int(kernel), ctypes.byref(v))
        return v.value


class DeviceCsr:
    """A sparse m x n matrix and its transpose in compressed sparse row form on
    a CUDA device: the arrays rxr_rsvd reads (int64 row pointers, int32
    indices, float64 values)."""

    def __init__(self, m, n, indptr, indices, data, t_indptr, t_indices, t_data, device="cuda"):
        import torch

        def dev(a, dt):
            return torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt)

        self.m, self.n = int(m), int(n)
        self.indptr, self.t_indptr = dev(indptr, torch.int64), dev(t_indptr, torch.int64)
        self.indices, self.t_indices = dev(indices, torch.int32), dev(t_indices, torch.int32)
        self.data, self.t_data = dev(data, torch.float64), dev(t_data, torch.float64)

    @classmethod
    def from_host(cls, A, device="cuda") -> "DeviceCsr":
        """Copy an object with fields m, n, indptr, indices, data, t_indptr,
        t_indices, t_data (numpy arrays) to the device."""
        return cls(A.m, A.n, A.indptr, A.indices, A.data, A.t_indptr, A.t_indices, A.t_data, device)

    @property
    def nnz(self) -> int:
        return int(self.indices.numel())


def omega(seed: int, s: int, row0: int, rows: int, device="cuda", stream=None):
    """z values of the Gaussian sketch computed on the GPU: tensor (rows, s) float32."""
    import torch

    z = torch.empty((rows, s), dtype=torch.float32, device=device)
    _check(load().rxr_omega(seed, s, row0, rows, _ptr(z), _stream(stream)), "rxr_omega")
    return z


def sketch_noalloc(A, s: int, seed: int = 0, Y=None, stream=None):
    """Y = Omega A through the allocation-free entry point (no handle)."""
    m, n = A.shape
    if Y is None:
        Y = empty_colmajor(s, n, device=A.device)
    _check(load().rxr_sketch_noalloc(_ptr(A), m, n, _ld(A), s, seed, _ptr(Y), _ld(Y), _stream(stream)),
           "rxr_sketch_noalloc")
    return Y


def fp64_peak_tflops(stream=None) -> float:
    v = ctypes.c_double()
    _check(load().rxr_fp64_peak(ctypes.byref(v), _stream(stream)), "rxr_fp64_peak")
    return v.value


def workspace_bytes(m: int, n: int, s: int, prec="fp64") -> int:
    v = ctypes.c_size_t()
    _check(load().rxr_workspace_bytes(m, n, s, _PRECS[prec], ctypes.byref(v)), "rxr_workspace_bytes")
    return v.value
