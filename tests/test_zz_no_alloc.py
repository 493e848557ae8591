"""The allocation-free sketch entry point (rxr_sketch_noalloc), for callers
that cannot allocate device memory, agrees with the ordinary sketch entry
point within the sketch tolerance, call after call.  This file is collected
last so that a run stopping at its first failure has run everything else."""
import ctypes
import math

import numpy as np
import pytest

import oracle as o
from gpu_util import U, to_dev, to_host
from paper_2111_11148_gb300.inputs import usv_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402


def _noalloc(A, s, seed):
    """Call the C ABI directly: device pointers and sizes only."""
    lib = rxr.load()
    m, n = A.shape
    Y = rxr.empty_colmajor(s, n, device=A.device)
    code = lib.rxr_sketch_noalloc(ctypes.c_void_p(A.data_ptr()), m, n, A.stride(1), s, seed,
                                  ctypes.c_void_p(Y.data_ptr()), Y.stride(1),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return Y, code


def _bound(A_np, s, seed):
    # the sketch tolerance of the parity tests: 8 (log2 m + 4) u (|Omega| |A|), entrywise
    Om = o.omega(seed, s, A_np.shape[0])
    return 8 * (math.log2(A_np.shape[0]) + 4) * U * (np.abs(Om) @ np.abs(A_np))


def test_noalloc_sketch_matches_workspace_sketch_on_consecutive_calls():
    # the third case is the largest admissible sketch (s = 2048, n = 128): there
    # the scratch array holds 7 row chunks' partial sums, fewer than the launch
    # geometry asks for (10), so the chunk cap binds
    cases = [(20000, 64, 128, 0, 1e4), (5000, 16, 33, 7, 1e10), (20000, 128, 2048, 3, 1e6),
             (20000, 64, 128, 0, 1e4)]
    with rxr.Handle(0) as h:
        first = None
        for m, n, s, seed, kappa in cases:
            A_np = usv_matrix(m, n, kappa, seed=seed + 1)
            A = to_dev(A_np)
            Y, code = _noalloc(A, s, seed)
            assert code == 0
            Yref = to_host(h.sketch(A, s, seed=seed))
            Yn = to_host(Y)
            assert np.all(np.abs(Yn - Yref) <= 2 * _bound(A_np, s, seed))
            if first is None:
                first = Yn
        # the array keeps the previous call's contents; the last call repeats the
        # first and must not depend on what the calls between left behind
        assert np.array_equal(first, Yn)


def test_noalloc_rejects_invalid_and_oversized_requests():
    lib = rxr.load()
    A = to_dev(usv_matrix(100, 4, 10.0, seed=0))
    Y = rxr.empty_colmajor(8, 4)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.rxr_sketch_noalloc(None, 100, 4, 100, 8, 0, p(Y), 8, None) == -1
    assert lib.rxr_sketch_noalloc(p(A), 100, 4, 99, 8, 0, p(Y), 8, None) == -4
    assert lib.rxr_sketch_noalloc(p(A), 100, 4, 100, 8, 0, p(Y), 7, None) == -8
    assert lib.rxr_sketch_noalloc(p(A), 100, 200, 100, 8, 0, p(Y), 8, None) == -2
