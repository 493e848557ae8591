"""Error paths that correct inputs never reach, made to run on request
through the library's test hooks (rxr_set_test_hook), without faulting or
hanging the GPU:

* a bounded device-side wait that runs out: one CTA skips its first TMA copy
  and waits on an mbarrier that nothing arrives at; the kernel records
  RXR_ERR_TIMEOUT and returns, the later kernels of the call return at once,
  the call reports the timeout in about a second per wait, and the handle
  then factorises bit for bit as before (FP64 path: the sketch kernel; split
  path: the fused substitution, which also holds tensor memory);
* the randomized SVD's Jacobi SVD stopped by a sweep cap before it converged
  reports RXR_ERR_NO_CONVERGENCE, and the default cap converges again."""
import time

import numpy as np
import pytest

from gpu_util import to_dev
from paper_2111_11148_gb300.inputs import sparse_operator, start_block, usv_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_bounded_wait_times_out_and_handle_recovers(h, prec):
    A = to_dev(usv_matrix(20000, 64, 1e6, seed=9))   # 16-byte aligned, even lda: the TMA path
    Q0, R0, code = h.cholqr(A, variant="qr", seed=1, prec=prec)
    assert code == 0
    h.set_test_hook(rxr.HOOK_STALL, 1)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Q1, R1, code = h.cholqr(A, variant="qr", seed=1, prec=prec, raise_on_error=False)
        dt = time.perf_counter() - t0
    finally:
        h.set_test_hook(rxr.HOOK_STALL, 0)
    assert code == rxr.TIMEOUT, code
    assert dt < 20.0, dt
    print(f"{prec}: the stalled call returned RXR_ERR_TIMEOUT after {dt:.2f} s")
    # the asynchronous form reports it in the device status word
    h.set_test_hook(rxr.HOOK_STALL, 1)
    try:
        st = torch.zeros(4, dtype=torch.int32, device="cuda")
        Q2 = rxr.empty_colmajor(*A.shape)
        R2 = rxr.empty_colmajor(A.shape[1], A.shape[1])
        h.cholqr_async(A, Q2, R2, st, variant="qr", seed=1, prec=prec)
        torch.cuda.synchronize()
    finally:
        h.set_test_hook(rxr.HOOK_STALL, 0)
    assert st[0].item() == rxr.TIMEOUT
    # the context and the handle are still usable: the same factorisation again
    Q3, R3, code = h.cholqr(A, variant="qr", seed=1, prec=prec)
    assert code == 0
    assert torch.equal(Q3, Q0) and torch.equal(R3, R0)


def test_jacobi_sweep_cap_reports_no_convergence(h):
    P = sparse_operator(3000, 4.83, seed=3)
    A = rxr.DeviceCsr.from_host(P)
    X = to_dev(start_block(P.n, 24, 2))
    h.set_test_hook(rxr.HOOK_JACOBI_SWEEPS, 1)
    try:
        U, S, V, code = h.rsvd(A, X, 1, raise_on_error=False)
    finally:
        h.set_test_hook(rxr.HOOK_JACOBI_SWEEPS, 0)
    assert code == rxr.NO_CONVERGENCE, code
    U, S, V, code = h.rsvd(A, X, 1, raise_on_error=False)
    assert code == 0
    assert np.all(np.diff(S.cpu().numpy()) <= 0)


def test_test_hook_argument_errors(h):
    lib = rxr.load()
    assert lib.rxr_set_test_hook(None, rxr.HOOK_STALL, 1) == -1
    assert lib.rxr_set_test_hook(h._h, 99, 1) == -2
    assert lib.rxr_set_test_hook(h._h, rxr.HOOK_JACOBI_SWEEPS, 41) == -3
