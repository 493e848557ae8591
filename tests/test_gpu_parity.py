"""Parity of the CUDA path (through the C ABI) with the CPU oracle, step by
step and end to end, on seeded synthetic inputs A = U Sigma V^T (Section 4.1)
at sizes that span several panels plus a ragged tail.

Tolerances: Omega is compared bit for bit (FP32 arithmetic with explicit
rounding on both sides).  Floating-point results are compared against a bound
derived from the arithmetic: the sketch and Gram sums entrywise against
c log2(m) u (|Omega||A|) and c m u (|X|^T|X|); the factors against the spread
between the oracle and LAPACK (two independent correct FP64 implementations);
the final factorisation against the accuracy targets ||Q^T Q - I||_F <= 1e-13,
||A - QR||_F / ||A||_F <= 1e-14 and the R-factor bound 100 kappa u."""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as o
from gpu_util import R_TOL, U, r_rel, to_dev, to_host
from paper_2111_11148_gb300.inputs import usv_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402

OV = {"lu": o.VARIANT_LU, "qr": o.VARIANT_QR, "none": o.VARIANT_NONE}


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


# ------------------------------------------------------------------ Omega
@pytest.mark.parametrize("seed,s,row0,rows", [(0, 128, 0, 1000), (1, 7, 5, 333), (123456789, 1, 0, 70),
                                              (2**63 + 11, 33, 2**32 - 3, 50), (0, 256, 10**9, 64)])
def test_omega_bit_exact(seed, s, row0, rows):
    z = rxr.omega(seed, s, row0, rows).cpu().numpy()
    ref = o.omega_z(seed, s, row0, rows)
    assert np.array_equal(z.view(np.uint32), ref.view(np.uint32))


def test_omega_matches_stored_golden():
    from test_golden import read_omega

    for seed, i, s, r, bits in read_omega():
        z = rxr.omega(seed, s, i, 1).cpu().numpy()
        assert int(z[0, r].view(np.uint32)) == bits


def test_philox_matches_curand():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = os.path.join(os.path.dirname(__file__), "cuda", "curand_philox.cu")
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, "libcp.so")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fPIC",
                        src, "-o", so], check=True)
        import ctypes

        lib = ctypes.CDLL(so)
        rng = np.random.default_rng(0)
        cnt = 64
        i = rng.integers(0, 2**40, cnt, dtype=np.uint64)
        k = rng.integers(0, 2**20, cnt, dtype=np.uint64)
        stream = np.zeros(cnt, dtype=np.uint64)
        subseq = torch.tensor((stream << np.uint64(32)) | k, dtype=torch.int64).cuda()
        offset = torch.tensor(i * np.uint64(4), dtype=torch.int64).cuda()
        out = torch.zeros(4 * cnt, dtype=torch.int32).cuda()
        seed = 0x0123456789ABCDEF
        assert lib.curand_philox_outputs(ctypes.c_uint64(seed), ctypes.c_void_p(subseq.data_ptr()),
                                         ctypes.c_void_p(offset.data_ptr()), cnt,
                                         ctypes.c_void_p(out.data_ptr())) == 0
        got = out.cpu().numpy().view(np.uint32).reshape(cnt, 4)
        for t in range(cnt):
            ctr = [int(i[t]) & 0xFFFFFFFF, int(i[t]) >> 32, int(k[t]), 0]
            ref = o.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
            assert np.array_equal(got[t], ref), t


# ------------------------------------------------------------------ sketch
@pytest.mark.parametrize("m,n,s", [(1, 1, 1), (63, 3, 7), (64, 16, 32), (1000, 16, 33), (4097, 64, 128),
                                   (3000, 70, 140), (2500, 128, 256), (700, 5, 300), (2100, 100, 200),
                                   (1000, 40, 128), (900, 52, 104), (1500, 100, 256)])
def test_sketch_parity(h, m, n, s):
    A = usv_matrix(m, n, 1e3, seed=m + n)
    Y = to_host(h.sketch(to_dev(A), s, seed=7))
    ref = o.sketch(A, s, seed=7)
    Om = o.omega(7, s, m)
    bound = 8 * (math.log2(m) + 4) * U * (np.abs(Om) @ np.abs(A))
    assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)


# ------------------------------------------------------------------ XR factor of the sketch
@pytest.mark.parametrize("variant", ["qr", "lu"])
@pytest.mark.parametrize("s,n,kappa", [(32, 16, 1e4), (128, 64, 1e10), (17, 16, 1e2), (256, 128, 1e6), (3, 1, 1),
                                         (1024, 512, 1e13), (300, 150, 1e12), (64, 33, 1e8)])
def test_xr_factor_parity(h, variant, s, n, kappa):
    if s * n <= 40000:
        A = usv_matrix(max(40 * n, 100), n, kappa, seed=3)
        Y = o.sketch(A, s, seed=1)
    else:
        # wide sketches (the blocked multi-CTA QR): a sketch-shaped matrix of the
        # same conditioning, directly
        Y = usv_matrix(s, n, kappa, seed=3)
    Rs, code = h.xr_factor(to_dev(Y), variant)
    assert code == 0
    Rg = to_host(Rs)
    if variant == "qr":
        Ro = o.sign_normalise(o.geqr_r(Y))
        Rl = np.linalg.qr(Y, mode="r")
    else:
        Ro, _, _ = o.getrf_u(Y)
        Ro = o.sign_normalise(Ro)
        Rl = sla.lu(Y)[2][:n]
    d = np.sign(np.diag(Rl))
    d[d == 0] = 1
    Rl = d[:, None] * Rl
    spread = np.linalg.norm(Ro - Rl, axis=0)
    colnorm = np.linalg.norm(Ro, axis=0)
    err = np.linalg.norm(Rg - Ro, axis=0)
    assert np.all(err <= 10 * spread + 64 * n * U * colnorm * max(1.0, np.linalg.cond(Y) * U * 1e3))
    assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)


def test_xr_factor_reports_singular_sketch(h):
    Y = np.asfortranarray(np.random.default_rng(0).standard_normal((20, 6)))
    Y[:, 3] = 0.0
    for v in ("qr", "lu"):
        _, code = h.xr_factor(to_dev(Y), v, raise_on_error=False)
        assert code == rxr.SKETCH_SINGULAR


# ------------------------------------------------------------------ substitution + Gram
@pytest.mark.parametrize("m,n", [(1, 1), (127, 8), (128, 16), (1000, 64), (5000, 70), (2049, 128), (300, 100)])
def test_precond_gram_parity(h, m, n):
    A = usv_matrix(m, n, 1e3, seed=11)
    ref = o.rxr_cholqr(A, o.VARIANT_QR, 2 * n, seed=2, passes=1)
    R = ref.Rs
    X, G = h.precond_gram(to_dev(A), to_dev(R))
    Xg, Gg = to_host(X), to_host(G)
    Xo = o.trsm_right_upper(A, R)
    # row-wise substitution error: |x^ - x| <~ n u |x^||R||R^-1|
    bound = 4 * n * U * (np.abs(Xo) @ np.abs(R) @ np.abs(np.linalg.inv(R))) + 1e-300
    assert np.all(np.abs(Xg - Xo) <= bound), np.max(np.abs(Xg - Xo) / bound)
    Go = o.gram(Xg)                                   # the Gram of the X the GPU produced
    gb = 4 * (m + 2) * U * (np.abs(Xg).T @ np.abs(Xg))
    assert np.all(np.abs(Gg - Go) <= gb)
    assert np.array_equal(Gg, Gg.T)


def test_precond_gram_without_x(h):
    A = usv_matrix(900, 12, 1e2, seed=5)
    R = o.rxr_cholqr(A, o.VARIANT_QR, 24, seed=0, passes=1).Rs
    X, G = h.precond_gram(to_dev(A), to_dev(R))
    _, G2 = h.precond_gram(to_dev(A), to_dev(R), write_x=False)
    assert np.array_equal(to_host(G), to_host(G2))


# ------------------------------------------------------------------ Cholesky
@pytest.mark.parametrize("n", [1, 2, 16, 64, 65, 128, 200, 512])
def test_cholesky_parity(h, n):
    X = np.random.default_rng(n).standard_normal((4 * n + 10, n))
    G = np.asfortranarray(X.T @ X)
    R, code = h.cholesky(to_dev(G))
    assert code == 0
    Ro, info = o.potrf_u(G)
    Rg = to_host(R)
    assert np.linalg.norm(Rg - Ro) <= 64 * n * U * np.linalg.norm(Ro) * np.linalg.cond(Ro)
    assert np.all(np.tril(Rg, -1) == 0)


def test_cholesky_breakdown_column(h):
    G = np.asfortranarray(np.diag([4.0, 1.0, -2.0, 3.0]))
    _, code = h.cholesky(to_dev(G), raise_on_error=False)
    assert code == rxr.CHOL_BREAKDOWN
    assert h.last_info()[1] == 2
    # the blocked form (n > 64) reports the global column, here in the third panel
    d = np.ones(150)
    d[77] = -1.0
    _, code = h.cholesky(to_dev(np.asfortranarray(np.diag(d))), raise_on_error=False)
    assert code == rxr.CHOL_BREAKDOWN
    assert h.last_info()[1] == 77


# ------------------------------------------------------------------ end to end
def _check_factorisation(A, Qg, Rg, ref, kappa):
    assert o.orth_error(Qg) <= 1e-13
    assert o.resid_error(A, Qg, Rg) <= 1e-14
    assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)
    rel = np.linalg.norm(Rg - ref.R) / np.linalg.norm(ref.R)
    assert rel <= R_TOL, rel
    return rel


@pytest.mark.parametrize("variant", ["lu", "qr"])
@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e12, 1e15])
def test_cholqr_parity_kappa_sweep(h, variant, kappa):
    m, n = 5000, 16
    A = usv_matrix(m, n, kappa, seed=1)
    Q, R, code = h.cholqr(to_dev(A), variant=variant, s=32, seed=0, passes=2)
    assert code == 0
    ref = o.rxr_cholqr(A, OV[variant], 32, seed=0, passes=2)
    _check_factorisation(A, to_host(Q), to_host(R), ref, kappa)


def test_cholqr_small_config_lu_kappa_1e8(h):
    # m = 20000, n = 16, kappa = 1e8, s = 2n, seed 0, two passes, rLU
    A = usv_matrix(20000, 16, 1e8, seed=0)
    Q, R, code = h.cholqr(to_dev(A), variant="lu", s=32, seed=0, passes=2)
    ref = o.rxr_cholqr(A, o.VARIANT_LU, 32, seed=0, passes=2)
    rel = _check_factorisation(A, to_host(Q), to_host(R), ref, 1e8)
    Qh, Rh = o.householder_qr(A)
    assert r_rel(to_host(R), Rh) <= R_TOL
    print("R rel diff vs oracle", rel)


@pytest.mark.parametrize("m,n,s,passes,variant", [(1, 1, 1, 2, "qr"), (16, 16, 16, 2, "qr"), (65, 3, 7, 1, "lu"),
                                                  (129, 64, 129, 3, "qr"), (3001, 100, 201, 2, "lu"),
                                                  (2048, 128, 256, 2, "qr"), (777, 9, 9, 2, "none")])
def test_cholqr_shapes_and_passes(h, m, n, s, passes, variant):
    kappa = 1e5 if variant != "none" else 1e3
    A = usv_matrix(m, n, kappa, seed=m)
    Q, R, code = h.cholqr(to_dev(A), variant=variant, s=s, seed=4, passes=passes)
    assert code == 0
    ref = o.rxr_cholqr(A, OV[variant], s, seed=4, passes=passes)
    assert ref.status == 0
    Qg, Rg = to_host(Q), to_host(R)
    tol_o = 1e-13 if passes > 1 else 1e-11
    assert o.orth_error(Qg) <= tol_o
    assert o.resid_error(A, Qg, Rg) <= 1e-14
    assert r_rel(Rg, ref.R) <= R_TOL


def test_padded_leading_dimension_and_in_place(h):
    m, n = 1000, 12
    A = usv_matrix(m, n, 1e6, seed=9)
    Ad = to_dev(A, ld=m + 7)                       # odd leading dimension: plain-load path
    Q, R, _ = h.cholqr(Ad, variant="qr", seed=0)
    Ad2 = to_dev(A, ld=m + 6)                      # even padding: TMA path
    Q2, R2, _ = h.cholqr(Ad2, variant="qr", seed=0)
    assert np.array_equal(to_host(Q), to_host(Q2)) and np.array_equal(to_host(R), to_host(R2))
    Ain = to_dev(A)
    Qi, Ri, _ = h.cholqr(Ain, variant="qr", seed=0, Q=Ain)   # Q overwrites A
    assert np.array_equal(to_host(Qi), to_host(Q)) and np.array_equal(to_host(Ri), to_host(R))


def test_deterministic_and_r_less(h):
    A = to_dev(usv_matrix(3000, 24, 1e9, seed=2))
    Q1, R1, _ = h.cholqr(A, variant="lu", seed=5)
    Q2, R2, _ = h.cholqr(A, variant="lu", seed=5)
    Q3, R3, _ = h.cholqr(A, variant="lu", seed=5, want_r=False)
    assert R3 is None
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2) and torch.equal(Q1, Q3)


def test_failure_statuses(h):
    A = usv_matrix(600, 8, 1e3, seed=1)
    B = A.copy(order="F")
    B[100, 3] = np.inf
    for v in ("qr", "lu", "none"):
        _, _, code = h.cholqr(to_dev(B), variant=v, raise_on_error=False)
        assert code == rxr.NONFINITE, v
    Z = A.copy(order="F")
    Z[:, 5] = 0.0
    for v in ("qr", "lu"):
        _, _, code = h.cholqr(to_dev(Z), variant=v, raise_on_error=False)
        assert code == rxr.SKETCH_SINGULAR
    bad = usv_matrix(2000, 10, 1e12, seed=8)
    _, _, code = h.cholqr(to_dev(bad), variant="none", raise_on_error=False)
    assert code == rxr.CHOL_BREAKDOWN and h.last_info()[0] == 1
    for v in ("qr", "lu"):
        _, _, code = h.cholqr(to_dev(bad), variant=v, raise_on_error=False)
        assert code == 0


def test_invalid_arguments(h):
    lib = rxr.load()
    A = to_dev(usv_matrix(100, 4, 10, seed=0))
    Q = rxr.empty_colmajor(100, 4)
    p = lambda t: t.data_ptr()
    assert lib.rxr_cholqr(h._h, None, 100, 4, 100, 1, 8, 0, 2, p(Q), 100, None, 4, 0, None) == -1
    assert lib.rxr_cholqr(h._h, p(A), 3, 4, 100, 1, 8, 0, 2, p(Q), 100, None, 4, 0, None) == -2
    assert lib.rxr_cholqr(h._h, p(A), 100, 4, 99, 1, 8, 0, 2, p(Q), 100, None, 4, 0, None) == -4
    assert lib.rxr_cholqr(h._h, p(A), 100, 4, 100, 7, 8, 0, 2, p(Q), 100, None, 4, 0, None) == -5
    assert lib.rxr_cholqr(h._h, p(A), 100, 4, 100, 1, 3, 0, 2, p(Q), 100, None, 4, 0, None) == -6
    assert lib.rxr_cholqr(h._h, p(A), 100, 4, 100, 1, 8, 0, 0, p(Q), 100, None, 4, 0, None) == -8
    assert lib.rxr_cholqr(h._h, p(A), 100, 4, 100, 1, 8, 0, 2, None, 100, None, 4, 0, None) == -9


def test_invalid_arguments_of_the_later_entry_points(h):
    lib = rxr.load()
    A = to_dev(usv_matrix(100, 4, 10, seed=0))
    b = to_dev(np.ones((100, 2)))
    Q = rxr.empty_colmajor(100, 4)
    x = rxr.empty_colmajor(4, 2)
    Y = rxr.empty_colmajor(8, 4)
    R = to_dev(np.eye(4))
    p = lambda t: t.data_ptr()
    # row extraction only with a sketch: not with RXR_NONE or RXR_SHIFTED
    assert lib.rxr_cholqr(h._h, p(A), 100, 4, 100, 2 | 16, 8, 0, 2, p(Q), 100, None, 4, 0, None) == -5
    assert lib.rxr_cholqr(h._h, p(A), 100, 4, 100, 3 | 16, 8, 0, 3, p(Q), 100, None, 4, 0, None) == -5
    # least squares: k in [1, 64], ldb >= m, LU or QR, x non-null
    ls = lambda k, ldb, v, xp: lib.rxr_lstsq(h._h, p(A), 100, 4, 100, p(b), k, ldb, v, 8, 0, xp, 4, 0, None)
    assert ls(0, 100, 1, p(x)) == -7
    assert ls(65, 100, 1, p(x)) == -7
    assert ls(2, 99, 1, p(x)) == -8
    assert ls(2, 100, 2, p(x)) == -9
    assert ls(2, 100, 1, None) == -12
    # row sketch: s >= 1, ldy >= s
    assert lib.rxr_sketch_rows(h._h, p(A), 100, 4, 100, 0, 0, p(Y), 8, None) == -6
    assert lib.rxr_sketch_rows(h._h, p(A), 100, 4, 100, 8, 0, p(Y), 7, None) == -9
    # X R^{-1}: ldx >= m, ldr >= n
    assert lib.rxr_apply_rinv(h._h, p(Q), 100, 4, 99, p(R), 4, 0, None) == -5
    assert lib.rxr_apply_rinv(h._h, p(Q), 100, 4, 100, p(R), 3, 0, None) == -7


# ------------------------------------------------------------------ async / graph / host / batched
def test_async_status_and_graph_capture(h):
    A = to_dev(usv_matrix(4000, 32, 1e10, seed=3))
    Q = rxr.empty_colmajor(4000, 32)
    R = rxr.empty_colmajor(32, 32)
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    h.cholqr_async(A, Q, R, st, variant="qr", seed=1)
    torch.cuda.synchronize()
    assert st.tolist() == [0, 0, 0, 0]
    Qb, Rb, _ = h.cholqr(A, variant="qr", seed=1)
    assert torch.equal(Q, Qb) and torch.equal(R, Rb)
    s = torch.cuda.Stream()
    Q2 = rxr.empty_colmajor(4000, 32)
    R2 = rxr.empty_colmajor(32, 32)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        h.cholqr_async(A, Q2, R2, st, variant="qr", seed=1, stream=s)   # warm-up outside capture
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            h.cholqr_async(A, Q2, R2, st, variant="qr", seed=1, stream=s)
    Q2.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(Q2, Qb) and torch.equal(R2, Rb)


def test_host_entry_point_matches_device(h):
    A = usv_matrix(3333, 20, 1e7, seed=4)
    Qh, Rh = h.cholqr_host(A, variant="lu", seed=2)
    Q, R, _ = h.cholqr(to_dev(A), variant="lu", seed=2)
    assert np.array_equal(Qh, to_host(Q)) and np.array_equal(Rh, to_host(R))


def test_batched_matches_single_calls(h):
    # one launch per stage for the whole batch; row chunks differ from the
    # single-call plan, so results agree to rounding (R-factor bound), not bitwise
    shapes = [(5000, 8, 1e3), (700, 16, 1e9), (4096, 32, 1e12), (129, 64, 1e5), (3000, 128, 1e2), (1, 1, 1.0),
              (40, 40, 1e4), (20000, 24, 1e15)]
    As_np = [usv_matrix(m, n, k, seed=i) for i, (m, n, k) in enumerate(shapes)]
    As = [to_dev(a) for a in As_np]
    Qs, Rs, st = h.cholqr_batched(As, variant="qr", seeds=list(range(len(As))))
    assert np.all(st == 0)
    for i, (A, (m, n, kappa)) in enumerate(zip(As, shapes)):
        Q, R, _ = h.cholqr(A, variant="qr", seed=i)
        Qb, Rb = to_host(Qs[i]), to_host(Rs[i])
        assert o.orth_error(Qb) <= 1e-13
        assert o.resid_error(As_np[i], Qb, Rb) <= 1e-14
        rel = np.linalg.norm(Rb - to_host(R)) / np.linalg.norm(to_host(R))
        assert rel <= max(100 * kappa * U, 1e-14), (i, rel)


@pytest.mark.parametrize("variant", ["lu", "none"])
def test_batched_mixed_statuses(h, variant):
    rng = np.random.default_rng(7)
    shapes = [(int(m), int(n)) for m, n in zip(rng.integers(64, 3000, 24), rng.choice([1, 3, 8, 16, 33, 64, 100], 24))]
    shapes = [(max(m, n), n) for m, n in shapes]
    As_np = [usv_matrix(m, n, 1e3, seed=i) for i, (m, n) in enumerate(shapes)]
    bad = {3: "nan", 11: "zero"}
    As_np[3] = As_np[3].copy(order="F")
    As_np[3][0, 0] = np.nan
    if shapes[11][1] > 1:
        As_np[11] = As_np[11].copy(order="F")
        As_np[11][:, -1] = 0.0
    As = [to_dev(a) for a in As_np]
    Qs, Rs, st = h.cholqr_batched(As, variant=variant)
    for i in range(len(As)):
        if i == 3:
            assert st[i, 0] == rxr.NONFINITE
        elif i == 11 and shapes[11][1] > 1:
            assert st[i, 0] in (rxr.SKETCH_SINGULAR, rxr.CHOL_BREAKDOWN)
        else:
            assert st[i, 0] == 0, (i, st[i])
            Qb, Rb = to_host(Qs[i]), to_host(Rs[i])
            assert o.orth_error(Qb) <= 1e-13 and o.resid_error(As_np[i], Qb, Rb) <= 1e-14


# ------------------------------------------------------------------ evaluators
def test_gpu_evaluators_match_oracle(h):
    A = usv_matrix(3000, 20, 1e6, seed=6)
    ref = o.rxr_cholqr(A, o.VARIANT_QR, 40, seed=0, passes=1)   # orthogonality ~1e-15..1e-14
    Qd, Rd = to_dev(ref.Q), to_dev(ref.R)
    e1 = h.orth_error(Qd)
    e2 = h.resid_error(to_dev(A), Qd, Rd)
    assert abs(e1 - o.orth_error(ref.Q)) <= 1e-3 * o.orth_error(ref.Q)
    assert abs(e2 - o.resid_error(A, ref.Q, ref.R)) <= 1e-3 * o.resid_error(A, ref.Q, ref.R)


# ------------------------------------------------------------------ wide panels (n > 128)
@pytest.mark.parametrize("m,n,kappa,variant,prec", [(400, 129, 1e4, "qr", "fp64"), (1000, 200, 1e8, "lu", "fp64"),
                                                    (700, 256, 1e12, "qr", "split"), (1500, 512, 1e13, "qr", "fp64"),
                                                    (1100, 512, 1e6, "lu", "split")])
def test_wide_panel_cholqr(h, m, n, kappa, variant, prec):
    A = usv_matrix(m, n, kappa, seed=n)
    Q, R, code = h.cholqr(to_dev(A), variant=variant, s=2 * n, seed=1, passes=2, prec=prec)
    assert code == 0
    Qg, Rg = to_host(Q), to_host(R)
    assert o.orth_error(Qg) <= 1e-13
    assert o.resid_error(A, Qg, Rg) <= 1e-14
    assert abs(h.orth_error(Q) - o.orth_error(Qg)) <= 1e-3 * o.orth_error(Qg) + 1e-30
    ref = o.rxr_cholqr(A, OV[variant], 2 * n, seed=1, passes=2)
    assert r_rel(Rg, ref.R) <= R_TOL


def test_wide_panel_precond_gram_parity(h):
    m, n = 777, 200
    A = usv_matrix(m, n, 1e3, seed=3)
    R = o.rxr_cholqr(A, o.VARIANT_QR, 2 * n, seed=2, passes=1).Rs
    X, G = h.precond_gram(to_dev(A), to_dev(R))
    Xg, Gg = to_host(X), to_host(G)
    Xo = o.trsm_right_upper(A, R)
    bound = 4 * n * U * (np.abs(Xo) @ np.abs(R) @ np.abs(np.linalg.inv(R))) + 1e-300
    assert np.all(np.abs(Xg - Xo) <= bound), np.max(np.abs(Xg - Xo) / bound)
    assert np.all(np.abs(Gg - o.gram(Xg)) <= 4 * (m + 2) * U * (np.abs(Xg).T @ np.abs(Xg)))


@pytest.mark.parametrize("m,n", [((1 << 18) + 77, 40), (300000, 64), (5000, 100)])
def test_host_entry_point_split_matches_device(h, m, n):
    # the split path brings A in row chunks (the sketch's CTAs of a chunk start
    # once it has landed) and sends Q out in row chunks after the last apply:
    # the same partition and arithmetic as the device-buffer call, bit for bit
    A = usv_matrix(m, n, 1e9, seed=n)
    Qh, Rh = h.cholqr_host(A, variant="qr", seed=3, prec="split")
    Q, R, code = h.cholqr(to_dev(A), variant="qr", seed=3, prec="split")
    assert code == 0
    assert np.array_equal(Qh, to_host(Q)) and np.array_equal(Rh, to_host(R))


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("m,n", [(2100, 100), (1000, 40), (3000, 70), (900, 52), (5000, 64), (4000, 128),
                                 (3000, 33), (700, 1)])
def test_preconditioner_quality(h, prec, m, n):
    # Theorem 3.4: with a Gaussian sketch of s = 2n rows, X = A R_s^{-1} is well
    # conditioned whatever cond(A) is.  The final QR is unique, so a weak
    # preconditioner would not show in the factorisation tests; this does.
    A = usv_matrix(m, n, 1e8, seed=n + 7)
    Y = h.sketch(to_dev(A), 2 * n, seed=3, prec=prec)
    Rs, code = h.xr_factor(Y, "qr")
    assert code == 0
    X = np.linalg.solve(to_host(Rs).T, A.T).T
    assert np.linalg.cond(X) <= 30
