"""The row-sharded factorisation through the library's kernels (rxr_sketch_part,
rxr_sum_parts, rxr_trmm_upper and the stage calls), its shards run as threads
of one process on the one GPU, each with its own handle, exchanging their
partials through the host (no kernel waits on another).

* every shard ends with the same R, bit for bit, and the stacked Q and R meet
  Section 4.2's targets, with R within R_TOL of the oracle's and of the
  single-call factorisation's, on both precisions and both variants;
* the partial sketches add up to the whole sketch (Omega follows the global
  rows), against the oracle's shard sketches;
* rxr_sum_parts sums in the order of the blocks (bit-equal to a sequential
  sum), rxr_trmm_upper equals the oracle's product."""
import threading

import numpy as np
import pytest

import oracle as o
from gpu_util import R_TOL, U, r_rel, to_dev, to_host
from paper_2111_11148_gb300.inputs import usv_matrix
from shard_util import ThreadGather, shard_bounds

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402
from paper_2111_11148_gb300.sharded import LibraryOps, cholqr_sharded  # noqa: E402


def _run_shards(A_np, world, variant, prec, seed=3):
    m, n = A_np.shape
    tg = ThreadGather(world, lambda blocks: torch.stack([b.t().contiguous() for b in blocks]))
    res = [None] * world
    errs = []

    def run(rank):
        try:
            r0, r1 = shard_bounds(m, world)[rank]
            with rxr.Handle(0) as h:
                A = to_dev(A_np[r0:r1])
                Q, R, code = cholqr_sharded(LibraryOps(h), A, r0, tg.for_rank(rank), variant=variant, seed=seed,
                                            prec=prec)
                torch.cuda.synchronize()
                res[rank] = (to_host(Q), to_host(R), code)
        except Exception as e:  # reported by the main thread
            errs.append(e)
            tg.barrier.abort()

    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs
    return res


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("world,variant,m,n,kappa", [(2, "qr", 60001, 64, 1e12), (3, "lu", 30000, 16, 1e8),
                                                     (2, "qr", 20002, 128, 1e14), (4, "qr", 9000, 33, 1e6)])
def test_shards_factorise_the_whole_matrix(prec, world, variant, m, n, kappa):
    A = usv_matrix(m, n, kappa, seed=world + n)
    res = _run_shards(A, world, variant, prec)
    assert [r[2] for r in res] == [0] * world
    R = res[0][1]
    for r in range(1, world):
        assert np.array_equal(res[r][1], R)
    Q = np.vstack([r[0] for r in res])
    assert o.orth_error(Q) <= 1e-13 and o.resid_error(A, Q, R) <= 1e-14
    ref = o.rxr_cholqr(A, o.VARIANT_QR if variant == "qr" else o.VARIANT_LU, 2 * n, seed=3, passes=2)
    assert r_rel(R, ref.R) <= R_TOL
    with rxr.Handle(0) as h:
        _, R1, code = h.cholqr(to_dev(A), variant=variant, seed=3, prec=prec)
    assert code == 0 and r_rel(R, to_host(R1)) <= R_TOL


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_shard_sketches_sum_to_the_whole(prec):
    m, n, s, seed = 50000, 24, 48, 9
    A = usv_matrix(m, n, 1e6, seed=1)
    cuts = [0, 12345, 30000, m]
    with rxr.Handle(0) as h:
        parts = [h.sketch_part(to_dev(A[a:b]), s, seed=seed, row0=a, prec=prec) for a, b in zip(cuts, cuts[1:])]
        total = to_host(h.sum_parts(torch.stack([p.t().contiguous() for p in parts])).t())
        whole = to_host(h.sketch(to_dev(A), s, seed=seed, prec=prec))
    if prec == "fp64":
        ref = sum(o.sketch(A[a:b], s, seed, row0=a) for a, b in zip(cuts, cuts[1:]))
    else:  # the split sketch's Omega on the 2^-12 grid (the oracle's quantised sketch)
        ref = o.sketch_quantised(A, s, seed)
    scale = np.abs(o.omega(seed, s, m)) @ np.abs(A)
    assert np.all(np.abs(total - ref) <= 64 * np.log2(m) * U * scale + 2.0**-50 * np.abs(A).max() * m)
    assert np.all(np.abs(total - whole) <= 64 * np.log2(m) * U * scale + 2.0**-50 * np.abs(A).max() * m)


def test_sum_parts_and_trmm():
    rng = np.random.default_rng(4)
    blocks = rng.standard_normal((5, 37, 11))
    with rxr.Handle(0) as h:
        out = h.sum_parts(torch.from_numpy(blocks).cuda()).cpu().numpy()
        seq = blocks[0].copy()
        for k in range(1, 5):
            seq = seq + blocks[k]
        assert np.array_equal(out, seq)
        Ra = np.triu(rng.standard_normal((70, 70))) + 5 * np.eye(70)
        Rb = np.triu(rng.standard_normal((70, 70))) + 5 * np.eye(70)
        C = to_host(h.trmm_upper(to_dev(Ra), to_dev(Rb)))
    ref = o.trmm_upper(Ra, Rb)
    assert np.all(np.tril(C, -1) == 0)
    assert np.max(np.abs(C - ref)) <= 140 * U * np.max(np.abs(Ra) @ np.abs(Rb))
