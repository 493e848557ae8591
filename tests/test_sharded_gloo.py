"""The row-sharded factorisation's protocol (Section 2.4's parallel scheme:
shard-local sketch and Gram partials, one allgather per stage summed in rank
order, the small factorisations on every shard) on CPU: two and three gloo
ranks, each factorising its row block with the oracle's steps.

* every rank ends with the same R, bit for bit;
* the stacked Q and R are the thin QR of the whole A (Section 4.2's measures),
  with R within R_TOL of the single-process oracle's;
* the gloo run gives the same bits as the same shards run as threads of one
  process (the result depends on the partition only, not on the transport);
* one shard is the oracle's own factorisation, bit for bit."""
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle as o  # noqa: E402
from gpu_util import R_TOL, r_rel  # noqa: E402
from paper_2111_11148_gb300.inputs import usv_matrix  # noqa: E402
from paper_2111_11148_gb300.sharded import cholqr_sharded  # noqa: E402
from shard_util import OracleOps, ThreadGather, gloo_gather_numpy, shard_bounds  # noqa: E402

M, N, KAPPA = 6001, 12, 1e10


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, variant, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        A = usv_matrix(M, N, KAPPA, seed=3)
        r0, r1 = shard_bounds(M, world)[rank]
        Q, R, code = cholqr_sharded(OracleOps(), np.asfortranarray(A[r0:r1]), r0, gloo_gather_numpy(),
                                    variant=variant, seed=5)
        out[rank] = (code, Q, R)
    finally:
        dist.destroy_process_group()


def _threads(world, variant):
    A = usv_matrix(M, N, KAPPA, seed=3)
    tg = ThreadGather(world, lambda blocks: np.stack([np.asfortranarray(b).T for b in blocks]))
    res = [None] * world
    import threading

    def run(rank):
        r0, r1 = shard_bounds(M, world)[rank]
        res[rank] = cholqr_sharded(OracleOps(), np.asfortranarray(A[r0:r1]), r0, tg.for_rank(rank),
                                   variant=variant, seed=5)

    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return res


@pytest.mark.parametrize("world,variant", [(2, "qr"), (3, "lu")])
def test_gloo_ranks_factorise_their_row_blocks(world, variant):
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), variant, out), nprocs=world, join=True)
    codes = [out[r][0] for r in range(world)]
    assert codes == [0] * world
    Rs = [out[r][2] for r in range(world)]
    for r in range(1, world):
        assert np.array_equal(Rs[r], Rs[0])
    A = usv_matrix(M, N, KAPPA, seed=3)
    Q = np.vstack([out[r][1] for r in range(world)])
    assert o.orth_error(Q) <= 1e-13
    assert o.resid_error(A, Q, Rs[0]) <= 1e-14
    ref = o.rxr_cholqr(A, o.VARIANT_QR if variant == "qr" else o.VARIANT_LU, 2 * N, seed=5, passes=2)
    assert r_rel(Rs[0], ref.R) <= R_TOL
    # the same shards as threads of one process: the same bits
    th = _threads(world, variant)
    for r in range(world):
        Qt, Rt, ct = th[r]
        assert ct == 0
        assert np.array_equal(Qt, out[r][1]) and np.array_equal(Rt, out[r][2])


def test_one_shard_is_the_oracle_factorisation():
    # a single shard sums one partial: the same arithmetic as the oracle's own
    # factorisation, bit for bit
    A = usv_matrix(M, N, KAPPA, seed=3)
    tg = ThreadGather(1, lambda blocks: np.stack([np.asfortranarray(b).T for b in blocks]))
    Q, R, code = cholqr_sharded(OracleOps(), np.asfortranarray(A), 0, tg.for_rank(0), variant="qr", seed=5)
    assert code == 0
    ref = o.rxr_cholqr(A, o.VARIANT_QR, 2 * N, seed=5, passes=2)
    assert np.array_equal(R, ref.R) and np.array_equal(Q, ref.Q)
