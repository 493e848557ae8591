"""Every kernel writes what it later reads: with the handle's workspace handed
over filled with NaN (rxr_set_workspace), single and batched factorisations
give the same bits as with a fresh workspace, on both precisions.  A read of
scratch that the call itself did not write first shows up here as NaN."""
import numpy as np
import pytest

from gpu_util import to_dev, to_host
from paper_2111_11148_gb300.inputs import batch_specs, usv_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402


def _poisoned(nbytes):
    return torch.full((nbytes // 8 + 1,), float("nan"), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec", ["fp64", "split", "split_precond"])
@pytest.mark.parametrize("m,n,variant", [(20000, 16, "lu"), (140000, 64, "qr"), (5000, 100, "qr"),
                                         (3000, 200, "lu"), (777, 9, "none")])
def test_poisoned_workspace_single(prec, m, n, variant):
    A = to_dev(usv_matrix(m, n, 1e9 if variant != "none" else 1e3, seed=n))
    with rxr.Handle(0) as h:
        Q0, R0, c0 = h.cholqr(A, variant=variant, seed=3, prec=prec)
    with rxr.Handle(0) as h:
        h.set_workspace(_poisoned(rxr.workspace_bytes(m, n, 2 * n, prec)))
        Q1, R1, c1 = h.cholqr(A, variant=variant, seed=3, prec=prec)
        Q2, R2, c2 = h.cholqr(A, variant=variant, seed=3, prec=prec)   # and with the first call's leftovers
        h.set_workspace(None)
    assert c0 == c1 == c2 == 0
    assert torch.equal(Q0, Q1) and torch.equal(R0, R1) and torch.equal(Q0, Q2) and torch.equal(R0, R2)


def test_poisoned_workspace_batched():
    specs = batch_specs(48, seed=0, log2m=(7, 15))
    As = [to_dev(usv_matrix(sp.m, sp.n, sp.kappa, seed=sp.seed)) for sp in specs]
    seeds = [sp.seed for sp in specs]
    with rxr.Handle(0) as h:
        Q0, R0, s0 = h.cholqr_batched(As, variant="qr", seeds=seeds)
    with rxr.Handle(0) as h:
        h.set_workspace(_poisoned(1 << 30))
        Q1, R1, s1 = h.cholqr_batched(As, variant="qr", seeds=seeds)
        h.set_workspace(None)
    assert np.all(s0 == 0) and np.all(s1 == 0)
    bad = [i for i in range(len(As)) if not (torch.equal(Q0[i], Q1[i]) and torch.equal(R0[i], R1[i]))]
    assert not bad, [(i, specs[i]) for i in bad]
