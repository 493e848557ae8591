"""Batched plans (rxr_batch_create / rxr_batch_run): a set of problems with
the batched workload's spread of shapes and conditionings, prepared once and
run repeatedly, each problem's Q and R checked against the oracle's
rQR-/rLU-CholeskyQR2 (Algorithms 4/5 with Algorithm 2).

* FP64 over the persistent stage kernels (work-queue items of every problem
  in one launch per stage) and the per-problem form of the split precision;
* a run is asynchronous: captured into a CUDA graph and replayed it gives the
  same bits as a plain run, after the inputs change in place too;
* consecutive runs give the same bits (the work queue's order does not change
  the arithmetic: each item's partial sum has a fixed slot)."""
import numpy as np
import pytest

import oracle as o
from gpu_util import R_TOL, r_rel, to_dev, to_host
from paper_2111_11148_gb300.inputs import batch_specs, usv_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402

OV = {"lu": o.VARIANT_LU, "qr": o.VARIANT_QR}


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


def _problems(count, seed, log2m=(7, 15)):
    specs = batch_specs(count, seed=seed, log2m=log2m)
    return specs, [usv_matrix(sp.m, sp.n, sp.kappa, seed=sp.seed) for sp in specs]


def _against_oracle(specs, As_np, plan, variant):
    st = plan.status.cpu().numpy()
    assert np.all(st[:, 0] == 0), st[st[:, 0] != 0][:4]
    for i, sp in enumerate(specs):
        Qg, Rg = to_host(plan.Qs[i]), to_host(plan.Rs[i])
        assert o.orth_error(Qg) <= 1e-13 and o.resid_error(As_np[i], Qg, Rg) <= 1e-14, (i, sp)
        ref = o.rxr_cholqr(As_np[i], OV[variant], 2 * sp.n, seed=sp.seed, passes=2)
        assert r_rel(Rg, ref.R) <= R_TOL, (i, sp)


@pytest.mark.parametrize("prec,variant", [("fp64", "qr"), ("fp64", "lu"), ("split", "qr"), ("split_precond", "lu")])
def test_plan_runs_match_the_oracle_and_each_other(h, prec, variant):
    specs, As_np = _problems(40 if prec == "fp64" else 24, seed=1 if variant == "qr" else 2)
    As = [to_dev(a) for a in As_np]
    plan = h.batch_plan(As, variant=variant, seeds=[sp.seed for sp in specs], prec=prec)
    try:
        plan.run()
        torch.cuda.synchronize()
        _against_oracle(specs, As_np, plan, variant)
        Q1 = [q.clone() for q in plan.Qs]
        R1 = [r.clone() for r in plan.Rs]
        for q in plan.Qs:
            q.zero_()
        plan.run()
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(Q1, plan.Qs))
        assert all(torch.equal(a, b) for a, b in zip(R1, plan.Rs))
    finally:
        plan.close()


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_plan_run_is_graph_capturable(h, prec):
    specs, As_np = _problems(16, seed=3)
    As = [to_dev(a) for a in As_np]
    plan = h.batch_plan(As, variant="qr", seeds=[sp.seed for sp in specs], prec=prec)
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            plan.run(stream=s)  # first run outside the capture
            s.synchronize()
            Q0 = [q.clone() for q in plan.Qs]
            R0 = [r.clone() for r in plan.Rs]
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                plan.run(stream=s)
        for q in plan.Qs:
            q.zero_()
        plan.status.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert (plan.status[:, 0] == 0).all()
        assert all(torch.equal(a, b) for a, b in zip(Q0, plan.Qs))
        assert all(torch.equal(a, b) for a, b in zip(R0, plan.Rs))
        # new inputs in place: the replay factorises them
        A2 = [usv_matrix(sp.m, sp.n, 10.0, seed=sp.seed + 100) for sp in specs]
        for a, a2 in zip(As, A2):
            a.copy_(torch.from_numpy(a2))
        g.replay()
        torch.cuda.synchronize()
        for i, sp in enumerate(specs):
            ref = o.rxr_cholqr(A2[i], o.VARIANT_QR, 2 * sp.n, seed=sp.seed, passes=2)
            assert r_rel(to_host(plan.Rs[i]), ref.R) <= R_TOL
    finally:
        plan.close()


def test_plan_argument_errors(h):
    lib = rxr.load()
    import ctypes

    p = ctypes.c_void_p()
    assert lib.rxr_batch_create(None, 1, None, None, None, None, 1, None, None, 2, None, None, None, None, 0, None,
                                ctypes.byref(p)) == -1
    assert lib.rxr_batch_run(None, None) == -1
    assert lib.rxr_batch_destroy(None) == 0
    A = to_dev(usv_matrix(300, 200, 10.0, seed=0))
    with pytest.raises(rxr.RxrError):  # the FP64 stage kernels take n <= 128
        h.batch_plan([A], variant="qr")
