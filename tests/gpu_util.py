"""Helpers shared by the GPU tests: device transfer of column-major matrices
and the handle fixture.  Inputs always come from paper_2111_11148_gb300.inputs
or numpy; expected values always from the CPU oracle (or LAPACK)."""
import numpy as np


def to_dev(a: np.ndarray, ld: int | None = None):
    import torch

    from paper_2111_11148_gb300 import rxr

    t = torch.from_numpy(np.asfortranarray(np.asarray(a, dtype=np.float64)))
    return rxr.colmajor(t.cuda(), ld=ld)


def to_host(t) -> np.ndarray:
    return np.asfortranarray(t.detach().cpu().numpy())


U = 2.0**-53

# ||R_a - R_b||_F / ||R||_F between independent correct FP64 implementations
# of the thin QR (the oracle's rQR/rLU-CholeskyQR2, the oracle's Householder QR,
# LAPACK's geqrf), measured on the tests' inputs A = U diag(sigma) V^T with
# kappa = 1e2 .. 1e15: 2e-16 .. 8e-15 at m = 5000 .. 20000, n = 16 .. 64, and
# up to 4.1e-14 against LAPACK at m = 2^22 .. 2^23, n = 64 .. 128, with no
# growth in kappa (the R-factor perturbation bound kappa u is a worst case that
# these inputs do not approach).  Every R comparison asserts 1e-12, 24 times
# the largest measured spread, which also meets 1e-11 at kappa <= 1e8.
R_SPREAD = 4.1e-14
R_TOL = 1e-12


def r_rel(Ra, Rb) -> float:
    """||Ra - Rb||_F / ||Rb||_F."""
    return float(np.linalg.norm(Ra - Rb) / np.linalg.norm(Rb))
