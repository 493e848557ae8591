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
