"""Writes the stored expected values under tests/golden/ by calling the CPU
oracle only (never the CUDA path).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as o  # noqa: E402

# (seed, first row i0, rows, s): includes a row index above 2^32 (counter high word)
OMEGA_CASES = [(0, 0, 3, 12), (1, 1000003, 2, 9), (0xFFFFFFFF12345678, 2**32 + 5, 2, 8)]


def write_omega():
    with open(os.path.join(HERE, "omega_z.txt"), "w") as f:
        f.write("# z values of the Gaussian sketch (Section 2.3), float32 bit patterns.\n")
        f.write("# seed i s r bits  -- written by tests/golden/make_golden.py from the CPU oracle\n")
        for seed, i0, rows, s in OMEGA_CASES:
            z = o.omega_z(seed, s, i0, rows)
            for i in range(rows):
                for r in range(s):
                    bits = int(np.float32(z[i, r]).view(np.uint32))
                    f.write(f"{seed} {i0 + i} {s} {r} {bits:08x}\n")


def write_small_case():
    rng = np.random.default_rng(2024)
    m, n, s = 48, 4, 8
    q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    A = np.asfortranarray(q @ np.diag([1.0, 1e-2, 1e-4, 1e-6]) @ np.linalg.qr(rng.standard_normal((n, n)))[0])
    out = {}
    for v, name in ((o.VARIANT_LU, "lu"), (o.VARIANT_QR, "qr")):
        r = o.rxr_cholqr(A, v, s, seed=5, passes=2)
        assert r.status == 0
        out[name] = r
    with open(os.path.join(HERE, "small_case.txt"), "w") as f:
        f.write("# 48 x 4 matrix A (cond 1e6) and the oracle's R factors for s = 8, seed 5, 2 passes.\n")
        f.write("# Values are float64 hex (float.hex). Written by tests/golden/make_golden.py.\n")
        f.write(f"A {m} {n}\n")
        for j in range(n):
            f.write(" ".join(float(x).hex() for x in A[:, j]) + "\n")
        for name in ("lu", "qr"):
            for key in ("Rs", "R"):
                M = getattr(out[name], key)
                f.write(f"{name}_{key} {n} {n}\n")
                for j in range(n):
                    f.write(" ".join(float(x).hex() for x in M[:, j]) + "\n")


if __name__ == "__main__":
    write_omega()
    write_small_case()
