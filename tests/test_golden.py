"""Stored values: the paper's constants (cited in paper_constants.txt) and
regression fixtures written from the CPU oracle by tests/golden/make_golden.py."""
import math
import os

import numpy as np

import oracle as o

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_constants():
    out = {}
    for line in open(os.path.join(GOLD, "paper_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, val = line.split()[:2]
        out[name] = float(val)
    return out


def read_omega():
    rows = []
    for line in open(os.path.join(GOLD, "omega_z.txt")):
        if line.startswith("#"):
            continue
        seed, i, s, r, bits = line.split()
        rows.append((int(seed), int(i), int(s), int(r), int(bits, 16)))
    return rows


def read_small_case():
    mats, lines = {}, open(os.path.join(GOLD, "small_case.txt")).read().splitlines()
    k = 0
    while k < len(lines):
        if lines[k].startswith("#"):
            k += 1
            continue
        name, r, c = lines[k].split()
        r, c = int(r), int(c)
        cols = [[float.fromhex(t) for t in lines[k + 1 + j].split()] for j in range(c)]
        mats[name] = np.asfortranarray(np.array(cols).T)
        k += 1 + c
    return mats


def test_paper_constants_follow_from_the_formulas():
    c = read_constants()
    f = lambda r: (3 + math.sqrt(1 / r)) / (1 - math.sqrt(1 / r))   # Theorem 3.4 threshold at l = r n
    assert abs(f(2.0) - c["thm34_threshold_l_2n"]) < 1e-12
    assert abs(f(1.1) - c["remark35_threshold_l_1.1n"]) < 1e-4
    assert f(1.1) < c["remark35_ceiling"]


def test_oracle_reproduces_stored_normals():
    for seed, i, s, r, bits in read_omega():
        z = o.omega_z(seed, s, i, 1)[0, r]
        assert int(np.float32(z).view(np.uint32)) == bits, (seed, i, s, r)


def test_oracle_reproduces_stored_small_case():
    g = read_small_case()
    A = g["A"]
    for v, name in ((o.VARIANT_LU, "lu"), (o.VARIANT_QR, "qr")):
        r = o.rxr_cholqr(A, v, 8, seed=5, passes=2)
        assert r.status == 0
        for key in ("Rs", "R"):
            ref = g[f"{name}_{key}"]
            np.testing.assert_allclose(getattr(r, key), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
