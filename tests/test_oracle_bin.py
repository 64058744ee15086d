"""Pins for the oracle's periodic wrap, chaining-mesh cell rule and counting sort.

The cell rule (largest k with k L <= x nc, on the FP32 value, exact) is
checked against Python's exact rational arithmetic; the counting sort against
numpy's stable argsort; the candidate count against a brute-force loop.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def _exact_cell(x: np.float32, L: float, nc: int) -> int:
    k = (Fraction(float(x)) * nc) // Fraction(float(L))
    return int(min(max(k, 0), nc - 1))


def _exact_wrap(x: np.float32, L: float) -> np.float32:
    Lf = np.float32(L)
    v = np.float32(x)
    if v < 0:
        v = np.float32(v + Lf)
    elif v >= Lf:
        v = np.float32(v - Lf)
    if v >= Lf:
        v = np.float32(0.0)
    return v


@pytest.mark.parametrize("L,nc", [(32.0, 10), (256.0, 82), (float(np.float32(45.254834)), 14), (10.0, 3)])
def test_cell_rule_exact_on_boundaries(L, nc):
    rng = np.random.default_rng(7)
    xs = list(rng.uniform(0, L, 300).astype(np.float32))
    # faces k L / nc exactly where representable, and the floats right around them
    for k in range(nc + 1):
        b = np.float32(k * L / nc)
        for v in (np.nextafter(b, np.float32(-1e9)), b, np.nextafter(b, np.float32(1e9))):
            if 0 <= v < np.float32(L):
                xs.append(np.float32(v))
    xs += [np.float32(-1e-9), np.float32(-L), np.float32(L), np.float32(2 * L) - np.float32(1e-3),
           np.float32(-0.5), np.float32(L + 0.25)]
    n = len(xs)
    pos = np.zeros((n, 4), np.float32)
    pos[:, 0] = xs
    pos[:, 1] = xs[::-1]
    pos[:, 2] = np.roll(np.array(xs, np.float32), 5)
    wrapped, cell, ok = oracle.wrap_cell(pos, L, nc)
    assert ok
    for i in range(n):
        w = [_exact_wrap(pos[i, a], L) for a in range(3)]
        assert all(0 <= v < np.float32(L) for v in w)
        assert [wrapped[i, a] for a in range(3)] == w
        ix, iy, iz = (_exact_cell(v, L, nc) for v in w)
        assert cell[i] == (iz * nc + iy) * nc + ix


def test_wrap_rounding_up_to_L_goes_to_zero():
    pos = np.array([[-1e-9, 0.5, 0.5, 1.0]], np.float32)
    w, cell, ok = oracle.wrap_cell(pos, 256.0, 82)
    assert ok and w[0, 0] == 0.0 and cell[0] % 82 == 0


@pytest.mark.parametrize("bad", [np.nan, np.inf, -256.001, 512.0])
def test_wrap_rejects_out_of_range(bad):
    pos = np.array([[1.0, 1.0, 1.0, 1.0], [bad, 1.0, 1.0, 1.0]], np.float32)
    _, cell, ok = oracle.wrap_cell(pos, 256.0, 82)
    assert not ok and cell[1] == -1 and cell[0] >= 0


def test_counting_sort_is_stable_and_complete():
    pos = synth.blob_mixture(5000, 16.0, seed=3)
    _, cell, ok = oracle.wrap_cell(pos, 16.0, 5)
    assert ok
    count, start, perm = oracle.bin_cells(cell, 5)
    assert count.sum() == 5000 and start[-1] == 5000
    assert np.array_equal(perm, np.argsort(cell, kind="stable"))
    assert np.array_equal(np.diff(start), count)
    assert np.array_equal(np.bincount(cell, minlength=125), count)


def test_candidate_count_brute_force():
    nc, L = 4, 13.0
    pos = synth.blob_mixture(300, L, seed=11, n_blobs=3)
    _, cell, ok = oracle.wrap_cell(pos, L, nc)
    count, _, _ = oracle.bin_cells(cell, nc)
    ix, iy, iz = cell % nc, (cell // nc) % nc, cell // (nc * nc)

    def near(a, b):
        d = (a - b) % nc
        return d == 0 or d == 1 or d == nc - 1

    brute = 0
    for i in range(300):
        for j in range(300):
            if near(ix[i], ix[j]) and near(iy[i], iy[j]) and near(iz[i], iz[j]):
                brute += 1
    assert oracle.candidates(count, nc) == brute
