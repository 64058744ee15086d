"""Pins for the oracle's short-range force sums (Sec. 3.1, Eq. (force)).

What fixes the answer here: the plain all-pairs definition (brute force), the
cell list reproducing its exact pair set, Newton's third law, the symmetry of
a perfect lattice, the two-body Plummer law, and the periodic minimum image.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import split


@pytest.mark.parametrize("L,n,seed", [(10.0, 600, 1), (12.0, 1500, 2), (16.0, 2500, 3), (9.5, 400, 4)])
def test_cell_list_reproduces_brute_force(split_params, L, n, seed):
    pos = synth.blob_mixture(n, L, seed=seed, n_blobs=6)
    pos[:, 3] = np.random.default_rng(seed).uniform(0.5, 2.0, n).astype(np.float32)
    ab, wb = oracle.force_brute(pos, L, split_params)
    am, wm = oracle.force_mesh(pos, L, split_params)
    assert wb == wm and wb > 0
    scale = np.sqrt((ab ** 2).sum(1).mean())
    assert np.abs(am - ab).max() <= 1e-12 * scale * 10
    sel = np.array([0, n // 3, n - 1, 7], np.int64)
    asel, _ = oracle.force_mesh(pos, L, split_params, sel=sel)
    assert np.abs(asel - ab[sel]).max() <= 1e-11 * scale


def test_small_box_falls_back_to_brute_force(split_params):
    L = 8.0                          # fewer than 3 cells of width r_cut per side
    pos = synth.uniform(200, L, seed=5)
    ab, wb = oracle.force_brute(pos, L, split_params)
    am, wm = oracle.force_mesh(pos, L, split_params)
    assert wb == wm
    assert np.abs(am - ab).max() < 1e-12 * np.abs(ab).max()


@pytest.mark.parametrize("masses", ["equal", "random"])
def test_newton_third_law(split_params, masses):
    pos = synth.blob_mixture(3000, 20.0, seed=9)
    if masses == "random":
        pos[:, 3] = np.random.default_rng(1).uniform(0.1, 3.0, len(pos)).astype(np.float32)
    a, _ = oracle.force_mesh(pos, 20.0, split_params)
    m = pos[:, 3].astype(np.float64)
    net = (m[:, None] * a).sum(0)
    total = (m[:, None] * np.abs(a)).sum()
    assert np.abs(net).max() < 1e-13 * total


def test_lattice_has_zero_force(split_params):
    pos = synth.lattice(12)            # one particle per unit cell, L = 12
    a, w = oracle.force_mesh(pos, 12.0, split_params)
    assert w > 0
    assert np.abs(a).max() < 1e-12


def test_two_body_plummer_law(split_params):
    # one pair: the force on i points to j with magnitude m_j (r f_SR), and
    # r f_SR = softened Newton - grid force within the P5 fit residual
    sp = split_params
    rng = np.random.default_rng(4)
    L = 20.0
    for r in (0.02, 0.3, 1.0, 2.5, 3.0):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pos = np.array([[5.0, 5.0, 5.0, 1.0], [0, 0, 0, 2.5]], np.float64)
        pos[1, :3] = pos[0, :3] + r * u
        a, w = oracle.force_brute(pos, L, sp)
        assert w == 2
        mag = np.linalg.norm(a[0])
        expect = 2.5 * (r / (r * r + sp["eps"]) ** 1.5 - float(split.f_grid(r)))
        assert abs(mag - expect) <= 2.5 * 1e-3 / (r * r)
        assert np.dot(a[0], u) > 0                         # attractive, toward j
        assert np.allclose(a[1] * 2.5, -a[0] * 1.0, rtol=1e-13, atol=0)  # m1 a1 = -m0 a0


def test_minimum_image_across_the_boundary(split_params):
    L = 16.0
    pos = np.array([[0.1, 8.0, 8.0, 1.0], [L - 0.2, 8.0, 8.0, 1.0]], np.float64)
    a, w = oracle.force_brute(pos, L, split_params)
    assert w == 2
    assert a[0, 0] < 0 and a[1, 0] > 0                   # separation is 0.3, through the face
    ref = np.array([[0.1, 8.0, 8.0, 1.0], [-0.2, 8.0, 8.0, 1.0]], np.float64)
    ref[:, 0] += 4.0
    b, _ = oracle.force_brute(ref, L, split_params)
    assert np.allclose(a, b, rtol=1e-12, atol=0)


def test_cutoff_is_sharp(split_params):
    sp = split_params
    rc = sp["r_cut"]
    L = 20.0
    for r, inside in ((rc * (1 - 1e-9), True), (rc * (1 + 1e-12), False), (rc + 0.5, False)):
        pos = np.array([[5.0, 5.0, 5.0, 1.0], [5.0 + r, 5.0, 5.0, 1.0]], np.float64)
        a, w = oracle.force_brute(pos, L, sp)
        assert (w == 2) == inside
        if not inside:
            assert np.all(a == 0.0)


def test_force_scales_with_partner_mass_and_G(split_params):
    sp = dict(split_params)
    pos = synth.uniform(400, 12.0, seed=8).astype(np.float64)
    a1, _ = oracle.force_brute(pos, 12.0, sp)
    pos2 = pos.copy()
    pos2[:, 3] *= 3.0
    sp2 = dict(sp, G=0.5)
    a2, _ = oracle.force_brute(pos2, 12.0, sp2)
    assert np.allclose(a2, 1.5 * a1, rtol=1e-12, atol=1e-12)
