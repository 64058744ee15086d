"""Pins for the oracle's multi-level stepping (Sec. 3.1, Eq. (kicks)).

Fixed by: the density rule recomputed by hand (numpy cell counts), the
reduction to one SKS step when every particle takes one kick, the reduction
to n SKS sub-cycles when every particle takes n kicks, and time reversibility
of the symmetric event schedule with fixed kick counts.
"""
import numpy as np

import oracle
import synth


def _setup(n=1500, L=16.0, seed=61):
    pos = synth.blob_mixture(n, L, seed=seed, n_blobs=4, sigma=0.8)
    vel = synth.gaussian_velocities(n, seed=seed, sigma=0.05)
    return pos, vel, L


def test_levels_follow_cell_density(split_params):
    pos, _, L = _setup()
    nc = 5
    for d, lmax in ((1, 4), (3, 3), (20, 4)):
        lev = oracle.ml_levels(pos, L, nc, d, lmax)
        _, cell, ok = oracle.wrap_cell(pos, L, nc)
        cnt = np.bincount(cell, minlength=nc ** 3)
        ratio = (cnt[cell].astype(np.int64) * nc ** 3) // len(pos)
        assert np.array_equal(lev, np.minimum(ratio // d + 1, lmax))
        for lmin in (2, lmax):
            lev = oracle.ml_levels(pos, L, nc, d, lmax, lmin=lmin)
            assert np.array_equal(lev, np.clip(ratio // d + 1, lmin, lmax))
    assert np.all(oracle.ml_levels(pos, L, nc, 0, 3) == 3)
    assert np.all(oracle.ml_levels(pos, L, nc, 0, 3, lmin=2) == 3)


def test_single_kick_is_one_sks_step(split_params):
    pos, vel, L = _setup()
    lev = np.ones(len(pos), np.int32)
    x1, v1 = oracle.subcycle_ml(pos, vel, L, split_params, 0.2, 3, lev)
    x2, v2 = oracle.subcycle(pos, vel, L, split_params, 0.2, 1)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)


def test_uniform_kicks_equal_sks_subcycles(split_params):
    pos, vel, L = _setup()
    for k in (2, 3, 4):
        lev = np.full(len(pos), k, np.int32)
        x1, v1 = oracle.subcycle_ml(pos, vel, L, split_params, 0.2, k, lev)
        x2, v2 = oracle.subcycle(pos, vel, L, split_params, 0.2, k)
        d = x1 - x2
        d -= L * np.round(d / L)
        # same maps; only the rounding differs (one stream of h between kicks
        # here, two of h/2 there)
        assert np.abs(d).max() < 1e-9 and np.abs(v1 - v2).max() < 1e-9


def test_mixed_levels_reversible(split_params):
    pos, vel, L = _setup()
    sp = dict(split_params, eps=0.05)
    lev = oracle.ml_levels(pos, L, 5, 2, 4)
    assert len(np.unique(lev)) > 1
    x1, v1 = oracle.subcycle_ml(pos, vel, L, sp, 0.3, 4, lev)
    p1 = np.concatenate([x1, pos[:, 3:]], 1)
    x2, v2 = oracle.subcycle_ml(p1, -v1, L, sp, 0.3, 4, lev)
    d = x2 - pos[:, :3]
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-9 and np.abs(-v2 - vel[:, :3]).max() < 1e-9
