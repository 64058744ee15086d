"""Pins for the oracle's multi-level stepping (Sec. 3.1, Eq. (kicks)).

Fixed by: kick counts computed by hand for a box of known cell densities
(tests/golden/ml_kick_counts.txt), the
reduction to one SKS step when every particle takes one kick, the reduction
to n SKS sub-cycles when every particle takes n kicks, and time reversibility
of the symmetric event schedule with fixed kick counts.
"""
import os

import numpy as np

import oracle
import synth


def _setup(n=1500, L=16.0, seed=61):
    pos = synth.blob_mixture(n, L, seed=seed, n_blobs=4, sigma=0.8)
    vel = synth.gaussian_velocities(n, seed=seed, sigma=0.05)
    return pos, vel, L


def _golden_kick_counts():
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "ml_kick_counts.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, levels, _ = line.split("|")
            d, lmin, lmax = (int(v) for v in head.split())
            rows.append((d, lmin, lmax, [int(v) for v in levels.split()]))
    return rows


def _class_box():
    """The box of the golden file: L = 8, 4^3 cells of width 2; 37 cells with 2
    particles, 24 empty, and cells with 4, 10 and 40; returns the FP32 rows and
    the class (0: mean, 1: x2, 2: x5, 3: x20) of every particle."""
    rng = np.random.default_rng(5)
    counts = {}
    cells = [(ix, iy, iz) for iz in range(4) for iy in range(4) for ix in range(4)]
    order = rng.permutation(len(cells))
    special = {cells[order[0]]: (4, 1), cells[order[1]]: (10, 2), cells[order[2]]: (40, 3)}
    for k in order[3:40]:
        counts[cells[k]] = (2, 0)
    counts.update(special)
    rows, cls = [], []
    for (ix, iy, iz), (m, c) in counts.items():
        # strictly inside the cell: (0.1, 1.9) of its width 2
        u = rng.uniform(0.1, 1.9, (m, 3))
        rows.append(u + 2.0 * np.array([ix, iy, iz], dtype=np.float64))
        cls += [c] * m
    x = np.concatenate(rows)
    perm = rng.permutation(len(x))
    pos = np.ones((len(x), 4), np.float32)
    pos[:, :3] = x[perm]
    return pos, np.array(cls)[perm]


def test_kick_counts_match_hand_computed_values():
    pos, cls = _class_box()
    assert len(pos) == 128 and np.bincount(cls).tolist() == [74, 4, 10, 40]
    rows = _golden_kick_counts()
    assert len(rows) >= 10
    for d, lmin, lmax, want in rows:
        lev = oracle.ml_levels(pos, 8.0, 4, d, lmax, lmin=lmin)
        got = [sorted(set(lev[cls == c].tolist())) for c in range(4)]
        assert got == [[w] for w in want], (d, lmin, lmax, got, want)


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
