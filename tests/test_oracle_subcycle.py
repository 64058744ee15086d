"""Pins for the oracle's short-range sub-cycle (Sec. 2.5, SKS maps).

A symmetric stream-kick-stream composition is time reversible and second-order
accurate, and with a pair force that obeys Newton's third law it conserves
momentum exactly; energy error of a symplectic map stays bounded and scales
as h^2.  Each of those is checked on small boxes.
"""
import numpy as np
import pytest

import oracle
import synth


def _state(n=800, L=12.0, seed=21):
    pos = synth.blob_mixture(n, L, seed=seed, n_blobs=4, sigma=0.8)
    vel = synth.gaussian_velocities(n, seed=seed, sigma=0.05)
    return pos.astype(np.float64), vel.astype(np.float64), L


def _min_image_diff(x, y, L):
    d = x - y
    return d - L * np.round(d / L)


def test_time_reversible(split_params):
    pos, vel, L = _state()
    x1, v1 = oracle.subcycle(pos, vel, L, split_params, dt=0.2, nsub=4)
    p1 = np.concatenate([x1, pos[:, 3:]], axis=1)
    x2, v2 = oracle.subcycle(p1, -v1, L, split_params, dt=0.2, nsub=4)
    assert np.abs(_min_image_diff(x2, pos[:, :3], L)).max() < 1e-9
    assert np.abs(-v2 - vel[:, :3]).max() < 1e-9


def test_momentum_conserved(split_params):
    pos, vel, L = _state(seed=22)
    pos[:, 3] = np.random.default_rng(0).uniform(0.5, 1.5, len(pos))
    m = pos[:, 3]
    x1, v1 = oracle.subcycle(pos, vel, L, split_params, dt=0.3, nsub=5)
    p0 = (m[:, None] * vel[:, :3]).sum(0)
    p1 = (m[:, None] * v1).sum(0)
    assert np.abs(p1 - p0).max() < 1e-11


def test_second_order_convergence(split_params):
    # smooth regime (softening 0.1 keeps every encounter resolved at these h):
    # halving h cuts the error by 4
    sp = dict(split_params, eps=0.1)
    L = 12.0
    pos = synth.uniform(300, L, seed=23).astype(np.float64)
    vel = synth.gaussian_velocities(300, seed=23, sigma=0.05).astype(np.float64)
    T = 0.4
    _, vr = oracle.subcycle(pos, vel, L, sp, dt=T, nsub=512)
    errs = []
    for nsub in (8, 16):
        _, v = oracle.subcycle(pos, vel, L, sp, dt=T, nsub=nsub)
        errs.append(np.sqrt(((v - vr) ** 2).mean()))
    assert 3.6 < errs[0] / errs[1] < 4.4


def test_energy_error_bounded_and_second_order(split_params):
    # symplectic map: the energy error stays small and falls as h^2
    sp = dict(split_params, eps=0.1)
    L = 12.0
    pos = synth.uniform(400, L, seed=5).astype(np.float64)
    vel = synth.gaussian_velocities(400, seed=5, sigma=0.05).astype(np.float64)
    m = pos[:, 3]

    def energy(x, v):
        _, ke, pe = oracle.diagnostics(x, v, m, L, sp)
        return ke + pe

    e0 = energy(pos[:, :3], vel[:, :3])
    devs = []
    for nsub in (40, 80):
        x, v = oracle.subcycle(pos, vel, L, sp, dt=0.5, nsub=nsub)
        devs.append(abs(energy(x, v) - e0))
    assert devs[0] < 1e-3 * abs(e0)
    assert 3.6 < devs[0] / devs[1] < 4.4


def test_diagnostics_momentum_and_kinetic(split_params):
    pos, vel, L = _state(n=50, seed=25)
    m = np.random.default_rng(3).uniform(0.5, 2, 50)
    p, ke, pe = oracle.diagnostics(pos[:, :3], vel[:, :3], m, L, split_params)
    assert np.allclose(p, (m[:, None] * vel[:, :3]).sum(0), rtol=1e-14, atol=1e-15)
    assert ke == pytest.approx(0.5 * (m * (vel[:, :3] ** 2).sum(1)).sum(), rel=1e-14)
    # pair potential by a plain double loop in Python
    sp = split_params
    x = pos[:, :3]
    ref = 0.0
    for i in range(50):
        for j in range(i + 1, 50):
            d = _min_image_diff(x[j], x[i], L)
            s = float(d @ d)
            if s < sp["r_cut"] ** 2:
                ref += sp["G"] * m[i] * m[j] * oracle.phi(s, sp["eps"], sp["poly"], sp["r_cut"])
    assert pe == pytest.approx(ref, rel=1e-12, abs=1e-14)
