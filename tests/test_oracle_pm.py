"""Pins for the oracle's long-range spectral PM force (Sec. 2.3).

What fixes it: the printed constants of Eq. (greenf) and Eq. (filter)
(golden file), the orders the paper claims (sixth-order influence function,
fourth-order Super-Lanczos derivative), exact properties of CIC (mass
conservation, grid-point deposits), momentum conservation, and the paper's
own pair-force test (Fig. ppforce: the orientation-averaged PM force between
two particles follows Eq. (fitform), and Newton at large r).
"""
import os

import numpy as np
import pytest

from oracle import pm, split

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_g6_constants_and_cancellation():
    g = _golden("filter_constants.txt")
    assert g["g6_prefactor"] == 45.0 / 128.0
    assert g["g6_c2"] == -5.0 / 64.0 and g["g6_c3"] == 1.0 / 1024.0 and g["g6_c0"] == -2835.0 / 1024.0
    # the constant term cancels the k = 0 value of the three cosine sums exactly
    assert 3 * (g["g6_c1"] + g["g6_c2"] + g["g6_c3"]) + g["g6_c0"] == 0.0
    assert pm.g6_bracket(0.0, 0.0, 0.0, 64) == 0.0


def test_g6_is_sixth_order_inverse_laplacian():
    ng, L = 256, 256.0
    errs = []
    for k in (2, 4, 8):
        K = 2 * np.pi * k / L
        errs.append(abs(float(pm.green_g6(np.array(float(k)), np.array(0.0), np.array(0.0), ng, L)) * K * K + 1))
    assert errs[0] < 1e-9
    for a, b in zip(errs, errs[1:]):
        assert 50 < b / a < 80                       # 2^6 = 64 per doubling


def test_super_lanczos_is_fourth_order():
    ng, L = 128, 128.0
    errs = []
    for k in (2, 4, 8):
        K = 2 * np.pi * k / L
        errs.append(abs(float(pm.sl_derivative(np.array(float(k)), ng, L)) / K - 1))
    for a, b in zip(errs, errs[1:]):
        assert 14 < b / a < 18                       # 2^4 = 16 per doubling
    # and applied to a sampled sine it differentiates it to that accuracy
    x = np.arange(ng) * (L / ng)
    f = np.sin(2 * np.pi * 3 * x / L)
    fk = np.fft.rfft(f)
    kk = np.fft.rfftfreq(ng, d=1.0 / ng)
    df = np.fft.irfft(1j * pm.sl_derivative(kk, ng, L) * fk, n=ng)
    exact = 2 * np.pi * 3 / L * np.cos(2 * np.pi * 3 * x / L)
    assert np.abs(df - exact).max() < 1e-4 * np.abs(exact).max()


def test_filter_values():
    g = _golden("filter_constants.txt")
    D = 1.0
    assert pm.filter_s(np.array(0.0), D, g["sigma"], int(g["n_s"])) == 1.0
    # at the Nyquist wavenumber k D = pi the sinc factor is 2/pi
    v = float(pm.filter_s(np.array(np.pi), D, 0.0, 1))
    assert v == pytest.approx(2 / np.pi, rel=1e-15)
    v = float(pm.filter_s(np.array(1.0), D, 0.8, 3))
    assert v == pytest.approx(np.exp(-0.64 / 4) * (2 * np.sin(0.5)) ** 3, rel=1e-15)


def test_cic_conserves_mass_and_hits_grid_points():
    rng = np.random.default_rng(1)
    ng, L = 16, 16.0
    x = rng.uniform(0, L, (500, 3))
    m = rng.uniform(0.5, 2.0, 500)
    rho = pm.cic_deposit(x, m, ng, L)
    assert rho.sum() * (L / ng) ** 3 == pytest.approx(m.sum(), rel=1e-14)
    one = pm.cic_deposit(np.array([[3.0, 5.0, 7.0]]), np.array([2.0]), ng, L)
    assert one[3, 5, 7] == 2.0 and one.sum() == 2.0
    # CIC interpolation of a constant field is exact
    assert np.allclose(pm.cic_interp(np.full((ng, ng, ng), 1.5), x, ng, L), 1.5, rtol=1e-15)


def test_momentum_conserved():
    rng = np.random.default_rng(2)
    ng, L = 32, 32.0
    x = rng.uniform(0, L, (3000, 3))
    m = rng.uniform(0.5, 2.0, 3000)
    a = pm.pm_accel(x, m, L, ng)
    net = (m[:, None] * a).sum(0)
    assert np.abs(net).max() < 1e-10 * (m[:, None] * np.abs(a)).sum()


@pytest.mark.slow
def test_pair_force_follows_fitform_and_newton():
    # Fig. ppforce procedure: pairs at fixed separation, random orientations,
    # orientation-averaged force vs Eq. (fitform), which tends to 1/r^2
    ng = L = 32
    rng = np.random.default_rng(3)
    for r in (1.0, 1.5, 2.0, 3.0, 4.0, 5.0):
        f = []
        for _ in range(48):
            xa = rng.uniform(0, L, 3)
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            xb = xa + r * u
            acc = pm.pm_accel(xb[None, :], None, L, ng, sources=(xa[None, :], np.array([1.0])))
            f.append(-acc[0] @ u)
        mean = np.mean(f) * r * r
        assert abs(mean - float(split.f_grid(r)) * r * r) < 0.03, (r, mean)
    assert abs(mean - 1.0) < 0.03


def _min_image(d, L):
    return d - L * np.round(d / L)


def test_full_step_is_reversible_and_conserves_momentum(split_params):
    # Eq. (tstep) composes symmetric maps: running it backwards with reversed
    # velocities returns to the start; PM and SR forces both conserve momentum
    import oracle
    import synth
    L = 16.0
    pos = synth.blob_mixture(600, L, seed=41, n_blobs=3, sigma=0.8).astype(np.float64)
    vel = synth.gaussian_velocities(600, seed=41, sigma=0.05).astype(np.float64)
    sp = dict(split_params, eps=0.05)
    x1, v1 = oracle.step(pos, vel, L, sp, dt=0.2, n_c=3)
    p1 = np.concatenate([x1, pos[:, 3:]], axis=1)
    x2, v2 = oracle.step(p1, -v1, L, sp, dt=0.2, n_c=3)
    assert np.abs(_min_image(x2 - pos[:, :3], L)).max() < 1e-9
    assert np.abs(-v2 - vel[:, :3]).max() < 1e-9
    assert np.abs(v1.sum(0) - vel[:, :3].sum(0)).max() < 1e-10
