"""Pins for the oracle's force-split constants and the pair kernel f_SR.

The paper fixes Eq. (fitform) (printed constants), Eq. (force) (the kernel's
form) and the matching scale of about three grid cells (Sec. 2.3); these tests
pin the oracle to those and to closed forms derived independently here
(Taylor limits, derivatives, the Plummer law).
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import split

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_fitform_constants_match_paper():
    g = _golden("fitform_constants.txt")
    assert set(g) == set(split.FITFORM)
    for k, v in g.items():
        assert split.FITFORM[k] == v


def test_fgrid_large_r_is_newtonian():
    # tanh -> 1, every other term decays: r^2 F_grid -> 1
    for r in (16.0, 20.0, 40.0):
        assert abs(r * r * float(split.f_grid(r)) - 1.0) < 1e-6


def test_fgrid_small_r_taylor():
    # Taylor expansion by hand: tanh(br)/r^2 - b/(r cosh^2 br) = (2/3) b^3 r + O(r^3),
    # c r (1 + d r^2) e^{-d r^2} = c r + O(r^3), e(1+...)e^{-h r^2} = e + O(r^2)
    p = split.FITFORM
    for r in (1e-3, 3e-3):
        lin = p["e"] + (2.0 / 3.0 * p["b"] ** 3 + p["c"]) * r
        quad = p["e"] * (p["f"] - p["h"]) * r * r
        assert abs(float(split.f_grid(r)) - (lin + quad)) < 5e-7 * max(1.0, r * 1e3)


def test_rcut_is_three_grid_cells_match():
    rc = split.r_cut_default()
    assert abs(rc * rc * float(split.f_grid(rc)) - 1.0) < 1e-13
    assert 3.0 < rc < 3.2                          # "three grid cells", Sec. 2.3
    # below the match the grid force is weaker than Newton, above it is not
    assert 2.9 ** 2 * float(split.f_grid(2.9)) < 1.0 < 3.3 ** 2 * float(split.f_grid(3.3))


def test_poly5_fit_quality_and_constraint():
    rc = split.r_cut_default()
    c = split.fit_poly5(rc)
    r = np.linspace(0.05, rc, 20001)
    rel = np.abs(split.p5(r * r, c) - split.f_grid(r) / r) * r**3    # relative to 1/r^2
    assert rel.max() < 1e-3                       # fit errs well below 0.1% of Newton
    assert abs(float(split.p5(rc * rc, c)) - float(split.f_grid(rc)) / rc) < 1e-13
    cu = split.fit_poly5(rc, constrained=False)
    relu = np.abs(split.p5(r * r, cu) - split.f_grid(r) / r) * r**3
    assert relu.max() < 1e-3
    # the constraint costs accuracy nowhere near the cutoff's own step
    assert rel.max() < 2 * relu.max()


def test_fsr_is_plummer_minus_grid(split_params):
    # r f_SR(r^2) = softened Newton - grid force, within the fit residual
    sp = split_params
    for r in np.linspace(0.05, sp["r_cut"], 57):
        f = oracle.fsr(r * r, sp["eps"], sp["poly"]) * r
        plummer = r / (r * r + sp["eps"]) ** 1.5
        assert abs(f - (plummer - float(split.f_grid(r)))) < 1e-3 / (r * r)


def test_fsr_vanishes_at_cutoff_without_softening(split_params):
    sp = split_params
    s = sp["r_cut"] ** 2
    assert abs(oracle.fsr(s, 0.0, sp["poly"])) < 1e-12


def test_fsr_softening_slope(split_params):
    # d f_SR / d eps at eps = 0 is -3/2 s^(-5/2)
    sp = split_params
    for s in (0.25, 1.0, 4.0):
        e = 1e-7
        slope = (oracle.fsr(s, e, sp["poly"]) - oracle.fsr(s, 0.0, sp["poly"])) / e
        assert slope == pytest.approx(-1.5 * s ** -2.5, rel=1e-5)


def test_potential_derivative_gives_force(split_params):
    # phi'(s) = f_SR(s) / 2 by construction; check by central differences and phi(r_cut^2) = 0
    sp = split_params
    for s in (0.01, 0.3, 1.7, 5.0, 9.0):
        h = 1e-6 * max(s, 1e-2)
        dphi = (oracle.phi(s + h, sp["eps"], sp["poly"], sp["r_cut"])
                - oracle.phi(s - h, sp["eps"], sp["poly"], sp["r_cut"])) / (2 * h)
        assert dphi == pytest.approx(0.5 * oracle.fsr(s, sp["eps"], sp["poly"]), rel=1e-6)
    assert abs(oracle.phi(sp["r_cut"] ** 2, sp["eps"], sp["poly"], sp["r_cut"])) < 1e-15


def test_fsr_positive_inside_cutoff(split_params):
    # the short-range correction is attractive everywhere inside the match at eps=0
    sp = split_params
    s = np.linspace(1e-4, sp["r_cut"] ** 2 * (1 - 1e-6), 2001)
    assert all(oracle.fsr(x, 0.0, sp["poly"]) > 0 for x in s)
