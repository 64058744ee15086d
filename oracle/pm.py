"""FP64 oracle of the long-range spectral particle-mesh force (Sec. 2.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Steps, in the paper's order:
  1. CIC deposit of the particle masses on an ng^3 periodic grid (spacing
     D = L/ng, grid points at integer multiples of D), density = mass / D^3.
  2. FFT of the density.
  3. Multiply by the Gauss-sinc filter of Eq. (filter),
        S(k) = exp(-|k|^2 sigma^2 / 4) [ (2/(|k| D)) sin(|k| D / 2) ]^ns,
     with |k| the physical wavenumber and sigma in grid units (times D),
     and by 4 pi G times the sixth-order influence function of Eq. (greenf),
        G6(k) = (45/128) D^2 [ sum_i cos(2 pi k_i D / L) - (5/64) sum_i cos(4 pi k_i D / L)
                              + (1/1024) sum_i cos(8 pi k_i D / L) - 2835/1024 ]^(-1),
     k_i the integer mode numbers (G6 -> -1/K^2, the inverse Laplacian, at low K).
  4. For each direction, the fourth-order Super-Lanczos derivative of
     Eq. (sldiff), read as multiplication by i [ (4/3) sin(K_i D) - (1/6) sin(2 K_i D) ] / D,
     K_i = 2 pi k_i / L, and the acceleration a = -grad(phi); one inverse FFT per
     component.
  5. CIC interpolation of the three components back to the particles.
The k = 0 mode is dropped (the mean density exerts no force in a periodic box).
"""
from __future__ import annotations

import numpy as np


def _cic_weights(x, ng, L):
    u = np.asarray(x, dtype=np.float64) * (ng / L)
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    return i0 % ng, (i0 + 1) % ng, f


def cic_deposit(x, m, ng, L):
    """Mass density on the grid (mass / D^3)."""
    x = np.asarray(x, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    rho = np.zeros((ng, ng, ng), dtype=np.float64)
    a0, a1, fa = _cic_weights(x[:, 0], ng, L)
    b0, b1, fb = _cic_weights(x[:, 1], ng, L)
    c0, c1, fc = _cic_weights(x[:, 2], ng, L)
    for ia, wa in ((a0, 1 - fa), (a1, fa)):
        for ib, wb in ((b0, 1 - fb), (b1, fb)):
            for ic, wc in ((c0, 1 - fc), (c1, fc)):
                np.add.at(rho, (ia, ib, ic), m * wa * wb * wc)
    D = L / ng
    return rho / D ** 3


def cic_interp(field, x, ng, L):
    x = np.asarray(x, dtype=np.float64)
    a0, a1, fa = _cic_weights(x[:, 0], ng, L)
    b0, b1, fb = _cic_weights(x[:, 1], ng, L)
    c0, c1, fc = _cic_weights(x[:, 2], ng, L)
    out = np.zeros(len(x), dtype=np.float64)
    for ia, wa in ((a0, 1 - fa), (a1, fa)):
        for ib, wb in ((b0, 1 - fb), (b1, fb)):
            for ic, wc in ((c0, 1 - fc), (c1, fc)):
                out += field[ia, ib, ic] * wa * wb * wc
    return out


def mode_numbers(ng):
    """Integer mode numbers along a full axis and along the halved (rfft) axis."""
    return np.fft.fftfreq(ng, d=1.0 / ng), np.fft.rfftfreq(ng, d=1.0 / ng)


def g6_bracket(kx, ky, kz, ng):
    """The bracket of Eq. (greenf) for integer mode numbers (D/L = 1/ng)."""
    s = 0.0
    for k in (kx, ky, kz):
        ph = 2.0 * np.pi * k / ng
        s = s + np.cos(ph) - (5.0 / 64.0) * np.cos(2 * ph) + (1.0 / 1024.0) * np.cos(4 * ph)
    return s - 2835.0 / 1024.0


def green_g6(kx, ky, kz, ng, L):
    D = L / ng
    b = g6_bracket(kx, ky, kz, ng)
    with np.errstate(divide="ignore"):
        g = (45.0 / 128.0) * D * D / b
    return np.where(b == 0.0, 0.0, g)


def filter_s(kmag, D, sigma, ns):
    """Eq. (filter) at physical wavenumber |k|."""
    x = kmag * D
    with np.errstate(invalid="ignore", divide="ignore"):
        sinc = np.where(x == 0.0, 1.0, (2.0 / x) * np.sin(x / 2.0))
    return np.exp(-(kmag ** 2) * (sigma * D) ** 2 / 4.0) * sinc ** ns


def sl_derivative(k, ng, L):
    """Eq. (sldiff) multiplier (without the factor i) along one axis."""
    D = L / ng
    K = 2.0 * np.pi * k / L
    return ((4.0 / 3.0) * np.sin(K * D) - (1.0 / 6.0) * np.sin(2.0 * K * D)) / D


def pm_accel(x, m, L, ng, sigma=0.8, ns=3, G=1.0, sources=None):
    """Long-range acceleration (n x 3, FP64) at positions x.  `sources`
    (x_s, m_s) deposits other particles than the ones interpolated at."""
    xs, ms = (x, m) if sources is None else sources
    rho = cic_deposit(xs, ms, ng, L)
    rk = np.fft.rfftn(rho)
    kf, kh = mode_numbers(ng)
    kx, ky, kz = kf[:, None, None], kf[None, :, None], kh[None, None, :]
    D = L / ng
    kmag = 2.0 * np.pi / L * np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    phik = 4.0 * np.pi * G * green_g6(kx, ky, kz, ng, L) * filter_s(kmag, D, sigma, ns) * rk
    phik[0, 0, 0] = 0.0
    acc = np.empty((len(x), 3), dtype=np.float64)
    for a, k in enumerate((kx, ky, kz)):
        ak = -1j * sl_derivative(k, ng, L) * phik
        field = np.fft.irfftn(ak, s=(ng, ng, ng), axes=(0, 1, 2))
        acc[:, a] = cic_interp(field, x, ng, L)
    return acc
