"""Seeded synthetic inputs for the short-range force path.

This module holds only input generation: random positions, velocities and
request streams.  It contains none of the force method's arithmetic (no pair
force, no binning, no time stepping), so both the oracle and the CUDA path
may take their inputs from it.

All generators use numpy's PCG64 with an explicit seed, so x86-64 and aarch64
produce the same numbers.  Positions are FP32 in grid units, wrapped into
[0, L); masses are 1 (the fourth float of each (x, y, z, m) row).

Workloads (each stands in for a clustered, ~1 particle per grid cell
cosmological volume; no dataset is read):
  blob_mixture  half uniform, half in Gaussian blobs (sigma 0.5 grid units)
  zeldovich     lattice displaced by the Zel'dovich field of a Gaussian
                density with P(k) ~ k^-2, sigma_delta = 1 on the grid
  batch_boxes   many independent blob-mixture boxes of log-uniform size
  request_stream Poisson arrivals of box runs for the serving loop
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _wrap_f32(x64: np.ndarray, L: float) -> np.ndarray:
    """Wrap FP64 coordinates into [0, L) and round to FP32, keeping < L."""
    Lf = np.float32(L)
    x = np.mod(x64, float(Lf)).astype(np.float32)
    x[x >= Lf] = np.float32(0.0)
    x[x < 0] = np.float32(0.0)
    return x


def as_pos4(x: np.ndarray, m: np.ndarray | float = 1.0) -> np.ndarray:
    """Pack n x 3 positions and masses into n x 4 FP32 (x, y, z, m) rows."""
    n = x.shape[0]
    out = np.empty((n, 4), dtype=np.float32)
    out[:, :3] = x
    out[:, 3] = m
    return out


def box_size_f32(L: float) -> float:
    """Box sizes handed to the library must be FP32 values."""
    return float(np.float32(L))


def blob_mixture(n: int, L: float, seed: int, n_blobs: int = 64, sigma: float = 0.5,
                 frac_uniform: float = 0.5) -> np.ndarray:
    """n x 4 FP32: round(n*frac_uniform) uniform in [0,L)^3, the rest in n_blobs
    isotropic Gaussian blobs of width sigma around uniform random centres."""
    L = box_size_f32(L)
    g = _rng(seed)
    nu = int(round(n * frac_uniform))
    nb = n - nu
    xu = g.uniform(0.0, L, size=(nu, 3))
    centres = g.uniform(0.0, L, size=(n_blobs, 3))
    which = np.arange(nb) % n_blobs
    xb = centres[which] + g.normal(0.0, sigma, size=(nb, 3))
    x = np.concatenate([xu, xb], axis=0)
    return as_pos4(_wrap_f32(x, L))


def blob_mixture_scaled(n: int, L: float, seed: int, per_blob: int = 256, sigma: float = 0.5) -> np.ndarray:
    """The 32^3 blob mixture's statistics at any n: half uniform, half in
    Gaussian blobs of `per_blob` particles (n_blobs = n / (2 per_blob), at
    least 1), so that blob density does not grow with the box."""
    return blob_mixture(n, L, seed, n_blobs=max(1, int(round(n / (2.0 * per_blob)))), sigma=sigma)


def gaussian_velocities(n: int, seed: int, sigma: float = 0.1) -> np.ndarray:
    """n x 4 FP32 velocities, each component N(0, sigma^2), w = 0."""
    g = _rng(seed + 0x5eed)
    v = np.zeros((n, 4), dtype=np.float32)
    v[:, :3] = g.normal(0.0, sigma, size=(n, 3)).astype(np.float32)
    return v


def zeldovich(ng: int, seed: int, L: float | None = None, sigma_delta: float = 1.0,
              index: float = -2.0, return_stats: bool = False, return_f64: bool = False):
    """ng^3 particles displaced from the lattice q = (i + 1/2) dx by the
    Zel'dovich field psi of a Gaussian random density delta with power
    spectrum P(k) ~ k^index (k = 0 mode zero), normalised so that delta has
    standard deviation sigma_delta on the ng^3 grid:
        psi(k) = i k delta(k) / k^2,   x = q + psi(q)   (so div psi = -delta).
    Returns n x 4 FP32 positions (and optionally a stats dict); with
    return_f64, the FP64 positions (n x 3, wrapped into [0, L)) instead."""
    try:
        import scipy.fft as fft
        kw = dict(workers=-1)
    except Exception:  # pragma: no cover
        import numpy.fft as fft
        kw = {}
    L = float(ng) if L is None else box_size_f32(L)
    dx = L / ng
    g = _rng(seed)
    white = g.standard_normal(size=(ng, ng, ng), dtype=np.float64)
    wk = fft.rfftn(white, **kw)
    del white
    kx = 2.0 * np.pi * np.fft.fftfreq(ng, d=dx)
    kz = 2.0 * np.pi * np.fft.rfftfreq(ng, d=dx)
    k2 = (kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2)
    k2[0, 0, 0] = 1.0
    amp = k2 ** (index / 4.0)          # sqrt(P(k)) = k^(index/2)
    amp[0, 0, 0] = 0.0
    dk = wk * amp
    del wk, amp
    delta = fft.irfftn(dk, s=(ng, ng, ng), **kw)
    scale = sigma_delta / float(delta.std())
    del delta
    dk *= scale
    dk /= k2
    q1 = (np.arange(ng, dtype=np.float64) + 0.5) * dx
    x = np.empty((ng, ng, ng, 3), dtype=np.float64)
    # axis 0 of the grid is x, axis 1 is y, axis 2 is z (particle (i, j, k) at
    # q = ((i+.5), (j+.5), (k+.5)) dx); psi_a = irfft(i k_a delta / k^2)
    kvec = (kx[:, None, None], kx[None, :, None], kz[None, None, :])
    rms = 0.0
    for a in range(3):
        psi = fft.irfftn(1j * kvec[a] * dk, s=(ng, ng, ng), **kw)
        rms += float((psi ** 2).mean())
        shape = [1, 1, 1]
        shape[a] = ng
        x[..., a] = q1.reshape(shape) + psi
        del psi
    if return_f64:
        x = np.mod(x.reshape(-1, 3), L)
        x[x >= L] = 0.0
        return x
    pos = as_pos4(_wrap_f32(x.reshape(-1, 3), L))
    if return_stats:
        return pos, dict(rms_displacement=math.sqrt(rms), sigma_delta=sigma_delta, L=L)
    return pos


@dataclass
class BoxSpec:
    n: int
    L: float
    seed: int


def batch_boxes(n_boxes: int = 200, n_min: int = 16 ** 3, n_max: int = 128 ** 3,
                seed: int = 4) -> list[BoxSpec]:
    """Particle counts log-uniform in [n_min, n_max], box side N^(1/3) (FP32),
    one seed per box; positions come from blob_mixture(spec.n, spec.L, spec.seed)."""
    g = _rng(seed)
    ln = g.uniform(math.log(n_min), math.log(n_max), size=n_boxes)
    out = []
    for b in range(n_boxes):
        n = int(round(math.exp(ln[b])))
        out.append(BoxSpec(n=n, L=box_size_f32(n ** (1.0 / 3.0)), seed=seed * 100003 + b))
    return out


@dataclass
class Request:
    rid: int
    t_arrival: float
    n: int
    L: float
    steps: int
    seed: int


def request_stream(rate: float = 50.0, duration: float = 60.0,
                   sides=(32, 64, 128, 256), steps_lo: int = 5, steps_hi: int = 50,
                   seed: int = 5) -> list[Request]:
    """Poisson arrivals (exponential gaps of mean 1/rate) over [0, duration);
    N = side^3 with side uniform in `sides`, box L = side, steps uniform in
    [steps_lo, steps_hi], one blob-mixture seed per request."""
    g = _rng(seed)
    t, rid, out = 0.0, 0, []
    while True:
        t += float(g.exponential(1.0 / rate))
        if t >= duration:
            break
        side = int(sides[int(g.integers(0, len(sides)))])
        steps = int(g.integers(steps_lo, steps_hi + 1))
        out.append(Request(rid=rid, t_arrival=t, n=side ** 3, L=float(side), steps=steps,
                           seed=seed * 1000003 + rid))
        rid += 1
    return out


def lattice(side: int, L: float | None = None) -> np.ndarray:
    """Perfect cubic lattice, one particle per cell of side L/side at cell centres."""
    L = float(side) if L is None else box_size_f32(L)
    q = (np.arange(side, dtype=np.float64) + 0.5) * (L / side)
    x = np.stack(np.meshgrid(q, q, q, indexing="ij"), axis=-1).reshape(-1, 3)
    return as_pos4(_wrap_f32(x, L))


def uniform(n: int, L: float, seed: int) -> np.ndarray:
    L = box_size_f32(L)
    g = _rng(seed)
    return as_pos4(_wrap_f32(g.uniform(0.0, L, size=(n, 3)), L))
