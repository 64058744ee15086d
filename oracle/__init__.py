"""FP64 CPU oracle for the HACC short-range force path (arXiv 1410.2805).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline / reference legs of bench.py import this package.  The product
library (paper_1410_2805_gb300) never imports it, and it never imports the
product library: the two share no code.

The arithmetic lives in hacc_oracle.c (plain C, FP64, OpenMP over particles
only) and split.py (Eq. (fitform) and the P5 fit).  This module compiles the
C file on first use with gcc and wraps it with ctypes over numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import split  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hacc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hacc_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, i32, d, p = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            L.hacc_oracle_fsr.restype = d
            L.hacc_oracle_fsr.argtypes = [d, d, p]
            L.hacc_oracle_phi.restype = d
            L.hacc_oracle_phi.argtypes = [d, d, p, d]
            L.hacc_oracle_wrap_cell.restype = i32
            L.hacc_oracle_wrap_cell.argtypes = [i64, p, d, i32, p]
            L.hacc_oracle_bin.restype = None
            L.hacc_oracle_bin.argtypes = [i64, p, i64, p, p, p]
            L.hacc_oracle_candidates.restype = ctypes.c_uint64
            L.hacc_oracle_candidates.argtypes = [p, i32]
            L.hacc_oracle_force_brute.restype = None
            L.hacc_oracle_force_brute.argtypes = [i64, p, p, d, d, d, p, d, p, p]
            L.hacc_oracle_force_mesh.restype = None
            L.hacc_oracle_force_mesh.argtypes = [i64, p, p, d, d, d, p, d, i64, p, p, p]
            L.hacc_oracle_subcycle.restype = None
            L.hacc_oracle_subcycle.argtypes = [i64, p, p, p, d, d, d, p, d, d, i32]
            L.hacc_oracle_diagnostics.restype = None
            L.hacc_oracle_diagnostics.argtypes = [i64, p, p, p, d, d, d, p, d, p]
            L.hacc_oracle_ml_levels.restype = None
            L.hacc_oracle_ml_levels.argtypes = [i64, p, d, i32, i32, i32, i32, p]
            L.hacc_oracle_subcycle_ml.restype = None
            L.hacc_oracle_subcycle_ml.argtypes = [i64, p, p, p, d, d, d, p, d, d, i32, p]
            L.hacc_oracle_threads.restype = i32
            L.hacc_oracle_set_threads.argtypes = [i32]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(poly) -> np.ndarray:
    c = np.ascontiguousarray(poly, dtype=np.float64)
    assert c.shape == (6,)
    return c


def threads() -> int:
    return lib().hacc_oracle_threads()


def set_threads(n: int) -> None:
    lib().hacc_oracle_set_threads(int(n))


def fsr(s: float, eps: float, poly) -> float:
    """Eq. (force) at one s, FP64."""
    c = _c(poly)
    return lib().hacc_oracle_fsr(float(s), float(eps), _ptr(c))


def phi(s: float, eps: float, poly, r_cut: float) -> float:
    c = _c(poly)
    return lib().hacc_oracle_phi(float(s), float(eps), _ptr(c), float(r_cut))


def wrap_cell(pos4: np.ndarray, L: float, nc: int):
    """Wrap FP32 (x, y, z, m) rows into [0, L) and return (wrapped copy, cell ids, ok)."""
    p = np.ascontiguousarray(pos4, dtype=np.float32).copy()
    n = p.shape[0]
    cell = np.empty(n, dtype=np.int32)
    rc = lib().hacc_oracle_wrap_cell(n, _ptr(p), float(L), int(nc), _ptr(cell))
    return p, cell, rc == 0


def bin_cells(cell: np.ndarray, nc: int):
    """Stable counting sort by cell: (count, start, perm)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    ncell = nc ** 3
    count = np.empty(ncell, dtype=np.int32)
    start = np.empty(ncell + 1, dtype=np.int32)
    perm = np.empty(cell.shape[0], dtype=np.int32)
    lib().hacc_oracle_bin(cell.shape[0], _ptr(cell), ncell, _ptr(count), _ptr(start), _ptr(perm))
    return count, start, perm


def candidates(count: np.ndarray, nc: int) -> int:
    count = np.ascontiguousarray(count, dtype=np.int32)
    return int(lib().hacc_oracle_candidates(_ptr(count), int(nc)))


def _xm(pos):
    pos = np.asarray(pos)
    x = np.ascontiguousarray(pos[:, :3], dtype=np.float64)
    m = np.ascontiguousarray(pos[:, 3], dtype=np.float64) if pos.shape[1] > 3 else np.ones(pos.shape[0])
    return x, m


def force_brute(pos, L, split_params):
    """All-pairs FP64 forces; pos is n x 4 (x, y, z, m). Returns (acc n x 3, within)."""
    x, m = _xm(pos)
    c = _c(split_params["poly"])
    acc = np.empty_like(x)
    w = ctypes.c_uint64(0)
    lib().hacc_oracle_force_brute(x.shape[0], _ptr(x), _ptr(m), float(L), float(split_params["r_cut"]),
                                  float(split_params["eps"]), _ptr(c), float(split_params["G"]),
                                  _ptr(acc), ctypes.byref(w))
    return acc, int(w.value)


def force_mesh(pos, L, split_params, sel=None):
    """FP64 forces through the oracle's own cell list, for all or selected particles."""
    x, m = _xm(pos)
    c = _c(split_params["poly"])
    if sel is None:
        nsel, selp = x.shape[0], None
    else:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        nsel, selp = sel.shape[0], _ptr(sel)
    acc = np.empty((nsel, 3), dtype=np.float64)
    w = ctypes.c_uint64(0)
    lib().hacc_oracle_force_mesh(x.shape[0], _ptr(x), _ptr(m), float(L), float(split_params["r_cut"]),
                                 float(split_params["eps"]), _ptr(c), float(split_params["G"]),
                                 nsel, selp, _ptr(acc), ctypes.byref(w))
    return acc, int(w.value)


def subcycle(pos, vel, L, split_params, dt, nsub):
    """FP64 SKS sub-cycles; returns new (x n x 3, v n x 3) as float64."""
    x, m = _xm(pos)
    x = x.copy()
    v = np.ascontiguousarray(np.asarray(vel)[:, :3], dtype=np.float64).copy()
    c = _c(split_params["poly"])
    lib().hacc_oracle_subcycle(x.shape[0], _ptr(x), _ptr(v), _ptr(m), float(L),
                               float(split_params["r_cut"]), float(split_params["eps"]), _ptr(c),
                               float(split_params["G"]), float(dt), int(nsub))
    return x, v


def diagnostics(x, v, m, L, split_params):
    """(momentum[3], kinetic, potential) in FP64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    c = _c(split_params["poly"])
    out = np.empty(5, dtype=np.float64)
    lib().hacc_oracle_diagnostics(x.shape[0], _ptr(x), _ptr(v), _ptr(m), float(L),
                                  float(split_params["r_cut"]), float(split_params["eps"]), _ptr(c),
                                  float(split_params["G"]), _ptr(out))
    return out[:3].copy(), float(out[3]), float(out[4])


def step(pos, vel, L, split_params, dt, n_c, ng=None, sigma=0.8, ns=3):
    """One full step of Eq. (tstep), FP64: long-range kick dt/2 (spectral PM,
    oracle/pm.py), n_c short-range SKS sub-cycles of dt/n_c, long-range kick
    dt/2.  Returns new (x n x 3, v n x 3)."""
    from . import pm
    x, m = _xm(pos)
    v = np.ascontiguousarray(np.asarray(vel)[:, :3], dtype=np.float64).copy()
    ng = int(round(L)) if ng is None else int(ng)
    G = float(split_params["G"])
    v += 0.5 * dt * G * pm.pm_accel(x, m, L, ng, sigma=sigma, ns=ns)
    p1 = np.concatenate([x, m[:, None]], axis=1)
    x, v = subcycle(p1, v, L, split_params, dt, n_c)
    v += 0.5 * dt * G * pm.pm_accel(x, m, L, ng, sigma=sigma, ns=ns)
    return x, v


def ml_levels(pos32, L, nc, d, lmax, lmin=1):
    """Kick counts of Eq. (kicks) from the chaining-mesh densities of the FP32 start positions,
    clamped to [lmin, lmax]."""
    p = np.ascontiguousarray(pos32, dtype=np.float32)
    lev = np.empty(p.shape[0], dtype=np.int32)
    lib().hacc_oracle_ml_levels(p.shape[0], _ptr(p), float(L), int(nc), int(d), int(lmin), int(lmax), _ptr(lev))
    return lev


def subcycle_ml(pos, vel, L, split_params, dt, lmax, level):
    """One FP64 multi-level step with fixed kick counts; returns (x, v)."""
    x, m = _xm(pos)
    x = x.copy()
    v = np.ascontiguousarray(np.asarray(vel)[:, :3], dtype=np.float64).copy()
    c = _c(split_params["poly"])
    lev = np.ascontiguousarray(level, dtype=np.int32)
    lib().hacc_oracle_subcycle_ml(x.shape[0], _ptr(x), _ptr(v), _ptr(m), float(L), float(split_params["r_cut"]),
                                  float(split_params["eps"]), _ptr(c), float(split_params["G"]), float(dt),
                                  int(lmax), _ptr(lev))
    return x, v
