"""Python binding of the hacc GB300 library (short-range P3M force of HACC,
arXiv 1410.2805).

Argument marshalling only: every step of the path runs in the CUDA kernels of
libhacc.so (csrc/), reached through the C ABI declared in include/hacc.h.
PyTorch supplies device memory and streams.  There is no CPU fallback: if
the library has not been built, importing the binding's entry points raises.

    import torch, paper_1410_2805_gb300 as hacc
    ctx = hacc.Context()
    split = hacc.default_split()
    box = hacc.Box(L=32.0)
    acc = ctx.sr_force(box, split, pos)            # pos: (n, 4) float32 CUDA tensor
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhacc.so")

HACC_OK, HACC_EINVAL, HACC_EDOMAIN, HACC_ENOMEM, HACC_ECUDA, HACC_ETIMEOUT = range(6)
_STATUS_NAMES = {0: "HACC_OK", 1: "HACC_EINVAL", 2: "HACC_EDOMAIN", 3: "HACC_ENOMEM", 4: "HACC_ECUDA",
                 5: "HACC_ETIMEOUT"}


class HaccError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, status), message))
        self.status = status


class _Box(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("nc", ctypes.c_int32), ("ng", ctypes.c_int32)]


class _Split(ctypes.Structure):
    _fields_ = [("r_cut", ctypes.c_float), ("eps", ctypes.c_float), ("poly", ctypes.c_double * 6),
                ("G", ctypes.c_float)]


class _Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("force_launches", ctypes.c_int64),
                ("force_ms", ctypes.c_double), ("candidate_pairs", ctypes.c_uint64),
                ("within_pairs", ctypes.c_uint64), ("evaluated_pairs", ctypes.c_uint64),
                ("ml_rebins", ctypes.c_int64), ("build_ms", ctypes.c_double), ("builds", ctypes.c_int64)]


class _BatchBox(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("nc", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("offset", ctypes.c_int64), ("n", ctypes.c_int64), ("dt", ctypes.c_double)]


TICK_FIRST, TICK_LAST = 1, 2
FORCE_VARIANTS = 4   # HACC_FORCE_VARIANTS
BATCH_TUNE_SETTINGS = 48   # HACC_BATCH_TUNE_SETTINGS
TUNE_SETTINGS = 40   # HACC_TUNE_SETTINGS
# tuner settings: k = (cap index * 2 + queue order) * FORCE_VARIANTS + variant
TUNE_CAPS = (0, 16, 24, 32, 48)   # item caps of the single-box tuner
BATCH_TUNE_CAPS = (0, 32, 64, 96, 128, 160)   # item caps of the batched tuner


def tune_setting(k: int, caps) -> dict:
    """(item cap, heavy_first, variant) of tuner setting k."""
    return dict(item_cap=caps[k // (2 * FORCE_VARIANTS)], heavy_first=bool((k // FORCE_VARIANTS) % 2),
                variant=k % FORCE_VARIANTS)


@dataclass
class BatchBox:
    """One box of a batch: side L, rows [offset, offset + n) of the pool
    arrays, step dt (the full step for batch_subcycle, the sub-cycle step
    for batch_tick), tick flags TICK_FIRST / TICK_LAST."""
    L: float
    offset: int
    n: int
    dt: float
    nc: int = 0
    flags: int = 0


def _boxes_c(boxes):
    arr = (_BatchBox * max(1, len(boxes)))()
    for i, b in enumerate(boxes):
        arr[i] = _BatchBox(float(b.L), int(b.nc), int(b.flags), int(b.offset), int(b.n), float(b.dt))
    return arr


class _TickInfo(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int32), ("finished", ctypes.c_int32), ("active", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("particles", ctypes.c_int64), ("free_rows", ctypes.c_int64)]


class _Pm(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_float), ("ns", ctypes.c_int32)]


@dataclass
class Box:
    """Periodic cube: side L (an FP32 value, grid units), nc chaining-mesh
    cells per side (0 = default), ng PM grid points per side (0 = round(L))."""
    L: float
    nc: int = 0
    ng: int = 0

    def _c(self):
        return _Box(float(self.L), int(self.nc), int(self.ng))


@dataclass
class Split:
    """Force split: cutoff r_cut, softening eps (length^2), P5 coefficients in
    ascending powers of s, prefactor G."""
    r_cut: float
    eps: float
    poly: tuple = field(default_factory=lambda: (0.0,) * 6)
    G: float = 1.0

    def _c(self):
        return _Split(float(self.r_cut), float(self.eps), (ctypes.c_double * 6)(*[float(x) for x in self.poly]),
                      float(self.G))

    def as_dict(self):
        return dict(r_cut=float(self.r_cut), eps=float(self.eps), poly=list(self.poly), G=float(self.G))


@dataclass
class PM:
    """Gauss-sinc filter width sigma and sinc power ns (Eq. (filter))."""
    sigma: float = 0.8
    ns: int = 3

    def _c(self):
        return _Pm(float(self.sigma), int(self.ns))


_lib = None


def lib():
    """Load libhacc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhacc.so is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                               "or `python -m paper_1410_2805_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        p, i32, i64, d, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        sig = {
            "hacc_ctx_create": (st, [ctypes.POINTER(p), ctypes.c_int, ctypes.c_size_t]),
            "hacc_ctx_destroy": (None, [p]),
            "hacc_last_error": (ctypes.c_char_p, [p]),
            "hacc_ctx_sync": (st, [p, p]),
            "hacc_ctx_scratch_bytes": (ctypes.c_size_t, [p]),
            "hacc_split_default": (st, [ctypes.POINTER(_Split)]),
            "hacc_mesh_cells": (i32, [d, ctypes.c_float]),
            "hacc_bin": (st, [p, ctypes.POINTER(_Box), ctypes.c_float, i64, p, p, p, p, p]),
            "hacc_sr_force": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, p, p, p]),
            "hacc_subcycle": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, p, d, i32, p]),
            "hacc_step": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), ctypes.POINTER(_Pm), i64, p, p, d,
                               i32, p]),
            "hacc_pm_force": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Pm), i64, p, p, p]),
            "hacc_diagnostics": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, p, p, p]),
            "hacc_sr_force_host": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, p, p]),
            "hacc_subcycle_host": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, p, d, i32, p]),
            "hacc_step_host": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), ctypes.POINTER(_Pm), i64, p,
                                    p, d, i32, p]),
            "hacc_stats_enable": (st, [p, ctypes.c_int, ctypes.c_int]),
            "hacc_subcycle_ml": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, p, d, i32, i32,
                                      i32, ctypes.c_float, p, p]),
            "hacc_ml_mesh_cells": (i32, [d, ctypes.c_float, ctypes.c_float]),
            "hacc_ci_from_f64": (st, [p, ctypes.POINTER(_Box), ctypes.c_float, i64, p, p, p, p, p]),
            "hacc_ci_to_f64": (st, [p, ctypes.POINTER(_Box), ctypes.c_float, i64, p, p, p, p]),
            "hacc_sr_force_ci": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, p, p, p]),
            "hacc_subcycle_ci": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, p, p, d, i32, p]),
            "hacc_tune": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, i32,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32), p]),
            "hacc_set_variant": (st, [p, i32]),
            "hacc_set_queue_order": (st, [p, i32]),
            "hacc_set_item_cap": (st, [p, i32, i32]),
            "hacc_set_stencil": (st, [p, i32]),
            "hacc_batch_subcycle": (st, [p, ctypes.POINTER(_Split), i32, ctypes.POINTER(_BatchBox), p, p, i32, i32,
                                         p]),
            "hacc_batch_tick": (st, [p, ctypes.POINTER(_Split), i32, ctypes.POINTER(_BatchBox), p, p, p]),
            "hacc_server_create": (st, [ctypes.POINTER(p), p, ctypes.POINTER(_Split), ctypes.c_size_t, i64]),
            "hacc_server_destroy": (None, [p]),
            "hacc_server_submit": (st, [p, i64, d, i64, p, p, d, i32]),
            "hacc_server_tick": (st, [p, p, ctypes.POINTER(_TickInfo), ctypes.POINTER(i64), i32]),
            "hacc_stats_read": (st, [p, ctypes.POINTER(_Stats), ctypes.c_int]),
            "hacc_batch_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(_Split), i32, ctypes.POINTER(_BatchBox)]),
            "hacc_batch_tune": (st, [p, ctypes.POINTER(_Split), i32, ctypes.POINTER(_BatchBox), p, p, i32,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32), p]),
            "hacc_batch_diagnostics": (st, [p, ctypes.POINTER(_Split), i32, ctypes.POINTER(_BatchBox), p, p, p, p]),
            "hacc_diagnostics_ci": (st, [p, ctypes.POINTER(_Box), ctypes.POINTER(_Split), i64, p, p, p, p, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def default_split() -> Split:
    """The library's default split (host FP64 fit of Eq. (fitform))."""
    s = _Split()
    st = lib().hacc_split_default(ctypes.byref(s))
    if st != HACC_OK:
        raise HaccError(st, "hacc_split_default")
    return Split(r_cut=s.r_cut, eps=s.eps, poly=tuple(s.poly), G=s.G)


def mesh_cells(L: float, r_cut: float) -> int:
    return int(lib().hacc_mesh_cells(float(L), float(r_cut)))


def ml_mesh_cells(L: float, r_cut: float, skin: float = 0.05) -> int:
    """Cells per side of the multi-level step's chaining mesh (box nc = 0)."""
    return int(lib().hacc_ml_mesh_cells(float(L), float(r_cut), float(skin)))


def batch_scratch_bytes(split, boxes) -> int:
    """Context scratch of one batched tick over `boxes` (host arithmetic only)."""
    sp = _split_of(split)
    return int(lib().hacc_batch_scratch_bytes(ctypes.byref(sp._c()), len(boxes), _boxes_c(boxes)))


def _split_of(split) -> Split:
    if isinstance(split, Split):
        return split
    return Split(r_cut=split["r_cut"], eps=split["eps"], poly=tuple(split["poly"]), G=split.get("G", 1.0))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _dev_rows(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 2
            and t.shape[1] == 4 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous (n, 4) float32 CUDA tensor" % name)
    return t


class Context:
    """One hacc_ctx on a CUDA device; owns the scratch pool of the calls."""

    def __init__(self, device: int | None = None, hbm_budget_bytes: int = 0):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        self._h = ctypes.c_void_p()
        st = lib().hacc_ctx_create(ctypes.byref(self._h), self.device, int(hbm_budget_bytes))
        if st != HACC_OK:
            raise HaccError(st, "hacc_ctx_create(device=%d)" % self.device)

    def close(self):
        if self._h:
            lib().hacc_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def _check(self, st, what):
        if st != HACC_OK:
            msg = lib().hacc_last_error(self._h)
            raise HaccError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def sync(self, stream=None):
        self._check(lib().hacc_ctx_sync(self._h, self._stream(stream)), "hacc_ctx_sync")

    def tune(self, box: Box, split, pos, reps: int = 3, stream=None) -> dict:
        """Time every (item cap, kernel variant) setting on this machine (chaining-mesh build + pair
        force) and keep the fastest for this context."""
        _dev_rows(pos, "pos")
        sp = _split_of(split)
        times = (ctypes.c_double * TUNE_SETTINGS)()
        chosen = ctypes.c_int32(-1)
        self._check(lib().hacc_tune(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), pos.shape[0], _ptr(pos),
                                    int(reps), times, ctypes.byref(chosen), self._stream(stream)), "hacc_tune")
        k = int(chosen.value)
        return dict(chosen=k, **tune_setting(k, TUNE_CAPS), times_ms=[float(t) for t in times])

    def batch_subcycle(self, split, boxes, pos_pool, vel_pool, n_sub: int, use_graph: bool = False, stream=None):
        """n_sub SKS sub-cycles of every box of `boxes` (list of BatchBox) in one
        batched pass per sub-cycle; use_graph captures them as a CUDA graph."""
        _dev_rows(pos_pool, "pos_pool")
        _dev_rows(vel_pool, "vel_pool")
        sp = _split_of(split)
        arr = _boxes_c(boxes)
        self._check(lib().hacc_batch_subcycle(self._h, ctypes.byref(sp._c()), len(boxes), arr, _ptr(pos_pool),
                                              _ptr(vel_pool), int(n_sub), int(bool(use_graph)),
                                              self._stream(stream)), "hacc_batch_subcycle")

    def batch_tick(self, split, boxes, pos_pool, vel_pool, stream=None):
        """One sub-cycle of every box (dt = its sub-cycle step, flags TICK_FIRST/LAST)."""
        _dev_rows(pos_pool, "pos_pool")
        _dev_rows(vel_pool, "vel_pool")
        sp = _split_of(split)
        arr = _boxes_c(boxes)
        self._check(lib().hacc_batch_tick(self._h, ctypes.byref(sp._c()), len(boxes), arr, _ptr(pos_pool),
                                          _ptr(vel_pool), self._stream(stream)), "hacc_batch_tick")

    def batch_tune(self, split, boxes, pos_pool, vel_pool, reps: int = 2, stream=None) -> dict:
        """Time every (item cap, variant) setting of the batched pair launch on this batch and keep
        the fastest for its geometry."""
        _dev_rows(pos_pool, "pos_pool")
        _dev_rows(vel_pool, "vel_pool")
        sp = _split_of(split)
        times = (ctypes.c_double * BATCH_TUNE_SETTINGS)()
        chosen = ctypes.c_int32(-1)
        self._check(lib().hacc_batch_tune(self._h, ctypes.byref(sp._c()), len(boxes), _boxes_c(boxes),
                                          _ptr(pos_pool), _ptr(vel_pool), int(reps), times, ctypes.byref(chosen),
                                          self._stream(stream)), "hacc_batch_tune")
        k = int(chosen.value)
        return dict(chosen=k, **(tune_setting(k, BATCH_TUNE_CAPS) if k >= 0 else {}),
                    times_ms=[float(t) for t in times])

    def batch_diagnostics(self, split, boxes, pos_pool, vel_pool, stream=None):
        """FP64 (momentum[3], kinetic, potential) of every box: a (len(boxes), 5) float64 CUDA tensor."""
        import torch
        _dev_rows(pos_pool, "pos_pool")
        _dev_rows(vel_pool, "vel_pool")
        sp = _split_of(split)
        out = torch.empty((max(1, len(boxes)), 5), dtype=torch.float64, device=pos_pool.device)
        self._check(lib().hacc_batch_diagnostics(self._h, ctypes.byref(sp._c()), len(boxes), _boxes_c(boxes),
                                                 _ptr(pos_pool), _ptr(vel_pool), _ptr(out), self._stream(stream)),
                    "hacc_batch_diagnostics")
        return out[:len(boxes)]

    # ---- precision variant: positions as (cell id, FP32 in-cell offset) -----
    def diagnostics_ci(self, box: Box, split, cell, off, vel, stream=None):
        """FP64 (momentum[3], kinetic, potential, sum m x[3]) of (cell, offset) positions: 8 float64."""
        import torch
        sp = _split_of(split)
        out = torch.empty(8, dtype=torch.float64, device=off.device)
        self._check(lib().hacc_diagnostics_ci(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), cell.shape[0],
                                              _ptr(cell), _ptr(off), _ptr(vel), _ptr(out), self._stream(stream)),
                    "hacc_diagnostics_ci")
        return out

    def ci_from_f64(self, box: Box, r_cut: float, pos64, mass=None, stream=None):
        """(n, 3) float64 CUDA positions -> (cell int32 (n,), off_m float32 (n, 4))."""
        import torch
        assert pos64.is_cuda and pos64.dtype == torch.float64 and pos64.is_contiguous() and pos64.shape[1] == 3
        n = pos64.shape[0]
        cell = torch.empty(n, dtype=torch.int32, device=pos64.device)
        off = torch.empty((n, 4), dtype=torch.float32, device=pos64.device)
        self._check(lib().hacc_ci_from_f64(self._h, ctypes.byref(box._c()), float(r_cut), n, _ptr(pos64),
                                           _ptr(mass), _ptr(cell), _ptr(off), self._stream(stream)),
                    "hacc_ci_from_f64")
        return cell, off

    def ci_to_f64(self, box: Box, r_cut: float, cell, off, stream=None):
        import torch
        out = torch.empty((cell.shape[0], 3), dtype=torch.float64, device=cell.device)
        self._check(lib().hacc_ci_to_f64(self._h, ctypes.byref(box._c()), float(r_cut), cell.shape[0], _ptr(cell),
                                         _ptr(off), _ptr(out), self._stream(stream)), "hacc_ci_to_f64")
        return out

    def sr_force_ci(self, box: Box, split, cell, off, stream=None):
        import torch
        sp = _split_of(split)
        acc = torch.empty_like(off)
        self._check(lib().hacc_sr_force_ci(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), cell.shape[0],
                                           _ptr(cell), _ptr(off), _ptr(acc), self._stream(stream)),
                    "hacc_sr_force_ci")
        return acc

    def subcycle_ci(self, box: Box, split, cell, off, vel, dt: float, n_sub: int, stream=None):
        sp = _split_of(split)
        self._check(lib().hacc_subcycle_ci(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), cell.shape[0],
                                           _ptr(cell), _ptr(off), _ptr(vel), float(dt), int(n_sub),
                                           self._stream(stream)), "hacc_subcycle_ci")

    def set_queue_order(self, heavy_first: bool):
        """Work-item order of large force launches: largest first (True, default) or cell order."""
        self._check(lib().hacc_set_queue_order(self._h, int(bool(heavy_first))), "hacc_set_queue_order")

    def set_variant(self, variant: int):
        self._check(lib().hacc_set_variant(self._h, int(variant)), "hacc_set_variant")

    def set_item_cap(self, cap: int, split_max: int = 0):
        """Particles per force work item at most: 16..160 with the cell's particles in sub-cell
        order (cells above split_max particles keep items of up to 160, 0 = no such limit),
        0 for input-row order and items of up to 160, or -1 (default): 48 for calls of up to
        2^22 particles, else 0."""
        self._check(lib().hacc_set_item_cap(self._h, int(cap), int(split_max)), "hacc_set_item_cap")

    def set_stencil(self, cells_per_rcut: int):
        """1: cells >= r_cut, 27-cell search (default); 2: cells >= r_cut/2, 125-cell search."""
        self._check(lib().hacc_set_stencil(self._h, int(cells_per_rcut)), "hacc_set_stencil")

    def stats_enable(self, timing: bool = False, counting: bool = False):
        self._check(lib().hacc_stats_enable(self._h, int(timing), int(counting)), "hacc_stats_enable")

    def stats_read(self, reset: bool = True) -> dict:
        st = _Stats()
        self._check(lib().hacc_stats_read(self._h, ctypes.byref(st), int(reset)), "hacc_stats_read")
        return dict(kernel_launches=st.kernel_launches, force_launches=st.force_launches, force_ms=st.force_ms,
                    candidate_pairs=st.candidate_pairs, within_pairs=st.within_pairs, evaluated_pairs=st.evaluated_pairs,
                    ml_rebins=st.ml_rebins, build_ms=st.build_ms, builds=st.builds)

    def scratch_bytes(self) -> int:
        return int(lib().hacc_ctx_scratch_bytes(self._h))

    def bin(self, box: Box, r_cut: float, pos, stream=None):
        """Wrap pos in place and bin it; returns (cell_id, cell_start, perm) int32 tensors."""
        import torch
        _dev_rows(pos, "pos")
        n = pos.shape[0]
        nc = box.nc or mesh_cells(box.L, r_cut)
        cell = torch.empty(n, dtype=torch.int32, device=pos.device)
        start = torch.empty(nc ** 3 + 1, dtype=torch.int32, device=pos.device)
        perm = torch.empty(n, dtype=torch.int32, device=pos.device)
        self._check(lib().hacc_bin(self._h, ctypes.byref(box._c()), float(r_cut), n, _ptr(pos), _ptr(cell),
                                   _ptr(start), _ptr(perm), self._stream(stream)), "hacc_bin")
        return cell, start, perm

    def sr_force(self, box: Box, split, pos, acc=None, pair_counts=None, stream=None):
        import torch
        _dev_rows(pos, "pos")
        sp = _split_of(split)
        if acc is None:
            acc = torch.empty_like(pos)
        _dev_rows(acc, "acc")
        self._check(lib().hacc_sr_force(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), pos.shape[0],
                                        _ptr(pos), _ptr(acc), _ptr(pair_counts), self._stream(stream)),
                    "hacc_sr_force")
        return acc

    def pair_counts(self, box: Box, split, pos, stream=None):
        """(candidate pairs, pairs inside the cutoff) of one force evaluation."""
        import torch
        pc = torch.zeros(2, dtype=torch.int64, device=pos.device)
        self.sr_force(box, split, pos, pair_counts=pc, stream=stream)
        self.sync(stream)
        c, w = pc.tolist()
        return int(c), int(w)

    def subcycle(self, box: Box, split, pos, vel, dt: float, n_sub: int, stream=None):
        _dev_rows(pos, "pos")
        _dev_rows(vel, "vel")
        sp = _split_of(split)
        self._check(lib().hacc_subcycle(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), pos.shape[0],
                                        _ptr(pos), _ptr(vel), float(dt), int(n_sub), self._stream(stream)),
                    "hacc_subcycle")

    def subcycle_ml(self, box: Box, split, pos, vel, dt: float, d: int, lmax: int, skin: float = 0.05,
                    levels=None, stream=None, lmin: int = 1):
        """One multi-level short-range step (kick counts from cell densities, Eq. (kicks), clamped
        to [lmin, lmax]) on a chaining mesh of ml_mesh_cells(L, r_cut, skin) cells per side."""
        _dev_rows(pos, "pos")
        _dev_rows(vel, "vel")
        sp = _split_of(split)
        self._check(lib().hacc_subcycle_ml(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), pos.shape[0],
                                           _ptr(pos), _ptr(vel), float(dt), int(d), int(lmin), int(lmax),
                                           float(skin), _ptr(levels), self._stream(stream)), "hacc_subcycle_ml")

    def step(self, box: Box, split, pm: PM, pos, vel, dt: float, n_c: int, stream=None):
        _dev_rows(pos, "pos")
        _dev_rows(vel, "vel")
        sp = _split_of(split)
        self._check(lib().hacc_step(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), ctypes.byref(pm._c()),
                                    pos.shape[0], _ptr(pos), _ptr(vel), float(dt), int(n_c), self._stream(stream)),
                    "hacc_step")

    def pm_force(self, box: Box, pm: PM, pos, acc=None, stream=None):
        import torch
        _dev_rows(pos, "pos")
        if acc is None:
            acc = torch.empty_like(pos)
        self._check(lib().hacc_pm_force(self._h, ctypes.byref(box._c()), ctypes.byref(pm._c()), pos.shape[0],
                                        _ptr(pos), _ptr(acc), self._stream(stream)), "hacc_pm_force")
        return acc

    def diagnostics(self, box: Box, split, pos, vel, stream=None):
        """FP64 (momentum[3], kinetic, potential) as a 5-element float64 CUDA tensor."""
        import torch
        _dev_rows(pos, "pos")
        _dev_rows(vel, "vel")
        sp = _split_of(split)
        out = torch.empty(5, dtype=torch.float64, device=pos.device)
        self._check(lib().hacc_diagnostics(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), pos.shape[0],
                                           _ptr(pos), _ptr(vel), _ptr(out), self._stream(stream)),
                    "hacc_diagnostics")
        return out

    # ---- host-buffer entry points (numpy or pinned CPU tensors) -------------
    @staticmethod
    def _host_ptr(a):
        import numpy as np
        if isinstance(a, np.ndarray):
            assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"] and a.ndim == 2 and a.shape[1] == 4
            return ctypes.c_void_p(a.ctypes.data)
        assert (not a.is_cuda) and a.is_contiguous() and a.dtype.is_floating_point
        return ctypes.c_void_p(a.data_ptr())

    def sr_force_host(self, box: Box, split, pos, acc, stream=None):
        sp = _split_of(split)
        self._check(lib().hacc_sr_force_host(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), len(pos),
                                             self._host_ptr(pos), self._host_ptr(acc), self._stream(stream)),
                    "hacc_sr_force_host")

    def subcycle_host(self, box: Box, split, pos, vel, dt: float, n_sub: int, stream=None):
        sp = _split_of(split)
        self._check(lib().hacc_subcycle_host(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()), len(pos),
                                             self._host_ptr(pos), self._host_ptr(vel), float(dt), int(n_sub),
                                             self._stream(stream)), "hacc_subcycle_host")

    def step_host(self, box: Box, split, pm: PM, pos, vel, dt: float, n_c: int, stream=None):
        sp = _split_of(split)
        self._check(lib().hacc_step_host(self._h, ctypes.byref(box._c()), ctypes.byref(sp._c()),
                                         ctypes.byref(pm._c()), len(pos), self._host_ptr(pos), self._host_ptr(vel),
                                         float(dt), int(n_c), self._stream(stream)), "hacc_step_host")


class Server:
    """Continuous-batching server over one Context (see hacc_server_* in include/hacc.h)."""

    def __init__(self, ctx: Context, split, pool_bytes: int, max_active_particles: int = 0):
        self.ctx = ctx
        self._h = ctypes.c_void_p()
        sp = _split_of(split)
        ctx._check(lib().hacc_server_create(ctypes.byref(self._h), ctx._h, ctypes.byref(sp._c()), int(pool_bytes),
                                            int(max_active_particles)), "hacc_server_create")
        self._keep = {}
        self._ids = (ctypes.c_int64 * 4096)()
        self._ids_cap = len(self._ids)

    def close(self):
        if self._h:
            lib().hacc_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, rid: int, L: float, pos_host, vel_host, h: float, steps: int):
        """Queue a run on host arrays (n, 4) float32 (numpy or pinned torch), updated in place when done."""
        self._keep[int(rid)] = (pos_host, vel_host)
        self.ctx._check(lib().hacc_server_submit(self._h, int(rid), float(L), len(pos_host),
                                                 Context._host_ptr(pos_host), Context._host_ptr(vel_host),
                                                 float(h), int(steps)), "hacc_server_submit")

    def tick(self, stream=None) -> dict:
        info = _TickInfo()
        cap = max(0, min(int(self._ids_cap), len(self._ids)))
        self.ctx._check(lib().hacc_server_tick(self._h, self.ctx._stream(stream), ctypes.byref(info), self._ids,
                                               cap), "hacc_server_tick")
        done = [int(self._ids[i]) for i in range(min(info.finished, cap))]
        for rid in done:
            self._keep.pop(rid, None)
        return dict(admitted=info.admitted, finished=info.finished, active=info.active, queued=info.queued,
                    particles=info.particles, free_rows=info.free_rows, finished_ids=done)
