"""Argument errors of the C ABI, called directly through ctypes: every entry
point returns its documented status, records a message, and leaves the
context usable."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_2805_gb300 as hacc
    from paper_1410_2805_gb300 import build
    build.build()
    ctx = hacc.Context()
    yield torch, hacc, ctx
    ctx.close()


def _p(t, byte_offset=0):
    return ctypes.c_void_p(t.data_ptr() + byte_offset)


def test_entry_points_refuse_bad_arguments(env, split_params):
    torch, hacc, ctx = env
    L = 16.0
    lib = hacc.lib()
    h = ctx._h
    box = hacc.Box(L=L)._c()
    sp = hacc.Split(**split_params)._c() if isinstance(split_params, dict) else split_params._c()
    pos = torch.from_numpy(synth.uniform(500, L, seed=3)).cuda()
    vel = torch.zeros_like(pos)
    acc = torch.empty_like(pos)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = pos.shape[0]
    E = hacc.HACC_EINVAL

    def last():
        return lib.hacc_last_error(h).decode()

    cases = [
        ("NULL split", lambda: lib.hacc_sr_force(h, ctypes.byref(box), None, n, _p(pos), _p(acc), None, s)),
        ("n < 0", lambda: lib.hacc_sr_force(h, ctypes.byref(box), ctypes.byref(sp), -1, _p(pos), _p(acc), None, s)),
        ("misaligned pos", lambda: lib.hacc_sr_force(h, ctypes.byref(box), ctypes.byref(sp), n - 1, _p(pos, 4),
                                                     _p(acc), None, s)),
        ("NULL acc", lambda: lib.hacc_sr_force(h, ctypes.byref(box), ctypes.byref(sp), n, _p(pos), None, None, s)),
        ("n_sub = 0", lambda: lib.hacc_subcycle(h, ctypes.byref(box), ctypes.byref(sp), n, _p(pos), _p(vel), 0.01,
                                                0, s)),
        ("NULL vel", lambda: lib.hacc_subcycle(h, ctypes.byref(box), ctypes.byref(sp), n, _p(pos), None, 0.01, 2, s)),
        ("lmax = 0", lambda: lib.hacc_subcycle_ml(h, ctypes.byref(box), ctypes.byref(sp), n, _p(pos), _p(vel), 0.01,
                                                  1, 1, 0, ctypes.c_float(0.05), None, s)),
        ("lmax = 17", lambda: lib.hacc_subcycle_ml(h, ctypes.byref(box), ctypes.byref(sp), n, _p(pos), _p(vel), 0.01,
                                                   1, 1, 17, ctypes.c_float(0.05), None, s)),
        ("lmin = 0", lambda: lib.hacc_subcycle_ml(h, ctypes.byref(box), ctypes.byref(sp), n, _p(pos), _p(vel), 0.01,
                                                  1, 0, 2, ctypes.c_float(0.05), None, s)),
        ("lmin > lmax", lambda: lib.hacc_subcycle_ml(h, ctypes.byref(box), ctypes.byref(sp), n, _p(pos), _p(vel),
                                                     0.01, 1, 3, 2, ctypes.c_float(0.05), None, s)),
        ("dt = nan", lambda: lib.hacc_subcycle_ml(h, ctypes.byref(box), ctypes.byref(sp), n, _p(pos), _p(vel),
                                                  float("nan"), 1, 1, 2, ctypes.c_float(0.05), None, s)),
        ("variant 4", lambda: lib.hacc_set_variant(h, hacc.FORCE_VARIANTS)),
        ("variant -1", lambda: lib.hacc_set_variant(h, -1)),
        ("stencil 0", lambda: lib.hacc_set_stencil(h, 0)),
        ("item cap 8", lambda: lib.hacc_set_item_cap(h, 8, 0)),
        ("item cap 161", lambda: lib.hacc_set_item_cap(h, 161, 0)),
        ("item cap -2", lambda: lib.hacc_set_item_cap(h, -2, 0)),
        ("split_max -1", lambda: lib.hacc_set_item_cap(h, 48, -1)),
        ("n_c = 0", lambda: lib.hacc_step(h, ctypes.byref(box), ctypes.byref(sp), ctypes.byref(hacc.PM()._c()), n,
                                          _p(pos), _p(vel), 0.01, 0, s)),
        ("NULL stats", lambda: lib.hacc_stats_read(h, None, 0)),
    ]
    for what, call in cases:
        st = call()
        assert st == E, (what, st)
        assert last(), what
    # a bad split: r_cut <= 0
    bad = hacc.Split(**dict(split_params, r_cut=0.0))._c() if isinstance(split_params, dict) else None
    assert lib.hacc_sr_force(h, ctypes.byref(box), ctypes.byref(bad), n, _p(pos), _p(acc), None, s) == E
    # the context still works
    a = ctx.sr_force(hacc.Box(L=L), split_params, pos)
    ctx.sync()
    assert torch.isfinite(a).all()


def test_zero_particles_is_a_no_op(env, split_params):
    torch, hacc, ctx = env
    p = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    v = torch.zeros_like(p)
    ctx.subcycle(hacc.Box(L=16.0), split_params, p, v, 0.01, 2)
    ctx.subcycle_ml(hacc.Box(L=16.0), split_params, p, v, 0.01, 1, 2)
    ctx.step(hacc.Box(L=16.0), split_params, hacc.PM(), p, v, 0.01, 2)
    ctx.sync()
