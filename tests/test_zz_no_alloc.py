"""hacc_sr_force_noalloc, the allocation-free short-range force.

It serves callers that may not allocate device memory (their memory belongs
to another allocator or runtime, or allocation is closed after set-up): it
takes all scratch from one fixed device array inside the library.  This file
is collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_2805_gb300 as hacc
    from paper_1410_2805_gb300 import build
    build.build()
    lib = hacc.lib()
    fn = lib.hacc_sr_force_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(hacc._Box), ctypes.POINTER(hacc._Split), ctypes.c_int64, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    ctx = hacc.Context()
    yield torch, hacc, fn, ctx
    ctx.close()


def _noalloc(torch, hacc, fn, box, split, pos):
    acc = torch.full_like(pos, float("nan"))
    st = fn(ctypes.byref(box._c()), ctypes.byref(split._c()), pos.shape[0], ctypes.c_void_p(pos.data_ptr()),
            ctypes.c_void_p(acc.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, acc


def test_noalloc_matches_context_path_on_two_calls(env):
    torch, hacc, fn, ctx = env
    split = hacc.default_split()
    # two calls in a row on different boxes: the second must not see the first's data
    for n, L, seed in ((32768, 32.0, 1), (9001, 20.0, 2)):
        pos = torch.from_numpy(synth.blob_mixture(n, L, seed=seed)).cuda()
        box = hacc.Box(L=L)
        st, a_na = _noalloc(torch, hacc, fn, box, split, pos)
        assert st == hacc.HACC_OK
        a_ctx = ctx.sr_force(box, split, pos)
        torch.cuda.synchronize()
        a, b = a_na.cpu().numpy(), a_ctx.cpu().numpy()
        rms = np.sqrt((b[:, :3] ** 2).sum(1).mean())
        assert np.isfinite(a).all()
        assert np.abs(a - b).max() / rms <= FORCE_TOL


def test_noalloc_rejects_sizes_beyond_its_array(env):
    torch, hacc, fn, ctx = env
    split = hacc.default_split()
    n = 400000                                   # 48 B x n alone exceeds 16 MiB
    pos = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    st, acc = _noalloc(torch, hacc, fn, hacc.Box(L=64.0), split, pos)
    assert st == hacc.HACC_ENOMEM
    torch.cuda.synchronize()
    assert torch.isnan(acc).all()                # nothing was enqueued
