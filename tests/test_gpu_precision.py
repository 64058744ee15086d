"""GPU tests of the precision variant: positions as (chaining-mesh cell id,
FP32 in-cell offset), FP64 only inside the stream.  At a box side of 512
cells, FP32 absolute positions round by up to ~3e-5 cells; the cell/offset
form keeps ~1e-7 cells.  Both are compared with the FP64 oracle on the same
FP64 positions."""
import numpy as np
import pytest

import oracle
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


def _f64_positions(n, L, seed):
    """FP64 positions that are not FP32 values (sub-ulp jitter on a blob mixture)."""
    p32 = synth.blob_mixture(n, L, seed=seed, n_blobs=max(2, n // 512))
    x = p32[:, :3].astype(np.float64)
    x += np.random.default_rng(seed).uniform(-0.5, 0.5, x.shape) * np.spacing(np.float32(L))
    return np.mod(x, L)


def _sp(split_params):
    sp = dict(split_params)
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    sp["eps"] = float(np.float32(sp["eps"]))
    return sp


def test_cell_offset_round_trip(env, split_params):
    torch, hacc, ctx = env
    L = 512.0
    x = _f64_positions(50000, L, 1)
    box = hacc.Box(L=L)
    cell, off = ctx.ci_from_f64(box, split_params["r_cut"], torch.from_numpy(x).cuda())
    back = ctx.ci_to_f64(box, split_params["r_cut"], cell, off).cpu().numpy()
    w = L / hacc.mesh_cells(L, split_params["r_cut"])
    assert np.abs(back - x).max() < 2.5e-7 * w
    o = off.cpu().numpy()
    assert np.all(np.abs(o[:, :3]) <= np.float32(w / 2) * (1 + 1e-6)) and np.all(o[:, 3] == 1)


@pytest.mark.parametrize("L,n", [(32.0, 32768), (512.0, 60000)])
def test_cell_offset_force_parity_and_precision(env, split_params, L, n):
    torch, hacc, ctx = env
    sp = _sp(split_params)
    x = _f64_positions(n, L, 2)
    ref, _ = oracle.force_mesh(np.concatenate([x, np.ones((n, 1))], 1), L, sp)
    rms = np.sqrt((ref ** 2).sum(1).mean())
    box = hacc.Box(L=L)
    cell, off = ctx.ci_from_f64(box, sp["r_cut"], torch.from_numpy(x).cuda())
    a_ci = ctx.sr_force_ci(box, sp, cell, off).cpu().numpy()[:, :3]
    err_ci = np.abs(a_ci - ref).max() / rms
    assert err_ci <= 1e-4, (err_ci, L)
    # the same positions rounded to FP32 absolute coordinates
    p32 = np.ones((n, 4), np.float32)
    p32[:, :3] = x.astype(np.float32)
    p32[:, :3][p32[:, :3] >= np.float32(L)] = 0
    a_abs = ctx.sr_force(box, sp, torch.from_numpy(p32).cuda()).cpu().numpy()[:, :3]
    err_abs = np.abs(a_abs - ref).max() / rms
    if L >= 512:
        assert err_abs > 5 * err_ci, (err_abs, err_ci)


def test_cell_offset_subcycle_against_oracle(env, split_params):
    torch, hacc, ctx = env
    L = 512.0
    n = 30000
    sp = dict(_sp(split_params), eps=float(np.float32(0.01)))
    x = _f64_positions(n, L, 3)
    vel = synth.gaussian_velocities(n, seed=3, sigma=0.1)
    pos = np.concatenate([x, np.ones((n, 1))], 1)
    xo, vo = oracle.subcycle(pos, vel, L, sp, 0.05, 4)
    box = hacc.Box(L=L)
    cell, off = ctx.ci_from_f64(box, sp["r_cut"], torch.from_numpy(x).cuda())
    v = torch.from_numpy(vel).cuda()
    ctx.subcycle_ci(box, sp, cell, off, v, 0.05, 4)
    xc = ctx.ci_to_f64(box, sp["r_cut"], cell, off).cpu().numpy()
    ctx.sync()
    d = xc - xo
    d -= L * np.round(d / L)
    err_ci = np.abs(d).max()
    # FP32 absolute path on the same run
    p32 = np.ones((n, 4), np.float32)
    p32[:, :3] = x.astype(np.float32)
    p = torch.from_numpy(p32).cuda()
    v2 = torch.from_numpy(vel).cuda()
    ctx.subcycle(box, sp, p, v2, 0.05, 4)
    d2 = p.cpu().numpy()[:, :3].astype(np.float64) - xo
    d2 -= L * np.round(d2 / L)
    err_abs = np.abs(d2).max()
    assert err_ci < 1e-5
    assert err_ci < err_abs / 10, (err_ci, err_abs)
    vscale = np.sqrt((vo ** 2).sum(1).mean())
    assert np.abs(v.cpu().numpy()[:, :3] - vo).max() < 1e-3 * vscale
