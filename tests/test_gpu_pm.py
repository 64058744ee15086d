"""GPU parity of the long-range PM stage and of the full step (Eq. (tstep))
against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from oracle import pm as opm

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


@pytest.mark.parametrize("L,ng,n,seed", [(32.0, 32, 32768, 1), (24.0, 48, 9000, 2), (20.0, 16, 5000, 3)])
def test_pm_force_parity(env, L, ng, n, seed):
    torch, hacc, ctx = env
    pos = synth.blob_mixture(n, L, seed=seed)
    pos[:, 3] = np.random.default_rng(seed).uniform(0.5, 2.0, n).astype(np.float32)
    a = ctx.pm_force(hacc.Box(L=L, ng=ng), hacc.PM(), torch.from_numpy(pos).cuda()).cpu().numpy()
    ref = opm.pm_accel(pos[:, :3].astype(np.float64), pos[:, 3].astype(np.float64), L, ng)
    rms = np.sqrt((ref ** 2).sum(1).mean())
    assert np.abs(a[:, :3] - ref).max() / rms <= 1e-4
    assert np.all(a[:, 3] == 0)


def test_full_step_parity(env, split_params):
    torch, hacc, ctx = env
    L = 16.0
    pos = synth.blob_mixture(3000, L, seed=51, n_blobs=6, sigma=0.8)
    vel = synth.gaussian_velocities(3000, seed=51, sigma=0.1)
    sp = dict(split_params, eps=float(np.float32(0.01)))
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    dt, n_c = 0.05, 3
    xo, vo = oracle.step(pos, vel, L, sp, dt, n_c)
    p, v = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    ctx.step(hacc.Box(L=L), sp, hacc.PM(), p, v, dt, n_c)
    ctx.sync()
    x = p.cpu().numpy().astype(np.float64)
    vv = v.cpu().numpy().astype(np.float64)
    d = x[:, :3] - xo
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 2e-5 * L
    vscale = np.sqrt((vo ** 2).sum(1).mean())
    assert np.abs(vv[:, :3] - vo).max() < 1e-3 * vscale


@pytest.mark.parametrize("n", [4000, 5])   # 5: fewer particles than the copy chunks
def test_step_host_equals_device(env, split_params, n):
    torch, hacc, ctx = env
    L = 16.0
    pos = synth.blob_mixture(n, L, seed=52)
    vel = synth.gaussian_velocities(n, seed=52)
    p, v = torch.from_numpy(pos.copy()).cuda(), torch.from_numpy(vel.copy()).cuda()
    ctx.step(hacc.Box(L=L), split_params, hacc.PM(), p, v, 0.1, 2)
    ctx.sync()
    hp, hv = pos.copy(), vel.copy()
    ctx.step_host(hacc.Box(L=L), split_params, hacc.PM(), hp, hv, 0.1, 2)
    assert np.array_equal(p.cpu().numpy(), hp) and np.array_equal(v.cpu().numpy(), hv)
