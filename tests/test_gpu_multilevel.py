"""GPU multi-level step against the FP64 oracle (Sec. 3.1, Eq. (kicks))."""
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


@pytest.mark.parametrize("d,lmax", [(2, 4), (1, 3), (0, 3), (1000, 4)])
def test_multilevel_step_against_oracle(env, split_params, d, lmax):
    torch, hacc, ctx = env
    L = 20.0
    n = 6000
    pos = synth.blob_mixture(n, L, seed=81, n_blobs=8, sigma=0.7)
    vel = synth.gaussian_velocities(n, seed=81, sigma=0.05)
    sp = dict(split_params, eps=float(np.float32(0.01)))
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    nc = hacc.mesh_cells(L, sp["r_cut"])
    lev_o = oracle.ml_levels(pos, L, nc, d, lmax)
    xo, vo = oracle.subcycle_ml(pos, vel, L, sp, 0.1, lmax, lev_o)
    p, v = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    lev = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.subcycle_ml(hacc.Box(L=L), sp, p, v, 0.1, d, lmax, levels=lev)
    ctx.sync()
    assert np.array_equal(lev.cpu().numpy(), lev_o)          # integer decision, bit-exact
    if d not in (0, 1000):
        assert len(np.unique(lev_o)) > 1
    x = p.cpu().numpy().astype(np.float64)
    dd = x[:, :3] - xo
    dd -= L * np.round(dd / L)
    assert np.abs(dd).max() < 2e-5 * L
    vscale = np.sqrt((vo ** 2).sum(1).mean())
    assert np.abs(v.cpu().numpy()[:, :3] - vo).max() < 1e-3 * vscale
    assert np.all((x[:, :3] >= 0) & (x[:, :3] < L))


def test_multilevel_uniform_count_matches_subcycle(env, split_params):
    # every particle with k kicks: the same maps as k SKS sub-cycles
    torch, hacc, ctx = env
    L = 16.0
    pos = synth.blob_mixture(4000, L, seed=82)
    vel = synth.gaussian_velocities(4000, seed=82)
    sp = dict(split_params, eps=float(np.float32(0.01)))
    p1, v1 = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    p2, v2 = p1.clone(), v1.clone()
    ctx.subcycle_ml(hacc.Box(L=L), sp, p1, v1, 0.04, 0, 3)
    ctx.subcycle(hacc.Box(L=L), sp, p2, v2, 0.04, 3)
    ctx.sync()
    d = (p1 - p2).cpu().numpy()[:, :3]
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-5
    assert torch.allclose(v1, v2, rtol=0, atol=1e-4 * float(v2.abs().max()))
