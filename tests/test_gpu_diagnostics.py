"""GPU parity of the FP64 diagnostics per box (momentum, kinetic energy,
short-range pair potential energy) for batches of boxes and for positions
stored as (cell, FP32 offset), against the FP64 oracle."""
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


def _sp(split_params):
    sp = dict(split_params)
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    sp["eps"] = float(np.float32(sp["eps"]))
    return sp


def _check(out, pos, vel, L, sp):
    mom, ke, pe = oracle.diagnostics(pos[:, :3].astype(np.float64), vel[:, :3].astype(np.float64),
                                     pos[:, 3].astype(np.float64), L, sp)
    assert np.allclose(out[:3], mom, rtol=1e-12, atol=1e-9)
    assert out[3] == pytest.approx(ke, rel=1e-12)
    assert out[4] == pytest.approx(pe, rel=1e-4)


def test_batch_diagnostics_per_box_and_alone_equals_mix(env, split_params):
    torch, hacc, ctx = env
    sp = _sp(split_params)
    specs = [(3000, 15.0, 1), (0, 12.0, 2), (9000, 21.0, 3), (700, 10.0, 4), (20000, 27.0, 5)]
    pos, vel, boxes, off = [], [], [], 0
    for n, L, seed in specs:
        p = synth.blob_mixture_scaled(n, L, seed=seed) if n else np.zeros((0, 4), np.float32)
        if n:
            p[:, 3] = np.random.default_rng(seed).uniform(0.5, 2.0, n).astype(np.float32)
        v = synth.gaussian_velocities(n, seed=seed)
        pos.append(p)
        vel.append(v)
        boxes.append(hacc.BatchBox(L=L, offset=off, n=n, dt=0.0))
        off += n
    P = torch.from_numpy(np.concatenate(pos)).cuda()
    V = torch.from_numpy(np.concatenate(vel)).cuda()
    P0, V0 = P.clone(), V.clone()
    out = ctx.batch_diagnostics(sp, boxes, P, V).cpu().numpy()
    ctx.sync()
    assert out.shape == (5, 5)
    assert torch.equal(P, P0) and torch.equal(V, V0)        # the pools are only read
    assert np.all(out[1] == 0)                               # the empty box
    for b, (n, L, _) in enumerate(specs):
        if n:
            _check(out[b], pos[b], vel[b], L, sp)
    # each box alone (at another pool offset) gives the same bits
    for b, (n, L, _) in enumerate(specs):
        if not n:
            continue
        Pb = torch.zeros((n + 13, 4), dtype=torch.float32, device="cuda")
        Vb = torch.zeros_like(Pb)
        Pb[13:] = P[boxes[b].offset:boxes[b].offset + n]
        Vb[13:] = V[boxes[b].offset:boxes[b].offset + n]
        alone = ctx.batch_diagnostics(sp, [hacc.BatchBox(L=L, offset=13, n=n, dt=0.0)], Pb, Vb).cpu().numpy()
        assert np.array_equal(alone[0], out[b])


def test_batch_diagnostics_match_the_single_box_call(env, split_params):
    torch, hacc, ctx = env
    sp = _sp(split_params)
    L = 20.0
    pos = synth.blob_mixture_scaled(8000, L, seed=9)
    vel = synth.gaussian_velocities(8000, seed=9)
    P, V = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    one = ctx.diagnostics(hacc.Box(L=L), sp, P, V).cpu().numpy()
    bat = ctx.batch_diagnostics(sp, [hacc.BatchBox(L=L, offset=0, n=8000, dt=0.0)], P, V).cpu().numpy()[0]
    assert np.allclose(bat[:4], one[:4], rtol=1e-12, atol=1e-12)
    assert bat[4] == pytest.approx(one[4], rel=1e-5)


def test_cell_offset_diagnostics(env, split_params):
    torch, hacc, ctx = env
    sp = _sp(split_params)
    L = 512.0
    n = 40000
    p32 = synth.blob_mixture(n, L, seed=12, n_blobs=80)
    x = p32[:, :3].astype(np.float64)
    x += np.random.default_rng(12).uniform(-0.5, 0.5, x.shape) * np.spacing(np.float32(L))
    x = np.mod(x, L)
    m = np.random.default_rng(13).uniform(0.5, 2.0, n).astype(np.float32)
    vel = synth.gaussian_velocities(n, seed=12)
    box = hacc.Box(L=L)
    cell, off = ctx.ci_from_f64(box, sp["r_cut"], torch.from_numpy(x).cuda(), mass=torch.from_numpy(m).cuda())
    out = ctx.diagnostics_ci(box, sp, cell, off, torch.from_numpy(vel).cuda()).cpu().numpy()
    # the stored positions in FP64: (c + 1/2) W + off, W the FP32 value nearest L / nc
    nc = hacc.mesh_cells(L, sp["r_cut"])
    W = float(np.float32(L / nc))
    c = cell.cpu().numpy().astype(np.int64)
    o = off.cpu().numpy().astype(np.float64)
    xs = np.stack([c % nc, (c // nc) % nc, c // (nc * nc)], 1) * W + 0.5 * W + o[:, :3]
    pos = np.concatenate([xs, m[:, None].astype(np.float64)], 1)
    _check(out[:5], pos, vel, L, sp)
    assert np.allclose(out[5:], (m[:, None].astype(np.float64) * xs).sum(0), rtol=1e-13)
