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


def _decode(cell, off, L, nc):
    """FP64 positions of stored (cell, FP32 offset) rows: (c + 1/2) W + off per
    axis, W = the FP32 value nearest L / nc (the storage definition)."""
    W = float(np.float32(L / nc))
    c = cell.astype(np.int64)
    idx = np.stack([c % nc, (c // nc) % nc, c // (nc * nc)], axis=1).astype(np.float64)
    return (idx + 0.5) * W + off[:, :3].astype(np.float64)


def test_cell_offset_round_trip(env, split_params):
    torch, hacc, ctx = env
    L = 512.0
    x = _f64_positions(50000, L, 1)
    # add points on the last cell and next to the box faces
    x[:6] = [[L - 1e-9, 0.0, 1e-12], [L - 1.5, L - 3.0, L - 0.25], [0.0, L / 2, L - 1e-6],
             [1e-9, 1e-9, 1e-9], [L * (1 - 1e-12), 3.1, 6.2], [255.0, 256.0, 257.0]]
    box = hacc.Box(L=L)
    nc = hacc.mesh_cells(L, split_params["r_cut"])
    cell, off = ctx.ci_from_f64(box, split_params["r_cut"], torch.from_numpy(x).cuda())
    back = ctx.ci_to_f64(box, split_params["r_cut"], cell, off).cpu().numpy()
    c, o = cell.cpu().numpy(), off.cpu().numpy()
    W = float(np.float32(L / nc))
    rem = L - nc * W
    assert abs(rem) < nc * np.spacing(np.float32(W)) and float(np.float32(rem)) == rem
    # the kernel's decode is the storage definition, and the storage rounds by
    # half an ulp of the offset at most
    assert np.array_equal(back, _decode(c, o, L, nc))
    assert np.abs(back - x).max() <= 2.0 ** -24 * 2
    # cells as defined: [c W, (c+1) W), the last one up to L
    idx = np.stack([c % nc, (c // nc) % nc, c // (nc * nc)], axis=1)
    lo = idx * W
    hi = np.where(idx == nc - 1, L, (idx + 1) * W)
    assert np.all((x >= lo) & (x < hi))
    assert np.all(np.abs(o[:, :3]) <= W / 2 + max(rem, 0.0) + 1e-6) and np.all(o[:, 3] == 1)


def test_cell_offset_close_pairs_across_faces_and_wrap(env, split_params):
    # Pairs closer than a few softening lengths that straddle chaining-mesh
    # faces, including the periodic wrap, on every axis: moving one offset into
    # the other's cell frame must not add rounding, so each particle's force
    # (dominated by its partner) matches the oracle on the stored positions to
    # a few FP32 roundings of the pair arithmetic.
    torch, hacc, ctx = env
    L = 512.0
    sp = _sp(split_params)
    nc = hacc.mesh_cells(L, sp["r_cut"])
    W = float(np.float32(L / nc))
    rng = np.random.default_rng(11)
    pts = []
    for axis in range(3):
        for face in [0.0, 1 * W, 57 * W, (nc - 1) * W, L]:   # 0 and L: the wrap
            for _ in range(6):
                sep = rng.uniform(0.005, 0.08)
                a = rng.uniform(0.0, sep)
                c = rng.uniform(20.0, L - 20.0, 3)
                c[axis] = face
                p, q = c.copy(), c.copy()
                p[axis] = face - a
                q[axis] = face - a + sep
                pts += [np.mod(p, L), np.mod(q, L)]
    x = np.array(pts)
    n = len(x)
    box = hacc.Box(L=L)
    cell, off = ctx.ci_from_f64(box, sp["r_cut"], torch.from_numpy(x).cuda())
    a = ctx.sr_force_ci(box, sp, cell, off).cpu().numpy()[:, :3].astype(np.float64)
    xs = _decode(cell.cpu().numpy(), off.cpu().numpy(), L, nc)
    ref, _ = oracle.force_mesh(np.concatenate([xs, np.ones((n, 1))], 1), L, sp)
    amag = np.sqrt((ref ** 2).sum(1))
    own = np.sqrt(((a - ref) ** 2).sum(1)) / amag
    assert own.max() <= 2e-6, own.max()


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
