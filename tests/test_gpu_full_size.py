"""GPU parity at the full sizes of the benchmark workloads, through the same
launches the benchmark times: the 256^3 Zel'dovich box of the full step (pair
force and PM force on seeded samples of particles that the oracle computes one
by one; sub-cycles and the full step through properties that hold at any
size), the 512^3 precision box (cell/offset forces on a sample), and the
200-box batch (the smallest boxes stepped whole by the oracle).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import pm as opm

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
    ctx = hacc.Context()
    yield torch, hacc, ctx
    ctx.close()


@pytest.fixture(scope="module")
def zel256():
    # the full-step workload: 256^3 particles from Zel'dovich displacements
    # (P(k) ~ k^-2), box 256, Gaussian velocities sigma 0.1 (the benchmark's seed)
    pos = synth.zeldovich(256, seed=2, L=256.0)
    vel = synth.gaussian_velocities(len(pos), seed=2, sigma=0.1)
    return pos, vel, 256.0


def _f32_split(split_params):
    sp = dict(split_params)
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    sp["eps"] = float(np.float32(sp["eps"]))
    return sp


def test_zeldovich256_pair_force_sampled(env, split_params, zel256):
    torch, hacc, ctx = env
    pos, _, L = zel256
    sp = _f32_split(split_params)
    p = torch.from_numpy(pos).cuda()
    acc = ctx.sr_force(hacc.Box(L=L), sp, p)
    cand, within = ctx.pair_counts(hacc.Box(L=L), sp, p)
    a = acc.cpu().numpy()
    sel = np.sort(np.random.default_rng(256).choice(len(pos), size=4096, replace=False))
    ref, _ = oracle.force_mesh(pos, L, sp, sel=sel)
    rms = np.sqrt((ref ** 2).sum(1).mean())
    assert np.abs(a[sel, :3] - ref).max() / rms <= FORCE_TOL
    assert np.all(a[:, 3] == 0) and np.isfinite(a).all()
    nc = hacc.mesh_cells(L, sp["r_cut"])
    _, cell_o, ok = oracle.wrap_cell(pos, L, nc)
    count_o, _, _ = oracle.bin_cells(cell_o, nc)
    assert ok and cand == oracle.candidates(count_o, nc)
    assert 0 < within < cand
    # every pair force enters i and j with opposite signs: no net force
    m = pos[:, 3].astype(np.float64)
    ma = m[:, None] * a[:, :3].astype(np.float64)
    assert np.abs(ma.sum(0)).max() < 1e-5 * np.abs(ma).sum()


def test_zeldovich256_pm_force_sampled(env, zel256):
    torch, hacc, ctx = env
    pos, _, L = zel256
    ng = 256
    a = ctx.pm_force(hacc.Box(L=L, ng=ng), hacc.PM(), torch.from_numpy(pos).cuda()).cpu().numpy()
    sel = np.sort(np.random.default_rng(257).choice(len(pos), size=4096, replace=False))
    x = pos[:, :3].astype(np.float64)
    m = pos[:, 3].astype(np.float64)
    ref = opm.pm_accel(x[sel], m[sel], L, ng, sources=(x, m))
    rms = np.sqrt((ref ** 2).sum(1).mean())
    assert np.abs(a[sel, :3] - ref).max() / rms <= FORCE_TOL
    assert np.all(a[:, 3] == 0)


def _stream_f32(x, v, d, L):
    """The stream of the sub-cycle as the library stores it: x + d v rounded
    once to FP32 (the product is exact in FP64), then the FP32 wrap."""
    y = (x.astype(np.float64) + np.float64(d) * v.astype(np.float64)).astype(np.float32)
    Lf = np.float32(L)
    y = np.where(y < 0, y + Lf, np.where(y >= Lf, y - Lf, y)).astype(np.float32)
    y[y >= Lf] = 0
    return y


def test_zeldovich256_one_subcycle_kick_sampled(env, split_params, zel256):
    # The launch the benchmark times: kick + stream with cell-wide work items
    # (2^24 particles).  One SKS sub-cycle of step h: the velocity change of
    # sampled particles is h times the oracle force at the streamed positions.
    torch, hacc, ctx = env
    pos, vel, L = zel256
    sp = _f32_split(split_params)
    h = 0.1
    p, v = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    ctx.subcycle(hacc.Box(L=L), sp, p, v, h, 1)
    ctx.sync()
    p1, v1 = p.cpu().numpy(), v.cpu().numpy()
    h_f, h2 = np.float32(h), np.float32(0.5 * h)
    x1 = pos.copy()
    x1[:, :3] = _stream_f32(pos[:, :3], vel[:, :3], h2, L)
    sel = np.sort(np.random.default_rng(258).choice(len(pos), size=4096, replace=False))
    ref, _ = oracle.force_mesh(x1, L, sp, sel=sel)
    rms = np.sqrt((ref ** 2).sum(1).mean())
    a = (v1[sel, :3].astype(np.float64) - vel[sel, :3]) / np.float64(h_f)
    slack = 2 * np.spacing(np.abs(v1[sel, :3])).max() / h_f    # rounding of the stored velocity
    assert np.abs(a - ref).max() <= FORCE_TOL * rms + slack
    # the closing half stream from the kicked velocities, to one FP32 rounding
    x2 = _stream_f32(x1[:, :3], v1[:, :3], h2, L)
    d = np.abs(p1[:, :3].astype(np.float64) - x2)
    d = np.minimum(d, L - d)
    assert d.max() <= np.spacing(np.float32(L)) and (d > 0).mean() < 1e-5
    assert np.all(v1[:, 3] == 0)


def test_zeldovich256_subcycles_and_step_properties(env, split_params, zel256):
    torch, hacc, ctx = env
    pos, vel, L = zel256
    box = hacc.Box(L=L)
    # 5 sub-cycles of the step 0.5: antisymmetric kicks leave the momentum
    # unchanged, positions stay wrapped, and the result is reproducible
    p1, v1 = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    p2, v2 = p1.clone(), v1.clone()
    ctx.subcycle(box, split_params, p1, v1, 0.5, 5)
    ctx.subcycle(box, split_params, p2, v2, 0.5, 5)
    ctx.sync()
    assert torch.equal(p1, p2) and torch.equal(v1, v2)
    x = p1.cpu().numpy()
    assert np.isfinite(x).all() and np.all((x[:, :3] >= 0) & (x[:, :3] < L))
    dv = v1.cpu().numpy()[:, :3].astype(np.float64) - vel[:, :3]
    m = pos[:, 3].astype(np.float64)
    assert np.abs((m[:, None] * dv).sum(0)).max() < 1e-5 * (m[:, None] * np.abs(dv)).sum()
    # one full step (PM half kicks around the sub-cycles), twice from the same state
    p1, v1 = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    p2, v2 = p1.clone(), v1.clone()
    ctx.step(box, split_params, hacc.PM(), p1, v1, 0.5, 5)
    ctx.step(box, split_params, hacc.PM(), p2, v2, 0.5, 5)
    ctx.sync()
    assert torch.equal(p1, p2) and torch.equal(v1, v2)
    x, v = p1.cpu().numpy(), v1.cpu().numpy()
    assert np.isfinite(x).all() and np.isfinite(v).all()
    assert np.all((x[:, :3] >= 0) & (x[:, :3] < L))


def test_precision512_cell_offset_sampled(env, split_params):
    # The precision workload: 512^3 Zel'dovich particles, box 512, stored as
    # (cell id, FP32 in-cell offset) from FP64 positions.  Parity of the
    # kernel's arithmetic: the oracle takes the stored positions, decoded in
    # FP64 as (c + 1/2) W + off with W the FP32 value nearest L / nc, and every
    # sampled force must match it to max |da| / rms |a| <= 1e-4.  The storage
    # rounding is checked on its own against the FP64 generator positions.
    torch, hacc, ctx = env
    L = 512.0
    x64 = synth.zeldovich(512, seed=3, L=L, return_f64=True)
    n = len(x64)
    sp = _f32_split(split_params)
    box = hacc.Box(L=L)
    nc = hacc.mesh_cells(L, sp["r_cut"])
    cell, off = ctx.ci_from_f64(box, sp["r_cut"], torch.from_numpy(x64).cuda())
    a = ctx.sr_force_ci(box, sp, cell, off).cpu().numpy()[:, :3].astype(np.float64)
    c, o = cell.cpu().numpy().astype(np.int64), off.cpu().numpy()[:, :3].astype(np.float64)
    del cell, off
    torch.cuda.empty_cache()
    W = float(np.float32(L / nc))
    xs = np.empty((n, 4))
    xs[:, 0] = (c % nc + 0.5) * W + o[:, 0]
    xs[:, 1] = ((c // nc) % nc + 0.5) * W + o[:, 1]
    xs[:, 2] = (c // (nc * nc) + 0.5) * W + o[:, 2]
    xs[:, 3] = 1.0
    del c, o
    # storage: within half an ulp of an offset below 2 grid units
    d = xs[:, :3] - x64
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= 2.0 ** -24 * 2
    del d, x64
    sel = np.sort(np.random.default_rng(512).choice(n, size=8192, replace=False))
    ref, _ = oracle.force_mesh(xs, L, sp, sel=sel)
    del xs
    rms = np.sqrt((ref ** 2).sum(1).mean())
    err = np.sqrt(((a[sel] - ref) ** 2).sum(1)).max() / rms
    assert err <= FORCE_TOL, err
    assert np.isfinite(a).all()


def test_batch200_smallest_boxes_against_oracle(env, split_params):
    # the 200-box batch in one launch per sub-cycle; the oracle steps the
    # three smallest boxes whole
    torch, hacc, ctx = env
    specs = synth.batch_boxes(200, seed=4)
    pos, vel, boxes, off = [], [], [], 0
    for s in specs:
        pos.append(synth.blob_mixture_scaled(s.n, s.L, seed=s.seed))
        vel.append(synth.gaussian_velocities(s.n, seed=s.seed))
        boxes.append((off, s.n, s.L))
        off += s.n
    sp = dict(_f32_split(split_params), eps=float(np.float32(0.01)))
    P = torch.from_numpy(np.concatenate(pos)).cuda()
    V = torch.from_numpy(np.concatenate(vel)).cuda()
    ctx.batch_subcycle(sp, [hacc.BatchBox(L=L, offset=o, n=k, dt=0.05) for (o, k, L) in boxes], P, V, n_sub=4)
    ctx.sync()
    for b in np.argsort([k for (_, k, _) in boxes])[:3]:
        o, k, L = boxes[b]
        xo, vo = oracle.subcycle(pos[b], vel[b], L, sp, 0.05, 4)
        d = P[o:o + k, :3].cpu().numpy().astype(np.float64) - xo
        d -= L * np.round(d / L)
        assert np.abs(d).max() < 2e-5 * L
        vscale = np.sqrt((vo ** 2).sum(1).mean())
        assert np.abs(V[o:o + k, :3].cpu().numpy() - vo).max() < 1e-3 * vscale
    x = P.cpu().numpy()
    assert np.isfinite(x).all()


def test_over_2_24_particles_in_sub_cell_order(env, split_params, zel256):
    # more than 2^24 particles with an item cap: the in-cell order takes the
    # path for rows beyond 24 bits (cells of up to the cap by row, the others
    # by (sub-cell, row) relative to the cell's first row); the pairs summed
    # do not depend on the order, the forces only through rounding
    torch, hacc, ctx = env
    pos, _, L = zel256
    extra = synth.uniform(4096, L, seed=224)
    allp = np.concatenate([pos, extra])
    assert len(allp) > 1 << 24
    sp = _f32_split(split_params)
    p = torch.from_numpy(allp).cuda()
    box = hacc.Box(L=L)
    try:
        ctx.set_item_cap(0)
        a0 = ctx.sr_force(box, sp, p).cpu().numpy()
        counts0 = ctx.pair_counts(box, sp, p)
        ctx.set_item_cap(48)
        a48 = ctx.sr_force(box, sp, p).cpu().numpy()
        counts48 = ctx.pair_counts(box, sp, p)
    finally:
        ctx.set_item_cap(-1)
    assert counts48 == counts0
    rms = np.sqrt((a0[:, :3].astype(np.float64) ** 2).sum(1).mean())
    assert np.abs(a48[:, :3] - a0[:, :3]).max() / rms <= FORCE_TOL
    sel = np.sort(np.random.default_rng(224).choice(len(allp), size=1024, replace=False))
    ref, _ = oracle.force_mesh(allp, L, sp, sel=sel)
    assert np.abs(a48[sel, :3] - ref).max() / np.sqrt((ref ** 2).sum(1).mean()) <= FORCE_TOL
