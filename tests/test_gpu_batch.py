"""GPU tests of the batched mode (many independent boxes per launch)."""
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


def _pool(specs, seed0=100):
    """Pack blob-mixture boxes (n, L) into one pool; returns pos, vel, boxes (offset, n, L)."""
    pos, vel, out, off = [], [], [], 0
    for k, (n, L) in enumerate(specs):
        pos.append(synth.blob_mixture(n, L, seed=seed0 + k, n_blobs=max(2, n // 400)))
        vel.append(synth.gaussian_velocities(n, seed=seed0 + k))
        out.append((off, n, L))
        off += n
    return np.concatenate(pos), np.concatenate(vel), out


SPECS = [(4096, 16.0), (9000, 20.0), (300, 10.0), (20000, float(np.float32(27.14))), (1, 12.0)]


def test_batch_matches_single_box_path(env, split_params):
    torch, hacc, ctx = env
    pos, vel, boxes = _pool(SPECS)
    P, V = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    bb = [hacc.BatchBox(L=L, offset=o, n=n, dt=0.1) for (o, n, L) in boxes]
    ctx.batch_subcycle(split_params, bb, P, V, n_sub=3)
    ctx.sync()
    for (o, n, L) in boxes:
        p1 = torch.from_numpy(pos[o:o + n].copy()).cuda()
        v1 = torch.from_numpy(vel[o:o + n].copy()).cuda()
        ctx.subcycle(hacc.Box(L=L), split_params, p1, v1, 0.1, 3)
        ctx.sync()
        d = (P[o:o + n] - p1).cpu().numpy()
        d[:, :3] -= L * np.round(d[:, :3] / L)
        assert np.abs(d).max() < 1e-5 * L
        assert torch.allclose(V[o:o + n], v1, rtol=0, atol=1e-4 * float(v1.abs().max()))
        xs = P[o:o + n, :3].cpu().numpy()
        assert np.all((xs >= 0) & (xs < L))


def test_batch_box_against_oracle(env, split_params):
    torch, hacc, ctx = env
    pos, vel, boxes = _pool(SPECS[:2])
    sp = dict(split_params, eps=float(np.float32(0.01)))
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    P, V = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    bb = [hacc.BatchBox(L=L, offset=o, n=n, dt=0.05) for (o, n, L) in boxes]
    ctx.batch_subcycle(sp, bb, P, V, n_sub=4)
    ctx.sync()
    for (o, n, L) in boxes:
        xo, vo = oracle.subcycle(pos[o:o + n], vel[o:o + n], L, sp, 0.05, 4)
        d = P[o:o + n, :3].cpu().numpy().astype(np.float64) - xo
        d -= L * np.round(d / L)
        assert np.abs(d).max() < 2e-5 * L
        vscale = np.sqrt((vo ** 2).sum(1).mean())
        assert np.abs(V[o:o + n, :3].cpu().numpy() - vo).max() < 1e-3 * vscale


def test_alone_equals_in_mix_bitwise(env, split_params):
    torch, hacc, ctx = env
    pos, vel, boxes = _pool(SPECS)
    P, V = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    ctx.batch_subcycle(split_params, [hacc.BatchBox(L=L, offset=o, n=n, dt=0.1) for (o, n, L) in boxes], P, V, 3)
    for k, (o, n, L) in enumerate(boxes):
        p1 = torch.from_numpy(pos[o:o + n].copy()).cuda()
        v1 = torch.from_numpy(vel[o:o + n].copy()).cuda()
        ctx.batch_subcycle(split_params, [hacc.BatchBox(L=L, offset=0, n=n, dt=0.1)], p1, v1, 3)
        assert torch.equal(P[o:o + n], p1) and torch.equal(V[o:o + n], v1), k


def test_graph_equals_direct_and_replays(env, split_params):
    torch, hacc, ctx = env
    pos, vel, boxes = _pool(SPECS)
    bb = [hacc.BatchBox(L=L, offset=o, n=n, dt=0.1) for (o, n, L) in boxes]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        P1, V1 = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
        P2, V2 = P1.clone(), V1.clone()
        for _ in range(2):
            ctx.batch_subcycle(split_params, bb, P1, V1, 4, use_graph=False, stream=s)
        for _ in range(2):      # first call captures, second replays the cached graph
            ctx.batch_subcycle(split_params, bb, P2, V2, 4, use_graph=True, stream=s)
    s.synchronize()
    assert torch.equal(P1, P2) and torch.equal(V1, V2)


def test_ticks_equal_subcycle(env, split_params):
    torch, hacc, ctx = env
    pos, vel, boxes = _pool(SPECS[:3])
    P1, V1 = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    P2, V2 = P1.clone(), V1.clone()
    ctx.batch_subcycle(split_params, [hacc.BatchBox(L=L, offset=o, n=n, dt=0.3) for (o, n, L) in boxes], P1, V1, 3)
    for k in range(3):
        flags = (hacc.TICK_FIRST if k == 0 else 0) | (hacc.TICK_LAST if k == 2 else 0)
        ctx.batch_tick(split_params, [hacc.BatchBox(L=L, offset=o, n=n, dt=0.1, flags=flags)
                                      for (o, n, L) in boxes], P2, V2)
    ctx.sync()
    assert torch.equal(P1, P2) and torch.equal(V1, V2)


def test_batch_candidate_count_exact(env, split_params):
    # at rest the batched sub-cycle bins the given positions; its 27-cell
    # candidate count is then the sum of every box's own count
    torch, hacc, ctx = env
    pos, _, boxes = _pool(SPECS)
    P = torch.from_numpy(pos).cuda()
    V = torch.zeros_like(P)
    bb = [hacc.BatchBox(L=L, offset=o, n=n, dt=0.1) for (o, n, L) in boxes]
    ctx.stats_read(reset=True)
    ctx.stats_enable(counting=True)
    ctx.batch_subcycle(split_params, bb, P, V, n_sub=1)
    st = ctx.stats_read(reset=True)
    ctx.stats_enable()
    want = 0
    for (o, n, L) in boxes:
        nc = hacc.mesh_cells(L, split_params["r_cut"])
        _, cell_o, _ = oracle.wrap_cell(pos[o:o + n], L, nc)
        count_o, _, _ = oracle.bin_cells(cell_o, nc)
        want += oracle.candidates(count_o, nc)
    assert st["candidate_pairs"] == want
    assert st["within_pairs"] <= st["evaluated_pairs"] <= st["candidate_pairs"]


def test_every_tuner_setting_sums_the_oracle_pairs(split_params):
    # Every (item cap, variant) setting the batched tuner can pick: with zero
    # velocities one tick is a pure kick, so v / h is each particle's force;
    # it matches the oracle per box, and the pairs inside the cutoff are the
    # oracle's.
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_2805_gb300 as hacc
    ctx = hacc.Context()
    sp = dict(split_params)
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    sp["eps"] = float(np.float32(sp["eps"]))
    pos, _, boxes = _pool(SPECS[:4], seed0=300)
    h = 0.01
    refs = []
    for (o, n, L) in boxes:
        a, w = oracle.force_mesh(pos[o:o + n], L, sp)
        refs.append((a, w))
    within_oracle = sum(w for _, w in refs)
    bb = [hacc.BatchBox(L=L, offset=o, n=n, dt=h, flags=hacc.TICK_FIRST | hacc.TICK_LAST) for (o, n, L) in boxes]
    seen = set()
    for k in range(hacc.BATCH_TUNE_SETTINGS):
        setting = hacc.tune_setting(k, hacc.BATCH_TUNE_CAPS)
        ctx.set_item_cap(setting["item_cap"])
        ctx.set_variant(setting["variant"])
        ctx.set_queue_order(setting["heavy_first"])
        P = torch.from_numpy(pos).cuda()
        V = torch.zeros_like(P)
        ctx.stats_read(reset=True)
        ctx.stats_enable(counting=True)
        ctx.batch_tick(sp, bb, P, V)
        st = ctx.stats_read(reset=True)
        ctx.stats_enable()
        ctx.sync()
        assert abs(st["within_pairs"] - within_oracle) <= 2
        seen.add(st["candidate_pairs"])
        v = V.cpu().numpy()[:, :3].astype(np.float64) / np.float64(np.float32(h))
        for (o, n, L), (a, _) in zip(boxes, refs):
            rms = np.sqrt((a ** 2).sum(1).mean())
            assert np.abs(v[o:o + n] - a).max() / rms <= 1e-4, (k, L)
    assert len(seen) == 1
    ctx.close()


def test_batch_tune_keeps_the_fastest_setting_for_the_geometry(split_params):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1410_2805_gb300 as hacc
    pos, vel, boxes = _pool(SPECS[:4], seed0=400)
    bb = [hacc.BatchBox(L=L, offset=o, n=n, dt=0.05) for (o, n, L) in boxes]
    ctx = hacc.Context()
    P, V = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    res = ctx.batch_tune(split_params, bb, P, V, reps=1)
    assert 0 <= res["chosen"] < hacc.BATCH_TUNE_SETTINGS and all(t > 0 for t in res["times_ms"])
    assert res["times_ms"][res["chosen"]] == min(res["times_ms"])
    assert torch.equal(P, torch.from_numpy(pos).cuda()) and torch.equal(V, torch.from_numpy(vel).cuda())
    ctx.batch_subcycle(split_params, bb, P, V, n_sub=3, use_graph=True)
    ctx.sync()
    # the same steps on a fresh context set to the chosen setting by hand
    ref = hacc.Context()
    ref.set_item_cap(res["item_cap"])
    ref.set_variant(res["variant"])
    ref.set_queue_order(res["heavy_first"])
    P2, V2 = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    ref.batch_subcycle(split_params, bb, P2, V2, n_sub=3, use_graph=True)
    ref.sync()
    assert torch.equal(P, P2) and torch.equal(V, V2)
    ctx.close()
    ref.close()
