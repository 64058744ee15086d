"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Binning (wrap, cell ids, cell starts, stable permutation) must match bit for
bit.  Forces must satisfy max_i |a_gpu - a_oracle| / rms_i |a_oracle| <= 1e-4
(FP32 pair arithmetic and accumulation against FP64).  The candidate-pair count
is exact; the inside-cutoff count may differ only by pairs whose FP32 and FP64
distances fall on opposite sides of r_cut (a few per million).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def hacc(torch):
    import paper_1410_2805_gb300 as h
    from paper_1410_2805_gb300 import build
    build.build()
    return h


@pytest.fixture(scope="module")
def ctx(hacc):
    c = hacc.Context()
    yield c
    c.close()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _force_err(a_gpu, a_ref):
    rms = np.sqrt((a_ref ** 2).sum(1).mean())
    return np.abs(a_gpu[:, :3] - a_ref).max() / rms


def _check_bin(torch, hacc, ctx, pos, L, r_cut):
    nc = hacc.mesh_cells(L, r_cut)
    wrapped_o, cell_o, ok = oracle.wrap_cell(pos, L, nc)
    assert ok
    count_o, start_o, perm_o = oracle.bin_cells(cell_o, nc)
    p = _dev(torch, pos)
    cell, start, perm = ctx.bin(hacc.Box(L=L), r_cut, p)
    ctx.sync()
    assert np.array_equal(p.cpu().numpy(), wrapped_o)
    assert np.array_equal(cell.cpu().numpy(), cell_o)
    assert np.array_equal(start.cpu().numpy(), start_o)
    assert np.array_equal(perm.cpu().numpy(), perm_o)


def test_bin_blob_mixture_bit_exact(torch, hacc, ctx, split_params):
    pos = synth.blob_mixture(32768, 32.0, seed=1)
    _check_bin(torch, hacc, ctx, pos, 32.0, np.float32(split_params["r_cut"]))


def test_bin_faces_and_wrap_bit_exact(torch, hacc, ctx, split_params):
    rc = np.float32(split_params["r_cut"])
    for L in (32.0, float(np.float32(45.254834)), 10.0):
        nc = hacc.mesh_cells(L, rc)
        rng = np.random.default_rng(5)
        xs = list(rng.uniform(-L, 2 * L, 2000).astype(np.float32))
        for k in range(nc + 1):
            b = np.float32(k * L / nc)
            xs += [np.nextafter(b, np.float32(-1e9)), b, np.nextafter(b, np.float32(1e9))]
        xs += [np.float32(-1e-9), np.float32(-L), np.float32(L), np.float32(-1e-30)]
        x = np.array(xs, np.float32)
        pos = np.stack([x, np.roll(x, 7), np.roll(x, 13), np.ones_like(x)], 1)
        _check_bin(torch, hacc, ctx, pos, L, rc)


def test_bin_empty_and_tiny(torch, hacc, ctx, split_params):
    rc = np.float32(split_params["r_cut"])
    for n in (0, 1, 2, 33):
        pos = synth.uniform(n, 16.0, seed=n) if n else np.zeros((0, 4), np.float32)
        if n == 0:
            p = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
            cell, start, perm = ctx.bin(hacc.Box(L=16.0), rc, p)
            ctx.sync()
            assert start.cpu().numpy().max() == 0
            continue
        _check_bin(torch, hacc, ctx, pos, 16.0, rc)


@pytest.mark.parametrize("case", ["c1", "ragged", "nc3", "odd_box", "masses_G", "eps0", "dense_cell"])
def test_sr_force_parity(torch, hacc, ctx, split_params, case):
    sp = dict(split_params)
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    sp["eps"] = float(np.float32(sp["eps"]))
    L = 32.0
    if case == "c1":
        pos = synth.blob_mixture(32768, L, seed=1)
    elif case == "ragged":
        pos = synth.blob_mixture(4099, 20.0, seed=2, n_blobs=7)
        L = 20.0
    elif case == "nc3":
        L = 9.5
        pos = synth.blob_mixture(900, L, seed=3, n_blobs=3)
    elif case == "odd_box":
        L = float(np.float32(45.254834))
        pos = synth.blob_mixture(20000, L, seed=4, n_blobs=40)
    elif case == "masses_G":
        L = 24.0
        pos = synth.blob_mixture(12000, L, seed=6, n_blobs=20)
        pos[:, 3] = np.random.default_rng(0).uniform(0.25, 4.0, len(pos)).astype(np.float32)
        sp["G"] = 0.75
    elif case == "eps0":
        L = 20.0
        pos = synth.uniform(6000, L, seed=7)
        sp["eps"] = 0.0
    else:   # one very crowded cell (several hundred particles) among sparse ones
        L = 24.0
        pos = synth.blob_mixture(6000, L, seed=8, n_blobs=2, sigma=0.4)
    a_ref, within_ref = oracle.force_mesh(pos, L, sp)
    p = _dev(torch, pos)
    acc = ctx.sr_force(hacc.Box(L=L), sp, p)
    cand, within = ctx.pair_counts(hacc.Box(L=L), sp, p)
    a = acc.cpu().numpy()
    assert np.all(a[:, 3] == 0)
    err = _force_err(a, a_ref)
    assert err <= FORCE_TOL, err
    # exact 27-cell candidate count from the oracle's own binning
    nc = hacc.mesh_cells(L, sp["r_cut"])
    _, cell_o, _ = oracle.wrap_cell(pos, L, nc)
    count_o, _, _ = oracle.bin_cells(cell_o, nc)
    assert cand == oracle.candidates(count_o, nc)
    assert abs(within - within_ref) <= max(2, within_ref // 200000)
    # counting variant gives bitwise the same forces
    acc2 = ctx.sr_force(hacc.Box(L=L), sp, p, pair_counts=torch.zeros(2, dtype=torch.int64, device="cuda"))
    assert torch.equal(acc, acc2)


def test_sr_force_deterministic_and_third_law(torch, hacc, ctx, split_params):
    pos = synth.blob_mixture(32768, 32.0, seed=11)
    p = _dev(torch, pos)
    a1 = ctx.sr_force(hacc.Box(L=32.0), split_params, p).clone()
    a2 = ctx.sr_force(hacc.Box(L=32.0), split_params, p)
    assert torch.equal(a1, a2)
    a = a1.double().cpu().numpy()[:, :3]
    m = pos[:, 3].astype(np.float64)
    assert np.abs((m[:, None] * a).sum(0)).max() < 1e-5 * (m[:, None] * np.abs(a)).sum()


def test_sr_force_lattice_zero(torch, hacc, ctx, split_params):
    pos = synth.lattice(16)
    a = ctx.sr_force(hacc.Box(L=16.0), split_params, _dev(torch, pos)).cpu().numpy()
    assert np.abs(a).max() < 1e-4


def test_sr_force_empty(torch, hacc, ctx, split_params):
    p = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    acc = ctx.sr_force(hacc.Box(L=16.0), split_params, p)
    ctx.sync()
    assert acc.shape == (0, 4)


def test_host_variant_equals_device(torch, hacc, ctx, split_params):
    pos = synth.blob_mixture(5000, 20.0, seed=12)
    a_dev = ctx.sr_force(hacc.Box(L=20.0), split_params, _dev(torch, pos)).cpu().numpy()
    a_host = np.zeros_like(pos)
    ctx.sr_force_host(hacc.Box(L=20.0), split_params, pos.copy(), a_host)
    assert np.array_equal(a_dev, a_host)


def test_errors(torch, hacc, ctx, split_params):
    p = _dev(torch, synth.uniform(100, 16.0, seed=1))
    with pytest.raises(hacc.HaccError) as e:
        ctx.sr_force(hacc.Box(L=8.0), split_params, p)          # < 3 cells
    assert e.value.status == hacc.HACC_EDOMAIN
    with pytest.raises(hacc.HaccError) as e:
        ctx.sr_force(hacc.Box(L=0.1 + 16.0), split_params, p)   # not an FP32 value
    assert e.value.status == hacc.HACC_EINVAL
    bad = synth.uniform(100, 16.0, seed=2)
    bad[5, 0] = 40.0                                            # outside [-L, 2L)
    ctx.sr_force(hacc.Box(L=16.0), split_params, _dev(torch, bad))
    with pytest.raises(hacc.HaccError) as e:
        ctx.sync()
    assert e.value.status == hacc.HACC_EDOMAIN
    ctx.sync()                                                  # flag was cleared


def test_subcycle_parity(torch, hacc, ctx, split_params):
    # FP32 drift/kick against the FP64 SKS oracle.  Positions carry FP32
    # rounding of ~ulp(L)/2 per stream; over 2*n_sub streams and the force
    # tolerance of 1e-4 per kick the trajectories stay within the bounds below.
    L = 16.0
    pos = synth.blob_mixture(3000, L, seed=21, n_blobs=6, sigma=0.8)
    vel = synth.gaussian_velocities(3000, seed=21, sigma=0.1)
    sp = dict(split_params, eps=float(np.float32(0.01)))
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    dt, nsub = 0.05, 4
    xo, vo = oracle.subcycle(pos, vel, L, sp, dt, nsub)
    p, v = _dev(torch, pos), _dev(torch, vel)
    ctx.subcycle(hacc.Box(L=L), sp, p, v, dt, nsub)
    ctx.sync()
    x = p.cpu().numpy().astype(np.float64)
    vv = v.cpu().numpy().astype(np.float64)
    d = x[:, :3] - xo
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 2e-5 * L
    vscale = np.sqrt((vo ** 2).sum(1).mean())
    assert np.abs(vv[:, :3] - vo).max() < 1e-3 * vscale
    assert np.all(x[:, 3] == pos[:, 3])
    assert np.all((x[:, :3] >= 0) & (x[:, :3] < L))


def test_diagnostics_parity(torch, hacc, ctx, split_params):
    L = 16.0
    pos = synth.blob_mixture(4000, L, seed=31, n_blobs=5)
    pos[:, 3] = np.random.default_rng(2).uniform(0.5, 2.0, len(pos)).astype(np.float32)
    vel = synth.gaussian_velocities(4000, seed=31)
    out = ctx.diagnostics(hacc.Box(L=L), split_params, _dev(torch, pos), _dev(torch, vel)).cpu().numpy()
    sp = dict(split_params)
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    sp["eps"] = float(np.float32(sp["eps"]))
    mom, ke, pe = oracle.diagnostics(pos[:, :3].astype(np.float64), vel[:, :3].astype(np.float64),
                                     pos[:, 3].astype(np.float64), L, sp)
    assert np.allclose(out[:3], mom, rtol=1e-12, atol=1e-9)
    assert out[3] == pytest.approx(ke, rel=1e-12)
    assert out[4] == pytest.approx(pe, rel=1e-4)


def test_every_kernel_variant_gives_the_same_forces(torch, hacc, ctx, split_params):
    pos = synth.blob_mixture(20000, 28.0, seed=61)
    p = _dev(torch, pos)
    box = hacc.Box(L=28.0)
    counts0 = ctx.pair_counts(box, split_params, p)
    res = ctx.tune(box, split_params, p, reps=1)
    assert 0 <= res["chosen"] < hacc.TUNE_SETTINGS and all(t > 0 for t in res["times_ms"])
    assert len(res["times_ms"]) == hacc.TUNE_SETTINGS and res["times_ms"][res["chosen"]] == min(res["times_ms"])
    assert res["item_cap"] in hacc.TUNE_CAPS and 0 <= res["variant"] < hacc.FORCE_VARIANTS
    # the tuned setting is the context's now: the same forces as setting it by hand
    a_tuned = ctx.sr_force(box, split_params, p).clone()
    ctx.set_item_cap(res["item_cap"])
    ctx.set_variant(res["variant"])
    assert torch.equal(ctx.sr_force(box, split_params, p), a_tuned)
    # every variant, at every cap the tuner tries, gives bitwise the same forces as variant 0
    sp = dict(split_params)
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    sp["eps"] = float(np.float32(sp["eps"]))
    ref_o, _ = oracle.force_mesh(pos, 28.0, sp)
    rms = np.sqrt((ref_o ** 2).sum(1).mean())
    for cap in hacc.TUNE_CAPS:
        ctx.set_item_cap(cap)
        ref = None
        for v in range(hacc.FORCE_VARIANTS):
            ctx.set_variant(v)
            a = ctx.sr_force(box, split_params, p).clone()
            if ref is None:
                assert np.abs(a.cpu().numpy()[:, :3] - ref_o).max() / rms <= 1e-4, (cap, v)
                ref = a
            assert torch.equal(a, ref), (cap, v)
            assert ctx.pair_counts(box, split_params, p) == counts0
    ctx.set_item_cap(-1)
    ctx.set_variant(0)
    ctx.set_queue_order(False)


def test_bin_crowded_cells_bit_exact(torch, hacc, ctx, split_params):
    # cells of several thousand particles take the block-level chunk + merge ordering
    pos = synth.blob_mixture(30000, 24.0, seed=71, n_blobs=3, sigma=0.3)
    _check_bin(torch, hacc, ctx, pos, 24.0, np.float32(split_params["r_cut"]))
    _, cell_o, _ = oracle.wrap_cell(pos, 24.0, hacc.mesh_cells(24.0, np.float32(split_params["r_cut"])))
    assert np.bincount(cell_o).max() > 4096


def test_bounding_box_cull_counts(torch, hacc, ctx, split_params):
    # the pair kernel evaluates the 27-cell candidates minus the j it drops
    # as farther than r_cut from the item's bounds: never fewer than the
    # pairs inside the cutoff, never more than the candidates, and on a
    # uniform box a clear share of the candidates is dropped
    L = 40.0
    pos = synth.uniform(40000, L, seed=91)
    p = _dev(torch, pos)
    ctx.stats_read(reset=True)
    ctx.stats_enable(counting=True)
    ctx.sr_force(hacc.Box(L=L), split_params, p)
    st = ctx.stats_read(reset=True)
    ctx.stats_enable()
    cand, within, ev = st["candidate_pairs"], st["within_pairs"], st["evaluated_pairs"]
    nc = hacc.mesh_cells(L, split_params["r_cut"])
    _, cell_o, _ = oracle.wrap_cell(pos, L, nc)
    count_o, _, _ = oracle.bin_cells(cell_o, nc)
    assert cand == oracle.candidates(count_o, nc)
    assert within < ev < 0.9 * cand


@pytest.mark.parametrize("case", ["zeldovich", "blob"])
def test_item_caps_against_oracle(torch, hacc, ctx, split_params, case):
    # every item cap sums the same pairs: forces within the bar of the oracle,
    # the same candidate and inside-cutoff counts; items that cover part of a
    # cell (sub-cell order) evaluate no more pairs than cell-wide ones when
    # every cell is a single cell-wide item, and fewer at the smallest cap
    if case == "zeldovich":
        L, pos = 32.0, synth.zeldovich(32, seed=95, L=32.0, sigma_delta=0.7)
    else:   # dense cells of several hundred and over 512 particles among sparse ones
        L, pos = 24.0, synth.blob_mixture(12000, 24.0, seed=96, n_blobs=3, sigma=0.35)
    sp = dict(split_params)
    a_ref, within_ref = oracle.force_mesh(pos, L, sp)
    nc = hacc.mesh_cells(L, sp["r_cut"])
    _, cell_o, _ = oracle.wrap_cell(pos, L, nc)
    count_o, _, _ = oracle.bin_cells(cell_o, nc)
    if case == "blob":
        assert count_o.max() > 512
    p = _dev(torch, pos)
    res = {}
    try:
        for cap, split_max in ((0, 0), (16, 100000), (24, 0), (40, 64), (160, 0)):
            ctx.set_item_cap(cap, split_max)
            a = ctx.sr_force(hacc.Box(L=L), sp, p).cpu().numpy()
            assert _force_err(a, a_ref) <= FORCE_TOL, (cap, _force_err(a, a_ref))
            ctx.stats_read(reset=True)
            ctx.stats_enable(counting=True)
            ctx.sr_force(hacc.Box(L=L), sp, p)
            st = ctx.stats_read(reset=True)
            ctx.stats_enable()
            res[cap] = (st["candidate_pairs"], st["within_pairs"], st["evaluated_pairs"])
    finally:
        ctx.set_item_cap(-1, 0)
    cand = oracle.candidates(count_o, nc)
    for cap, (c, w, e) in res.items():
        assert c == cand and w == res[0][1] and w <= e <= c, cap
    assert abs(res[0][1] - within_ref) <= max(2, within_ref // 200000)
    if count_o.max() <= 160:
        assert all(res[cap][2] <= res[0][2] for cap in res)
        assert res[16][2] < 0.9 * res[0][2]


def _candidates_numpy(pos, L, nc, R):
    # sum over cells of n_c times the particles of the (2R+1)^3 cells around it
    _, cell_o, _ = oracle.wrap_cell(pos, L, nc)
    cnt = np.bincount(cell_o, minlength=nc ** 3).reshape(nc, nc, nc).astype(np.int64)
    nb = np.zeros_like(cnt)
    for a in range(-R, R + 1):
        for b in range(-R, R + 1):
            for c in range(-R, R + 1):
                nb += np.roll(np.roll(np.roll(cnt, a, 0), b, 1), c, 2)
    return int((cnt * nb).sum())


@pytest.mark.parametrize("case", ["blob", "zeldovich"])
def test_fine_mesh_stencil_against_oracle(torch, hacc, ctx, split_params, case):
    # cells >= r_cut/2 searched over 125 cells: the same pairs as the 27-cell
    # search (the same image shifts, so the same FP32 separations)
    if case == "blob":
        L, pos = 24.0, synth.blob_mixture(6000, 24.0, seed=93, n_blobs=4, sigma=0.6)
    else:
        L, pos = 32.0, synth.zeldovich(32, seed=94, L=32.0)
    sp = split_params
    a_ref, _ = oracle.force_mesh(pos, L, sp)
    p = _dev(torch, pos)
    box = hacc.Box(L=L)
    cand1, within1 = ctx.pair_counts(box, sp, p)
    a1 = ctx.sr_force(box, sp, p).cpu().numpy()
    ctx.set_stencil(2)
    try:
        cand2, within2 = ctx.pair_counts(box, sp, p)
        a2 = ctx.sr_force(box, sp, p).cpu().numpy()
    finally:
        ctx.set_stencil(1)
    assert _force_err(a2, a_ref) <= FORCE_TOL
    assert within2 == within1
    nc2 = hacc.mesh_cells(L, np.float32(sp["r_cut"]) / 2)
    assert cand2 == _candidates_numpy(pos, L, nc2, 2)
    assert cand1 == _candidates_numpy(pos, L, hacc.mesh_cells(L, sp["r_cut"]), 1)
    assert cand2 < 0.75 * cand1
    # the two are FP32 sums of the same pairs in different orders
    assert _force_err(a2, a1[:, :3].astype(np.float64)) <= FORCE_TOL


def test_fine_mesh_subcycle_and_limits(torch, hacc, ctx, split_params):
    L = 24.0
    pos = synth.blob_mixture(8000, L, seed=95)
    vel = synth.gaussian_velocities(8000, seed=95)
    sp = dict(split_params, eps=float(np.float32(0.01)))
    p1, v1 = _dev(torch, pos), _dev(torch, vel)
    p2, v2 = p1.clone(), v1.clone()
    ctx.subcycle(hacc.Box(L=L), sp, p1, v1, 0.05, 3)
    ctx.set_stencil(2)
    try:
        ctx.subcycle(hacc.Box(L=L), sp, p2, v2, 0.05, 3)
        # fewer than 5 cells of width r_cut/2 per side
        with pytest.raises(hacc.HaccError) as e:
            ctx.sr_force(hacc.Box(L=7.0), sp, _dev(torch, synth.uniform(100, 7.0, seed=1)))
        assert e.value.status == hacc.HACC_EDOMAIN
    finally:
        ctx.set_stencil(1)
    d = (p1 - p2).cpu().numpy()[:, :3]
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-5 * L
    with pytest.raises(hacc.HaccError) as e:
        ctx.set_stencil(3)
    assert e.value.status == hacc.HACC_EINVAL


def test_fine_mesh_smallest_box_against_brute_force(torch, hacc, ctx, split_params):
    # L = 9 holds 5 cells of width >= r_cut/2 (the 125-cell stencil then spans
    # the whole box once) but fewer than 3 cells of width >= r_cut: only the
    # finer mesh can take it; brute force over all pairs is the reference
    L = 9.0
    sp = split_params
    assert hacc.mesh_cells(L, np.float32(sp["r_cut"]) / 2) == 5 and hacc.mesh_cells(L, sp["r_cut"]) == -1
    pos = synth.blob_mixture(700, L, seed=96, n_blobs=3, sigma=0.5)
    a_ref, _ = oracle.force_brute(pos, L, sp)
    p = _dev(torch, pos)
    ctx.set_stencil(2)
    try:
        a = ctx.sr_force(hacc.Box(L=L), sp, p).cpu().numpy()
    finally:
        ctx.set_stencil(1)
    assert _force_err(a, a_ref) <= FORCE_TOL
    with pytest.raises(hacc.HaccError) as e:
        ctx.sr_force(hacc.Box(L=L), sp, p)
    assert e.value.status == hacc.HACC_EDOMAIN


def test_bin_every_in_cell_ordering_path_bit_exact(torch, hacc, ctx, split_params):
    # cells holding counts on both sides of every ordering path's bound (the
    # register stretches and the 32-key network, the 64/128/256-key networks,
    # counting above 256, the big-cell sort above 512), with input rows
    # shuffled (few stretches), cell-sorted (long stretches) and in runs of 3
    # (lattice-like stretches); the order must be the stable one, bit for bit
    rc = np.float32(split_params["r_cut"])
    L = 32.0
    nc = hacc.mesh_cells(L, rc)
    w = L / nc
    counts = [1, 2, 16, 31, 32, 33, 48, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256, 257, 400, 511, 512, 513, 700]
    rng = np.random.default_rng(91)
    cells = rng.choice(nc ** 3, size=len(counts), replace=False)
    per_cell = np.full(nc ** 3, 20)
    per_cell[cells] = counts
    ids = np.repeat(np.arange(nc ** 3), per_cell)
    cz, cy, cx = ids // (nc * nc), (ids // nc) % nc, ids % nc
    frac = rng.uniform(0.02, 0.98, (len(ids), 3))
    xyz = (np.stack([cx, cy, cz], 1) + frac) * w
    base = np.concatenate([xyz, np.ones((len(ids), 1))], 1).astype(np.float32)
    orders = {"shuffled": rng.permutation(len(ids)), "cell_sorted": np.arange(len(ids))}
    runs = rng.permutation(len(ids) // 3)
    orders["runs_of_3"] = np.concatenate([(runs[:, None] * 3 + np.arange(3)[None, :]).ravel(),
                                          np.arange(len(ids) // 3 * 3, len(ids))])
    for name, order in orders.items():
        pos = base[order]
        _, cell_o, _ = oracle.wrap_cell(pos, L, nc)
        assert sorted(np.bincount(cell_o, minlength=nc ** 3)[cells]) == sorted(counts), name
        _check_bin(torch, hacc, ctx, pos, L, rc)
