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


# (d, lmin, lmax); (2, 2, 4) is the paper's test: every particle at least two
# kicks, up to two more levels in the dense cells
@pytest.mark.parametrize("d,lmin,lmax", [(2, 1, 4), (1, 1, 3), (0, 1, 3), (1000, 1, 4), (2, 2, 4), (1000, 3, 4)])
def test_multilevel_step_against_oracle(env, split_params, d, lmin, lmax):
    torch, hacc, ctx = env
    L = 20.0
    n = 6000
    pos = synth.blob_mixture(n, L, seed=81, n_blobs=8, sigma=0.7)
    vel = synth.gaussian_velocities(n, seed=81, sigma=0.05)
    sp = dict(split_params, eps=float(np.float32(0.01)))
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    nc = hacc.ml_mesh_cells(L, sp["r_cut"], 0.05)
    lev_o = oracle.ml_levels(pos, L, nc, d, lmax, lmin=lmin)
    xo, vo = oracle.subcycle_ml(pos, vel, L, sp, 0.1, lmax, lev_o)
    p, v = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    lev = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.subcycle_ml(hacc.Box(L=L), sp, p, v, 0.1, d, lmax, levels=lev, lmin=lmin)
    ctx.sync()
    assert np.array_equal(lev.cpu().numpy(), lev_o)          # integer decision, bit-exact
    assert lev_o.min() >= lmin
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


# The step bins on a chaining mesh with cells at least r_cut (1 + skin) wide
# and keeps it while no particle has drifted past half of the excess width;
# the cases take each way through that: a mesh widened from 7 to 6 cells that
# holds for the whole step, violent motion from rest (rebinned during the
# step), a 3-cell box that cannot be widened, and no skin at all.
@pytest.mark.parametrize("case", ["kept", "rebinned", "small_box", "no_skin"])
def test_multilevel_skin_paths_against_oracle(env, split_params, case):
    torch, hacc, ctx = env
    # box, particles, velocity sigma, blob sigma, step, skin
    L, n, sig, bsig, dt, skin = {"kept": (22.0, 7000, 0.1, 1.5, 0.06, 0.05),
                                 "rebinned": (20.0, 6000, 0.0, 0.7, 0.1, 0.05),
                                 "small_box": (10.0, 2000, 0.5, 0.7, 0.1, 0.05),
                                 "no_skin": (22.0, 7000, 0.1, 1.5, 0.06, 0.0)}[case]
    pos = synth.blob_mixture(n, L, seed=83, n_blobs=8, sigma=bsig)
    vel = synth.gaussian_velocities(n, seed=83, sigma=sig) if sig > 0 else np.zeros((n, 4), np.float32)
    sp = dict(split_params, eps=float(np.float32(0.01)))
    sp["r_cut"] = float(np.float32(sp["r_cut"]))
    nc = hacc.ml_mesh_cells(L, sp["r_cut"], skin)
    assert nc == {"kept": 6, "rebinned": 6, "small_box": 3, "no_skin": 7}[case]
    d, lmax = 1, 3
    lev_o = oracle.ml_levels(pos, L, nc, d, lmax)
    xo, vo = oracle.subcycle_ml(pos, vel, L, sp, dt, lmax, lev_o)
    p, v = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    lev = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.stats_read(reset=True)
    ctx.subcycle_ml(hacc.Box(L=L), sp, p, v, dt, d, lmax, skin=skin, levels=lev)
    st = ctx.stats_read(reset=True)
    assert np.array_equal(lev.cpu().numpy(), lev_o)
    if case == "kept":
        assert st["ml_rebins"] == 0
    else:
        assert st["ml_rebins"] >= 1
    x = p.cpu().numpy().astype(np.float64)
    dd = x[:, :3] - xo
    dd -= L * np.round(dd / L)
    assert np.abs(dd).max() < 2e-5 * L
    vscale = np.sqrt((vo ** 2).sum(1).mean())
    assert np.abs(v.cpu().numpy()[:, :3] - vo).max() < 1e-3 * vscale
    assert np.all((x[:, :3] >= 0) & (x[:, :3] < L))


def test_multilevel_rejects_a_bad_skin(env, split_params):
    torch, hacc, ctx = env
    p = torch.from_numpy(synth.uniform(100, 16.0, seed=1)).cuda()
    v = torch.zeros_like(p)
    for bad in (-0.1, float("nan"), float("inf")):
        with pytest.raises(hacc.HaccError) as e:
            ctx.subcycle_ml(hacc.Box(L=16.0), split_params, p, v, 0.01, 1, 2, skin=bad)
        assert e.value.status == hacc.HACC_EINVAL


@pytest.mark.parametrize("case", ["kept", "rebinned"])
def test_multilevel_graph_equals_host_loop(env, split_params, case):
    # without timing or counting the event loop runs as a CUDA graph whose
    # rebinnings are conditional nodes; with counting on it runs from the host
    # (one drift read per event): the same kernels in the same order
    torch, hacc, ctx = env
    L, n, sig, bsig, dt = {"kept": (22.0, 7000, 0.1, 1.5, 0.06), "rebinned": (20.0, 6000, 0.0, 0.7, 0.1)}[case]
    pos = synth.blob_mixture(n, L, seed=84, n_blobs=8, sigma=bsig)
    vel = synth.gaussian_velocities(n, seed=84, sigma=sig) if sig > 0 else np.zeros((n, 4), np.float32)
    sp = dict(split_params, eps=float(np.float32(0.01)))
    runs = []
    for counting in (True, False, False):   # the second graph call replays the cached graph
        p, v = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
        ctx.stats_enable(counting=counting)
        ctx.stats_read(reset=True)
        ctx.subcycle_ml(hacc.Box(L=L), sp, p, v, dt, 1, 3)
        st = ctx.stats_read(reset=True)
        runs.append((p, v, st["ml_rebins"]))
    ctx.stats_enable()
    for p, v, rb in runs[1:]:
        assert torch.equal(p, runs[0][0]) and torch.equal(v, runs[0][1])
        assert rb == runs[0][2]
    assert (runs[0][2] == 0) == (case == "kept")
