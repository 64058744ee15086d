"""GPU tests of the serving runtime (continuous batching of short-range runs)."""
import numpy as np
import pytest

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


def _run(n, L, seed):
    return synth.blob_mixture_scaled(n, L, seed=seed), synth.gaussian_velocities(n, seed=seed)


@pytest.fixture(scope="module")
def sp(split_params):
    # softer than the default so that the short runs below stay well inside the box
    return dict(split_params, eps=0.01)


def _drain(srv, max_ticks=1000):
    ticks = []
    for _ in range(max_ticks):
        t = srv.tick()
        ticks.append(t)
        if t["active"] == 0 and t["queued"] == 0:
            break
    return ticks


def test_result_is_the_same_alone_and_in_the_mix(env, sp):
    torch, hacc, ctx = env
    pa, va = _run(5000, 18.0, 1)
    # alone
    srv = hacc.Server(ctx, sp, pool_bytes=64 << 20)
    a_pos, a_vel = pa.copy(), va.copy()
    srv.submit(1, 18.0, a_pos, a_vel, h=0.01, steps=6)
    _drain(srv)
    srv.close()
    # in a mix: one run already resident, one arriving two ticks later
    srv = hacc.Server(ctx, sp, pool_bytes=64 << 20)
    pb, vb = _run(12000, 24.0, 2)
    pc, vc = _run(800, 12.0, 3)
    m_pos, m_vel = pa.copy(), va.copy()
    srv.submit(2, 24.0, pb, vb, h=0.01, steps=9)
    srv.tick()
    srv.submit(1, 18.0, m_pos, m_vel, h=0.01, steps=6)
    srv.tick()
    srv.tick()
    srv.submit(3, 12.0, pc, vc, h=0.02, steps=3)
    _drain(srv)
    srv.close()
    assert np.array_equal(a_pos, m_pos) and np.array_equal(a_vel, m_vel)
    # and it is the batched sub-cycle of the same run
    P, V = torch.from_numpy(pa.copy()).cuda(), torch.from_numpy(va.copy()).cuda()
    ctx.batch_subcycle(sp, [hacc.BatchBox(L=18.0, offset=0, n=5000, dt=0.06)], P, V, 6)
    ctx.sync()
    assert np.array_equal(P.cpu().numpy(), a_pos) and np.array_equal(V.cpu().numpy(), a_vel)


def test_admission_waits_for_rows(env, sp):
    torch, hacc, ctx = env
    srv = hacc.Server(ctx, sp, pool_bytes=32 * 6000)     # room for one 5000-particle run
    p1, v1 = _run(5000, 18.0, 4)
    p2, v2 = _run(5000, 18.0, 5)
    srv.submit(10, 18.0, p1, v1, h=0.01, steps=3)
    srv.submit(11, 18.0, p2, v2, h=0.01, steps=2)
    t = srv.tick()
    assert t["admitted"] == 1 and t["queued"] == 1 and t["active"] == 1
    srv.tick()
    t = srv.tick()
    assert t["finished_ids"] == [10]
    t = srv.tick()
    assert t["admitted"] == 1 and t["active"] == 1
    t = srv.tick()
    assert t["finished_ids"] == [11] and t["free_rows"] == 6000
    srv.close()


def test_per_tick_particle_cap(env, sp):
    torch, hacc, ctx = env
    srv = hacc.Server(ctx, sp, pool_bytes=64 << 20, max_active_particles=6000)
    runs = [_run(2500, 14.0, 20 + k) for k in range(3)]
    for k, (p, v) in enumerate(runs):
        srv.submit(k, 14.0, p, v, h=0.01, steps=2)
    t = srv.tick()
    assert t["admitted"] == 2 and t["particles"] == 5000 and t["queued"] == 1
    ticks = _drain(srv)
    assert sum(x["finished"] for x in ticks) == 3
    srv.close()


def test_oversized_run_is_refused(env, sp):
    torch, hacc, ctx = env
    srv = hacc.Server(ctx, sp, pool_bytes=32 * 1000)
    p, v = _run(2000, 16.0, 6)
    with pytest.raises(hacc.HaccError) as e:
        srv.submit(1, 16.0, p, v, h=0.01, steps=2)
    assert e.value.status == hacc.HACC_ENOMEM
    srv.close()
