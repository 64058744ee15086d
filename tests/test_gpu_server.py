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


def test_admission_waits_for_scratch_budget(env, sp):
    # A context with an HBM budget: the pool has rows for both runs, but the
    # scratch of one batched pass over both would not fit beside the pool, so
    # the second run waits for the first to finish although rows are free.
    torch, hacc, _ = env
    boxes1 = [hacc.BatchBox(L=18.0, offset=0, n=5000, dt=0.01)]
    boxes2 = boxes1 + [hacc.BatchBox(L=18.0, offset=5000, n=5000, dt=0.01)]
    s1, s2 = hacc.batch_scratch_bytes(sp, boxes1), hacc.batch_scratch_bytes(sp, boxes2)
    assert 0 < s1 < s2
    pool = 32 * 12000
    budget = pool + s1 + (s2 - s1) // 2
    ctx = hacc.Context(hbm_budget_bytes=budget)
    srv = hacc.Server(ctx, sp, pool_bytes=pool)
    p1, v1 = _run(5000, 18.0, 30)
    p2, v2 = _run(5000, 18.0, 31)
    srv.submit(1, 18.0, p1, v1, h=0.01, steps=3)
    srv.submit(2, 18.0, p2, v2, h=0.01, steps=2)
    t = srv.tick()
    assert t["admitted"] == 1 and t["queued"] == 1 and t["active"] == 1
    assert t["free_rows"] == 7000            # rows for the second run are free
    assert ctx.scratch_bytes() <= budget - pool
    ticks = [t] + _drain(srv)
    assert all(x["active"] <= 1 for x in ticks)
    done = [i for x in ticks for i in x["finished_ids"]]
    assert done == [1, 2]
    srv.close()
    ctx.close()
    # each result is the one the run gets alone without a budget
    for (p0, v0, p, v, steps) in ((*_run(5000, 18.0, 30), p1, v1, 3), (*_run(5000, 18.0, 31), p2, v2, 2)):
        P, V = torch.from_numpy(p0).cuda(), torch.from_numpy(v0).cuda()
        env[2].batch_subcycle(sp, [hacc.BatchBox(L=18.0, offset=0, n=5000, dt=0.01 * steps)], P, V, steps)
        env[2].sync()
        assert np.array_equal(P.cpu().numpy(), p) and np.array_equal(V.cpu().numpy(), v)


def test_finished_runs_beyond_the_cap_are_reported_next_tick(env, sp):
    torch, hacc, ctx = env
    srv = hacc.Server(ctx, sp, pool_bytes=64 << 20)
    srv._ids_cap = 1   # report (and retire) one run per tick at most
    runs = [_run(1500, 14.0, 40 + k) for k in range(3)]
    for k, (p, v) in enumerate(runs):
        srv.submit(k, 14.0, p, v, h=0.01, steps=2)
    t = srv.tick()
    assert t["admitted"] == 3 and t["finished"] == 0
    t = srv.tick()                            # all three finish; one is retired
    assert t["finished_ids"] == [0] and t["active"] == 3
    t = srv.tick()                            # the others are not advanced again
    assert t["finished_ids"] == [1] and t["active"] == 0 and t["particles"] == 0
    t = srv.tick()
    assert t["finished_ids"] == [2]
    srv.close()
    # the held runs' results equal a run retired at once
    ref = _run(1500, 14.0, 42)
    P, V = torch.from_numpy(ref[0]).cuda(), torch.from_numpy(ref[1]).cuda()
    ctx.batch_subcycle(sp, [hacc.BatchBox(L=14.0, offset=0, n=1500, dt=0.02)], P, V, 2)
    ctx.sync()
    assert np.array_equal(P.cpu().numpy(), runs[2][0]) and np.array_equal(V.cpu().numpy(), runs[2][1])


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
