"""Continuous-batching server (grng_server_*): each result is the same alone
and in the mix.

Requests arrive from a separate thread while earlier batches are on the GPU,
are admitted under a device-memory budget and packed into batches on two
stream slots.  Every completed output must equal the same parts generated
alone by grng_generate (the FastCaloSim layout: 3h FP32 uniforms then h FP32
gaussians from word 3h of the event's own Philox engine), the budget must
never be exceeded, and the latency statistics must cover every request.
"""

import threading
import time

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2109_01329_gb300 as grng

    return grng


def _event_parts(g, h):
    return [(g.Distribution.uniform(0.0, 1.0, g.F32), 3 * h),
            (g.Distribution.gaussian(0.0, 1.0, g.F32), h)]


def _alone(g, seed, h):
    """The event's numbers generated alone: the same engine, one call per part."""
    e = g.Engine(0, seed, 0)
    u = torch.empty(3 * h, dtype=torch.float32, device="cuda")
    z = torch.empty(h, dtype=torch.float32, device="cuda")
    g.generate(g.Distribution.uniform(0.0, 1.0, g.F32), e, u)
    g.generate(g.Distribution.gaussian(0.0, 1.0, g.F32), e, z)
    return torch.cat([u, z])


def test_results_alone_equal_in_the_mix(g):
    rng = np.random.Generator(np.random.PCG64(5))
    hits = [int(x) for x in np.clip(np.rint(np.exp(rng.normal(7.5, 0.9, 300))), 1, 60000)]
    srv = g.Server(64 << 20, num_streams=2)
    tickets = [None] * len(hits)

    def arrivals():
        for i, h in enumerate(hits):
            tickets[i] = srv.submit(g.serve_request(1000 + i, _event_parts(g, h)))
            if i % 7 == 0:
                time.sleep(0.0005)

    th = threading.Thread(target=arrivals)
    th.start()
    th.join()
    for i, h in enumerate(hits):
        out = srv.output(tickets[i]).view(torch.float32)
        assert out.numel() == 4 * h
        ref = _alone(g, 1000 + i, h)
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32)), f"event {i}"
        srv.release(tickets[i])
    st = srv.stats()
    assert st["completed"] == len(hits) and st["submitted"] == len(hits)
    assert st["samples"] == sum(4 * h for h in hits)
    assert 0 < st["latency_p50_us"] <= st["latency_p99_us"] <= st["latency_max_us"]
    assert st["peak_pool_bytes"] <= 64 << 20
    # one oracle spot check of the FastCaloSim layout
    h = hits[0]
    out = _alone(g, 1000, h).cpu().numpy()
    ref_u = oracle.generate(0, 1000, 0, 1, 1, 0.0, 1.0, 3 * h)
    ref_z = oracle.generate(0, 1000, 3 * h, 2, 1, 0.0, 1.0, h)
    assert np.array_equal(out[:3 * h].view(np.uint32), ref_u.view(np.uint32))
    assert np.all(np.abs(out[3 * h:] - ref_z) <= 2e-6 * np.maximum(1, np.abs(ref_z)))
    srv.close()


def test_budget_binds_and_waits_for_releases(g):
    # ~2.2 MB tables per slot plus a 6 MiB output budget; events of 0.4-1.6 MB
    srv = g.Server((2 * 1750 << 10) + (6 << 20), num_streams=2)
    hits = [100000, 350000, 250000, 300000, 150000, 340000, 50000, 330000]
    tickets = [srv.submit(g.serve_request(7 + i, _event_parts(g, h))) for i, h in enumerate(hits)]
    for i, h in enumerate(hits):
        out = srv.output(tickets[i]).view(torch.float32)
        assert torch.equal(out.view(torch.int32), _alone(g, 7 + i, h).view(torch.int32))
        srv.release(tickets[i])  # frees space for the requests still queued
    assert srv.stats()["peak_pool_bytes"] <= (6 << 20) + (256 << 10)
    # a request larger than the whole budget is refused
    with pytest.raises(g.GrngError) as ei:
        srv.submit(g.serve_request(1, _event_parts(g, 4_000_000)))
    assert ei.value.status == 6  # GRNG_ERR_BUDGET
    srv.close()


def test_replay_auto_release_and_stats(g):
    from paper_2109_01329_gb300 import workloads as W

    t, hits = W.fastcalosim_events(rate_hz=2000.0, duration_s=0.5, seed=3)
    reqs = [g.serve_request(i + 1, _event_parts(g, int(h))) for i, h in enumerate(hits)]
    srv = g.Server(256 << 20, num_streams=3, auto_release=True)
    srv.replay(t, reqs, time_scale=1.0)
    srv.drain()
    st = srv.stats()
    assert st["completed"] == len(reqs) == st["submitted"]
    assert st["samples"] == int(4 * hits.sum())
    assert st["latency_p99_us"] > 0 and st["batches"] >= 1
    srv.close()


def test_wait_times_out_then_completes(g):
    srv = g.Server(1 << 30, num_streams=1)
    big = [srv.submit(g.serve_request(50 + i, _event_parts(g, 20_000_000))) for i in range(3)]
    with pytest.raises(g.GrngError) as ei:
        srv.wait(big[-1], timeout_s=0.0)
    assert ei.value.status == 5  # GRNG_ERR_TIMEOUT
    for t in big:
        srv.wait(t, timeout_s=60.0)
        srv.release(t)
    srv.close()


def test_held_outputs_make_the_budget_bind(g):
    """Auto-released outputs held for a while after completion (a consumer
    keeping each event's numbers) fill the budget: admission then waits for
    held outputs to be let go, the pool never exceeds the budget, every
    request completes, and the waits show in the admission statistics."""
    budget = 8 << 20
    srv = g.Server((3 * 1750 << 10) + budget, num_streams=3, auto_release=True)
    srv.set_release_delay(0.05)
    hits = [200_000] * 24  # 3.2 MB per event: about two fit at a time
    t = np.arange(len(hits)) * 1e-4
    srv.replay(t, [g.serve_request(300 + i, _event_parts(g, h)) for i, h in enumerate(hits)])
    srv.drain(timeout_s=60)
    st = srv.stats()
    assert st["completed"] == len(hits) == st["submitted"]
    assert st["peak_pool_bytes"] <= budget + (256 << 10)
    # 24 events, two held at a time for 50 ms each: the last waits >= ~0.5 s
    assert st["admit_wait_max_us"] > 3e5
    assert st["admit_wait_p50_us"] <= st["admit_wait_p99_us"] <= st["admit_wait_max_us"]
    time.sleep(0.1)
    srv.set_release_delay(0.0)
    # the held outputs went back to the budget: a 6.4 MB request fits again
    srv.reset_stats()
    srv.submit(g.serve_request(999, _event_parts(g, 400_000)))
    srv.drain(timeout_s=30)
    assert srv.stats()["completed"] == 1
    srv.close()
