"""Continuous-batching server (hj_server_*) on the GPU.

Each result must be the same solved alone and solved in a mix with other
requests.  Warm starts from resident priors must reach the cold fixed
point.  The HBM budget must bound memory use.  Host-side failures
(malformed, oversized, cancelled or capped requests) must come back as
statuses, never as GPU faults.
"""
import threading
import time

import numpy as np
import pytest

from paper_2101_05916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
REL = 1e-4


@pytest.fixture(scope="module")
def hj():
    import torch
    assert torch.cuda.is_available()
    from paper_2101_05916_gb300 import build, hj as hjmod
    build.build()
    hjmod.lib()
    return hjmod


def specs_mix():
    return [(wl.quad_z(61, 0.5), 2, 0.0), (wl.quad_x4(15, 0.5), 5, 0.5),
            (wl.quad_z(83, 1.1), 5, 0.0), (wl.quad_x4(13, 0.8, 3.5, "y"), 5, 0.5),
            (wl.quad_z(101, 0.3, (0.6, 2.4)), 2, 0.0)]


def run(hj, s, spec, scheme, band, mode=0, key=0, **kw):
    req = hj.make_request(spec, mode, key, scheme=scheme, band=band, max_steps=20000, **kw)
    return hj.hj_server_submit(s, req)


def fetch(hj, s, t, spec):
    rc, st = hj.hj_server_wait(s, t, 120000.0)
    out = np.empty(spec.npts, dtype=np.float32)
    if rc == hj.HJ_OK:
        hj.hj_server_get_value(s, t, out)
    hj.hj_server_release(s, t)
    return rc, st, out.reshape(spec.n)


def test_each_result_same_alone_and_in_the_mix(hj):
    mix = specs_mix()
    s = hj.hj_server_create(8 << 30, 16)
    alone = []
    for spec, sc, band in mix:
        t = run(hj, s, spec, sc, band)
        alone.append(fetch(hj, s, t, spec))
    tickets = [run(hj, s, spec, sc, band) for spec, sc, band in mix]
    together = [fetch(hj, s, t, spec) for t, (spec, _, _) in zip(tickets, mix)]
    stats = hj.hj_server_get_stats(s)
    hj.hj_server_destroy(s)
    for (rc1, st1, W1), (rc2, st2, W2) in zip(alone, together):
        assert rc1 == hj.HJ_OK and rc2 == hj.HJ_OK
        assert st1["steps"] == st2["steps"]
        assert np.abs(W1 - W2).max() <= REL * np.abs(W1).max()
    assert stats["completed"] == 2 * len(mix)


def test_served_result_matches_single_grid_solve(hj):
    spec = wl.quad_z(81, 0.7)
    g = hj.Grid.from_spec(spec)
    st = g.solve(hj.HJ_COLD, scheme=2)
    ref = g.value()
    g.close()
    s = hj.hj_server_create(1 << 30, 4)
    rc, st2, W = fetch(hj, s, run(hj, s, spec, 2, 0.0), spec)
    hj.hj_server_destroy(s)
    assert rc == hj.HJ_OK and st2["steps"] == st["steps"]
    assert np.array_equal(W, ref)


def test_warm_start_from_resident_prior_is_exact(hj):
    """Increasing wind bounds on one key: each update warm-starts from the
    previous fixed point (it dominates) and lands on the cold fixed point."""
    s = hj.hj_server_create(4 << 30, 8)
    key = 77
    results = []
    for b in (0.0, 0.5, 1.0):
        spec = wl.quad_z(101, b)
        rc, st, W = fetch(hj, s, run(hj, s, spec, 2, 0.0, hj.HJ_WARM, key, tol=1e-6), spec)
        assert rc == hj.HJ_OK
        results.append((spec, st, W))
    stats = hj.hj_server_get_stats(s)
    # a shrunk wind bound does not dominate: must fall back to a cold start
    spec = wl.quad_z(101, 0.2)
    rc, st, W = fetch(hj, s, run(hj, s, spec, 2, 0.0, hj.HJ_WARM, key, tol=1e-6), spec)
    stats2 = hj.hj_server_get_stats(s)
    hj.hj_server_destroy(s)
    assert stats["warm_starts"] == 2 and stats["cold_starts"] == 1
    assert stats2["cold_starts"] == 2
    for spec, st, W in results[1:]:
        g = hj.Grid.from_spec(spec)
        g.solve(hj.HJ_COLD, scheme=2, tol=1e-6)
        Wc = g.value()
        g.close()
        assert np.abs(W - Wc).max() <= REL * np.abs(Wc).max()


def test_budget_bounds_memory_and_queues(hj):
    spec = wl.quad_x4(21, 0.5)
    one = 4 * 21 ** 4 * 4 + (1 << 16)
    s = hj.hj_server_create(int(1.5 * one), 8)
    tickets = [run(hj, s, spec, 5, 0.5, fixed_steps=20) for _ in range(4)]
    outs = [fetch(hj, s, t, spec) for t in tickets]
    stats = hj.hj_server_get_stats(s)
    assert all(rc == hj.HJ_OK for rc, _, _ in outs)
    assert stats["peak_bytes"] <= int(1.5 * one)
    assert stats["completed"] == 4
    big = wl.quad_x4(41, 0.5)
    with pytest.raises(hj.HJError) as e:
        run(hj, s, big, 5, 0.5)
    assert e.value.status == hj.HJ_ERR_OOM
    hj.hj_server_destroy(s)


def test_host_side_failures_come_back_as_statuses(hj):
    s = hj.hj_server_create(2 << 30, 4)
    # malformed: 2-node axis
    bad = wl.dataclasses.replace(wl.quad_z(11, 0.5), n=(2, 11))
    with pytest.raises(hj.HJError) as e:
        run(hj, s, bad, 2, 0.0)
    assert e.value.status == hj.HJ_ERR_ARG
    # wrong model dimension: accepted at submit, fails at admission
    wrong = wl.dataclasses.replace(wl.quad_x4(5, 0.5), model=wl.QUAD_Z)
    rc, _, _ = fetch(hj, s, run(hj, s, wrong, 2, 0.0), wrong)
    assert rc == hj.HJ_ERR_ARG
    # never converges within its cap
    spec = wl.quad_z(61, 0.5)
    req = hj.make_request(spec, 0, 0, scheme=2, tol=1e-12, max_steps=50)
    rc, st, W = fetch(hj, s, hj.hj_server_submit(s, req), spec)
    assert rc == hj.HJ_ERR_NOT_CONVERGED and st["steps"] == 50
    # cancelled while running
    req = hj.make_request(wl.quad_x4(31, 0.5), 0, 0, scheme=5, tol=1e-12, max_steps=10 ** 6)
    t = hj.hj_server_submit(s, req)
    time.sleep(0.3)
    hj.hj_server_cancel(s, t)
    rc, st = hj.hj_server_wait(s, t, 60000.0)
    hj.hj_server_release(s, t)
    assert rc == hj.HJ_ERR_ABORTED
    # the server still works afterwards
    rc, _, _ = fetch(hj, s, run(hj, s, wl.quad_z(41, 0.5), 2, 0.0), wl.quad_z(41, 0.5))
    assert rc == hj.HJ_OK
    hj.hj_server_destroy(s)


def test_concurrent_submitters(hj):
    s = hj.hj_server_create(4 << 30, 32)
    specs = [wl.quad_z(41 + 2 * i, 0.1 * i) for i in range(12)]
    tickets = [None] * len(specs)

    def worker(k):
        for i in range(k, len(specs), 3):
            tickets[i] = run(hj, s, specs[i], 2, 0.0)

    ths = [threading.Thread(target=worker, args=(k,)) for k in range(3)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    rcs = [fetch(hj, s, t, sp)[0] for t, sp in zip(tickets, specs)]
    stats = hj.hj_server_get_stats(s)
    hj.hj_server_destroy(s)
    assert all(rc == hj.HJ_OK for rc in rcs)
    assert stats["completed"] == len(specs)


def test_trace_replay_small(hj):
    from paper_2101_05916_gb300 import serve
    trace = wl.serving_trace(count=12, rate_hz=40.0, n2=(61, 101), n4=(13, 19))
    res = serve.replay_server(trace, budget_bytes=4 << 30, max_active=16)
    assert all(rc == 0 for rc in res["statuses"])
    assert res["server"]["completed"] == 12
    assert res["p99_ms"] >= res["p50_ms"] > 0.0


def test_shortest_first_policy_with_node_cap(hj):
    """With shortest-first admission and a node cap, small requests submitted
    after a large one run beside it and finish first; every result is the
    same as its single-grid solve."""
    s = hj.hj_server_create(8 << 30, 16)
    hj.hj_server_set_policy(s, hj.HJ_ORDER_SHORTEST, 30 ** 4)
    big = wl.quad_x4(31, 0.5)
    small = [wl.quad_z(41 + 4 * i, 0.5) for i in range(6)]
    tb = run(hj, s, big, 5, 0.5, clamp=1, fixed_steps=4000)
    ts = [run(hj, s, sp, 2, 0.0) for sp in small]
    outs = [fetch(hj, s, t, sp) for t, sp in zip(ts, small)]
    rb, stb, _ = fetch(hj, s, tb, big)
    hj.hj_server_destroy(s)
    assert rb == hj.HJ_OK and all(o[0] == hj.HJ_OK for o in outs)
    assert max(o[1]["wall_ms"] for o in outs) < stb["wall_ms"]
    for (rc, st, W), sp in zip(outs, small):
        g = hj.Grid.from_spec(sp)
        g.solve(hj.HJ_COLD, scheme=2, max_steps=20000)
        assert np.array_equal(W, g.value())
        g.close()
    s2 = hj.hj_server_create(1 << 20, 1)
    with pytest.raises(hj.HJError):
        hj.hj_server_set_policy(s2, 7, 0)
    hj.hj_server_destroy(s2)


def test_coarse_initialisation_in_the_server(hj):
    """A request with coarse_n runs coarse solve -> migration -> warm fine
    solve inside the server: bit-identical to doing those three calls by
    hand, and the same safe set as a cold fine solve up to the coarse
    start's conservatism (Sec. III-B/C)."""
    from paper_2101_05916_gb300 import scenarios
    spec = wl.quad_x4(25, 0.7)
    opts = dict(scenarios.X4_OPTS, max_wall_ms=0.0)
    s = hj.hj_server_create(4 << 30, 8)
    req = hj.make_request(spec, hj.HJ_COLD, 0, coarse_n=13, **opts)
    rc, st, W = fetch(hj, s, hj.hj_server_submit(s, req), spec)
    stats = hj.hj_server_get_stats(s)
    hj.hj_server_destroy(s)
    assert rc == hj.HJ_OK and stats["completed"] == 1
    gc, gf = hj.Grid.from_spec(wl.quad_x4(13, 0.7)), hj.Grid.from_spec(spec)
    gc.solve(hj.HJ_COLD, **opts)
    hj.prolong(gc, gf)
    stw = gf.solve(hj.HJ_WARM, **opts)
    Wm = gf.value()
    stc = gf.solve(hj.HJ_COLD, **opts)
    Wc = gf.value()
    gc.close()
    gf.close()
    assert st["steps"] == stw["steps"]
    assert np.array_equal(W, Wm)
    assert np.mean((W >= 0) == (Wc >= 0)) >= 0.99
    with pytest.raises(hj.HJError):
        s2 = hj.hj_server_create(1 << 30, 2)
        try:
            hj.hj_server_submit(s2, hj.make_request(spec, 0, 0, coarse_n=2, **opts))
        finally:
            hj.hj_server_destroy(s2)


def test_monotone_clamp_requests_never_warm_start(hj):
    """Under the monotone clamp a solve's limit depends on its start, so a
    request with it solves cold even when the key's prior dominates; its
    result is its own cold solve."""
    s = hj.hj_server_create(4 << 30, 8)
    key = 55
    for b in (0.2, 0.5):
        spec = wl.quad_z(61, b)
        rc, st, W = fetch(hj, s, run(hj, s, spec, 2, 0.0, hj.HJ_WARM, key, clamp=1, tol=1e-5),
                          spec)
        assert rc == hj.HJ_OK
    stats = hj.hj_server_get_stats(s)
    hj.hj_server_destroy(s)
    assert stats["warm_starts"] == 0 and stats["cold_starts"] == 2
    g = hj.Grid.from_spec(spec)
    g.solve(hj.HJ_COLD, scheme=2, tol=1e-5, clamp=1, max_steps=20000)
    Wc = g.value()
    g.close()
    assert np.abs(W - Wc).max() <= REL * np.abs(Wc).max()


def test_translated_prior_warm_start(hj):
    """With translated starts enabled, a key's resident prior whose
    constraint box, moved along the position axis, equals the new one
    warm-starts the request through hj_translate and reaches the cold fixed
    point; a moved box with a smaller wind bound does not dominate and starts
    cold."""
    s = hj.hj_server_create(4 << 30, 8)
    hj.hj_server_set_translated_starts(s, True)
    key = 91
    first = wl.quad_z(101, 0.5, (0.5, 2.5))
    rc, st0, _ = fetch(hj, s, run(hj, s, first, 2, 0.0, hj.HJ_WARM, key, tol=1e-5), first)
    moved = wl.quad_z(101, 0.6, (0.65, 2.65))
    rc, st1, W = fetch(hj, s, run(hj, s, moved, 2, 0.0, hj.HJ_WARM, key, tol=1e-5), moved)
    stats = hj.hj_server_get_stats(s)
    weaker = wl.quad_z(101, 0.3, (0.4, 2.4))
    rc2, _, _ = fetch(hj, s, run(hj, s, weaker, 2, 0.0, hj.HJ_WARM, key, tol=1e-5), weaker)
    stats2 = hj.hj_server_get_stats(s)
    hj.hj_server_destroy(s)
    assert rc == hj.HJ_OK and rc2 == hj.HJ_OK
    assert stats["translated_starts"] == 1 and stats["warm_starts"] == 1
    assert stats2["translated_starts"] == 1 and stats2["cold_starts"] == 2
    g = hj.Grid.from_spec(moved)
    stc = g.solve(hj.HJ_COLD, scheme=2, tol=1e-5)
    Wc = g.value()
    g.close()
    assert st1["steps"] < stc["steps"]
    assert np.abs(W - Wc).max() <= REL * np.abs(Wc).max()


def test_translated_starts_are_off_by_default(hj):
    """Without hj_server_set_translated_starts a moved-box prior is not used:
    the request solves cold and its result is its own cold solve bit for
    bit; the setting takes only 0 or 1."""
    s = hj.hj_server_create(4 << 30, 8)
    key = 92
    first = wl.quad_z(101, 0.5, (0.5, 2.5))
    fetch(hj, s, run(hj, s, first, 2, 0.0, hj.HJ_WARM, key, tol=1e-5), first)
    moved = wl.quad_z(101, 0.6, (0.65, 2.65))
    rc, st1, W = fetch(hj, s, run(hj, s, moved, 2, 0.0, hj.HJ_WARM, key, tol=1e-5), moved)
    stats = hj.hj_server_get_stats(s)
    with pytest.raises(hj.HJError):
        hj._check(hj.lib().hj_server_set_translated_starts(s, 2))
    hj.hj_server_destroy(s)
    assert rc == hj.HJ_OK
    assert stats["translated_starts"] == 0 and stats["warm_starts"] == 0
    assert stats["cold_starts"] == 2
    g = hj.Grid.from_spec(moved)
    stc = g.solve(hj.HJ_COLD, scheme=2, tol=1e-5)
    Wc = g.value()
    g.close()
    assert st1["steps"] == stc["steps"]
    assert np.array_equal(W, Wc)


def test_two_coarse_levels_and_coarse_scheme(hj):
    """coarse_n -> coarse_n2 -> n inside the server, with cheap gradients
    (ENO2) on the coarse levels: bit-identical to the same chain of calls by
    hand (Sec. III-C)."""
    from paper_2101_05916_gb300 import scenarios
    spec = wl.quad_x4(25, 0.7)
    opts = dict(scenarios.X4_OPTS, max_wall_ms=0.0)
    s = hj.hj_server_create(4 << 30, 8)
    req = hj.make_request(spec, hj.HJ_COLD, 0, coarse_n=9, coarse_n2=13,
                          coarse_scheme=hj.HJ_ENO2, **opts)
    rc, st, W = fetch(hj, s, hj.hj_server_submit(s, req), spec)
    stats = hj.hj_server_get_stats(s)
    assert rc == hj.HJ_OK and stats["completed"] == 1
    assert stats["bytes_in_use"] >= 0
    for bad in (dict(coarse_n=0, coarse_n2=13), dict(coarse_n=13, coarse_n2=9),
                dict(coarse_n=9, coarse_scheme=4)):
        with pytest.raises(hj.HJError):
            hj.hj_server_submit(s, hj.make_request(spec, hj.HJ_COLD, 0, **bad, **opts))
    hj.hj_server_destroy(s)
    coarse = dict(opts, scheme=hj.HJ_ENO2)
    g9, g13, g25 = (hj.Grid.from_spec(wl.quad_x4(n, 0.7)) for n in (9, 13, 25))
    g9.solve(hj.HJ_COLD, **coarse)
    hj.prolong(g9, g13)
    g13.solve(hj.HJ_WARM, **coarse)
    hj.prolong(g13, g25)
    stw = g25.solve(hj.HJ_WARM, **opts)
    Wm = g25.value()
    for g in (g9, g13, g25):
        g.close()
    assert st["steps"] == stw["steps"]
    assert np.array_equal(W, Wm)
