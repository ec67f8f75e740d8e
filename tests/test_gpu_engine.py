"""Many runs at once: the non-blocking run API (plse_run_issue / plse_run_query),
plse_solve_batch and the plse_server_* request server.  Every job's result must
equal that of plse_solve of the same job alone (and, for small cases, the
oracle's Alg. 2): best grid, score, generations and the summed work counters of
every walk, which pin every trajectory."""
import time

import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plse():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_10453_gb300 import plse as P
    P.load()
    return P


def grids():
    return [inputs.tiny_n10(), inputs.random_insertion(11, 0.7, 7), inputs.cyclic_delete(12, 0.5, 3)[0],
            inputs.random_insertion(16, 0.75, 8), inputs.random_insertion(20, 0.65, 9),
            inputs.random_insertion(14, 0.8, 10), inputs.random_insertion(25, 0.5, 11)]


JOBS = [(64, 20, 2000, 1), (24, 8, 150, 3), (32, 10, 200, 5), (40, 8, 150, 4), (48, 6, 150, 6),
        (56, 8, 150, 7), (96, 5, 300, 2)]


def same(a, b):
    assert a["score"] == b["score"]
    assert np.array_equal(a["best_grid"], b["best_grid"])
    assert a["generations"] == b["generations"]
    assert a["walks"] == b["walks"]


def alone(plse, grid, job, params=None):
    G = plse.Instance(grid)
    if params is not None:
        G.set_params(params)
    r = G.solve(*job, with_stats=True)
    G.close()
    return r


def test_issue_query_loop_equals_blocking_run(plse):
    for grid, job in [(grids()[2], (32, 10, 200, 5)), (grids()[3], (40, 8, 150, 4))]:
        ref = alone(plse, grid, job)
        G = plse.Instance(grid)
        pop, gens, iters, seed = job
        G.run_begin(pop, gens, iters, seed)
        seen_inflight = 0
        while True:
            G.run_issue()
            done, g, inflight = G.run_query()
            seen_inflight = max(seen_inflight, inflight)
            if done:
                break
        res = G.run_result(trace=True)
        same(res, ref)
        assert seen_inflight <= 2
        # resumable blocking steps give the same trace
        G.run_begin(pop, gens, iters, seed)
        G.run_step(3)
        G.run_step(gens)
        res2 = G.run_result(trace=True)
        same(res2, ref)
        assert np.array_equal(res["trace"], res2["trace"])
        G.close()


def test_concurrent_runs_on_streams_equal_runs_alone(plse):
    """Several runs driven by plse_run_issue on their own streams at once give
    each run's result alone; the populations are large enough for several
    Alg. 4 chunks, whose dataflow passes then share the GPU."""
    import torch
    gs = grids()[:3]
    jobs = [(300, 4, 150, 7), (260, 3, 120, 8), (200, 4, 100, 9)]
    refs = [alone(plse, g, j) for g, j in zip(gs, jobs)]
    for _ in range(2):
        insts, streams = [], []
        for g, (pop, gens, iters, seed) in zip(gs, jobs):
            G = plse.Instance(g)
            s = torch.cuda.Stream()
            G.run_begin(pop, gens, iters, seed, stream=s)
            insts.append(G)
            streams.append(s)
        while True:
            done = True
            for G, s in zip(insts, streams):
                G.run_issue(stream=s)
                done = G.run_query()[0] and done
            if done:
                break
        for G, s, ref in zip(insts, streams, refs):
            same(G.run_result(stream=s), ref)
            G.close()


def test_run_timeline_gives_each_generations_local_search_interval(plse):
    import torch
    ref = torch.cuda.Event(enable_timing=True)
    ref.record()
    torch.cuda.synchronize()
    G = plse.Instance(grids()[4])
    G.set_params(plse.default_params(stop_at_bound=0))
    G.run_begin(48, 4, 150, 3)
    G.run_step(3)
    tl = G.run_timeline(ref, 0, 3)
    res = G.run_result()
    assert tl.shape == (3, 2)
    assert np.all(tl[:, 0] > 0) and np.all(tl[:, 1] > tl[:, 0])
    assert np.all(tl[1:, 0] >= tl[:-1, 1])                 # one stream: one after another
    assert abs(float((tl[:, 1] - tl[:, 0]).sum()) - res["ms_local_search"]) < 1e-2
    assert np.array_equal(G.run_timeline(ref, 1, 2), tl[1:])
    with pytest.raises(plse.PlseError) as e:
        G.run_timeline(ref, 2, 2)                           # generation 3 has not run
    assert e.value.code == plse.PLSE_EINVAL
    G.close()


def test_batch_matches_solve_alone_and_oracle(plse, oracle_mod):
    gs = grids()
    insts = [plse.Instance(g) for g in gs]
    out, rc = plse.solve_batch(insts, JOBS, max_inflight=3)
    assert rc == plse.PLSE_OK
    for g, job, r in zip(gs, JOBS, out):
        assert r["status"] == 0
        same(r, alone(plse, g, job))
    # the first job against the oracle's Alg. 2 directly
    ref = oracle_mod.Instance(gs[0]).solve(*JOBS[0])
    assert out[0]["score"] == ref["score"] and np.array_equal(out[0]["best_grid"], ref["best_grid"])
    assert out[0]["walks"] == ref["stats"]
    for G in insts:
        G.close()


def test_batch_repeated_handle_and_inflight_widths(plse):
    gs = grids()
    G0, G1 = plse.Instance(gs[4]), plse.Instance(gs[1])
    jobs = [(48, 6, 150, 6), (48, 6, 150, 9), (24, 8, 150, 3), (48, 4, 100, 11)]
    refs = [alone(plse, gs[4], jobs[0]), alone(plse, gs[4], jobs[1]), alone(plse, gs[1], jobs[2]),
            alone(plse, gs[4], jobs[3])]
    for width in (1, 2, 4):
        out, rc = plse.solve_batch([G0, G0, G1, G0], jobs, max_inflight=width)
        assert rc == 0
        for r, ref in zip(out, refs):
            same(r, ref)
    G0.close()
    G1.close()


def test_batch_reports_per_job_errors(plse):
    gs = grids()
    insts = [plse.Instance(gs[0]), plse.Instance(gs[1])]
    out, rc = plse.solve_batch(insts, [(64, 3, 100, 1), (1, 3, 100, 1)], max_inflight=2)   # pop 1: invalid
    assert rc == plse.PLSE_EINVAL
    assert out[0]["status"] == 0 and out[1]["status"] == plse.PLSE_EINVAL
    same(out[0], alone(plse, gs[0], (64, 3, 100, 1)))


def test_server_results_match_solve_alone(plse):
    gs = grids()
    srv = plse.Server(max_inflight=3, max_queue=64)
    tickets = [srv.submit(g, *job) for g, job in zip(gs, JOBS)]
    outs = [srv.poll(t, wait_ms=-1) for t in tickets]
    for g, job, r in zip(gs, JOBS, outs):
        assert r["status"] == 0
        same(r, alone(plse, g, job))
        assert r["ms_wall"] >= r["ms_queue"] >= 0
    with pytest.raises(plse.PlseError):
        srv.poll(tickets[0])                      # released once polled
    # parameters travel with the request
    prm = plse.default_params(stop_at_bound=0, crossover=plse.XOVER_UX)
    t = srv.submit(gs[1], 24, 4, 150, 3, params=prm)
    same(srv.poll(t, wait_ms=-1), alone(plse, gs[1], (24, 4, 150, 3), params=prm))
    srv.close()


def test_server_admission_cancel_and_invalid_grid(plse):
    srv = plse.Server(max_inflight=1, max_queue=0)
    with pytest.raises(plse.PlseError) as e:
        srv.submit(grids()[0], 16, 2, 50, 1)
    assert e.value.code == plse.PLSE_EBUSY
    srv.close()

    srv = plse.Server(max_inflight=1, max_queue=2)
    long_grid = inputs.random_insertion(30, 0.5, 12)
    no_stop = plse.default_params(stop_at_bound=0)
    ta = srv.submit(long_grid, 256, 3000, 4000, 1, params=no_stop)   # runs for many seconds
    t0 = time.time()
    while srv.pending()[0] != 0 and time.time() - t0 < 30:
        time.sleep(0.01)
    assert srv.pending()[0] == 0                # A admitted
    tb = srv.submit(grids()[1], 24, 4, 150, 3)
    tc = srv.submit(grids()[2], 32, 4, 200, 5)
    with pytest.raises(plse.PlseError) as e:
        srv.submit(grids()[3], 16, 2, 50, 1)      # queue full
    assert e.value.code == plse.PLSE_EBUSY
    srv.cancel(tb)
    srv.cancel(ta)
    ra = srv.poll(ta, wait_ms=-1)
    assert ra["status"] == plse.PLSE_ECANCELLED and ra["generations"] < 3000
    assert srv.poll(tb, wait_ms=-1)["status"] == plse.PLSE_ECANCELLED
    rc = srv.poll(tc, wait_ms=-1)
    assert rc["status"] == 0
    same(rc, alone(plse, grids()[2], (32, 4, 200, 5)))
    bad = np.zeros((5, 5), dtype=np.int8)
    bad[0, 0] = bad[0, 1] = 3                     # symbol twice in a row
    tbad = srv.submit(bad, 16, 2, 50, 1)
    assert srv.poll(tbad, wait_ms=-1)["status"] == plse.PLSE_EINVAL
    # destroy with work still queued and running returns
    srv.submit(long_grid, 256, 3000, 4000, 2, params=no_stop)
    srv.submit(long_grid, 256, 3000, 4000, 3, params=no_stop)
    srv.close()


def test_server_mixed_sizes_against_solve_alone(plse):
    """Requests of the serving mix (n from 10 to 96, populations 32 to 512) admitted
    while others run: each handle is created and launched on a non-blocking
    stream at once, so the instance upload must be complete before its kernels."""
    gs = inputs.serve_mix(24)
    srv = plse.Server(max_inflight=16, max_queue=64)
    jobs = [(inputs.serve_pop(g), 2, 2 * int((g == 0).sum()), 1) for g in gs]
    tickets = [srv.submit(g, *job) for g, job in zip(gs, jobs)]
    outs = [srv.poll(t, wait_ms=-1) for t in tickets]
    srv.close()
    for g, job, r in zip(gs, jobs, outs):
        assert r["status"] == 0, r["detail"]
        same(r, alone(plse, g, job))


def test_server_admits_by_device_memory(plse):
    """A budget of 1.5 requests' footprint: requests wait for memory, never two
    run at once, every result equals plse_solve alone, and a request larger than
    the budget completes with PLSE_ENOMEM."""
    gs = [inputs.random_insertion(30, 0.5, 100 + k) for k in range(5)]
    jobs = [(128, 3, 200, 1 + k) for k in range(5)]
    probe = plse.Server(max_inflight=4, max_queue=16)
    one = probe.poll(probe.submit(gs[0], *jobs[0]), wait_ms=-1)
    probe.close()
    assert one["status"] == 0 and one["mem_bytes"] > 128 * 450
    budget = one["mem_bytes"] * 3 // 2
    srv = plse.Server(max_inflight=4, max_queue=16, mem_budget=budget)
    tickets = [srv.submit(g, *job) for g, job in zip(gs, jobs)]
    big = srv.submit(gs[0], 512, 3, 200, 9)        # about 4x the footprint: never fits
    outs = [srv.poll(t, wait_ms=-1) for t in tickets]
    rbig = srv.poll(big, wait_ms=-1)
    mem = srv.memory()
    srv.close()
    assert rbig["status"] == plse.PLSE_ENOMEM
    assert mem["budget"] == budget and mem["in_use"] == 0
    assert one["mem_bytes"] <= mem["peak"] <= budget
    assert mem["peak_running"] == 1 and mem["waited_for_memory"] >= 1
    for g, job, r in zip(gs, jobs, outs):
        assert r["status"] == 0, r["detail"]
        assert r["mem_bytes"] == one["mem_bytes"]
        same(r, alone(plse, g, job))


def test_batch_one_launch_per_generation_and_class(plse, oracle_mod):
    """Lockstep mode: the generations of all runs share one persistent
    multi-instance local-search launch per colour-word class
    (here n = 10..25, 40, 70: three classes, uneven populations and stops).
    Every result equals plse_solve alone, and one equals the oracle's Alg. 2."""
    gs = grids() + [inputs.random_insertion(40, 0.6, 21), inputs.cyclic_delete(45, 0.7, 22)[0],
                    inputs.random_insertion(70, 0.7, 23)]
    jobs = JOBS + [(80, 3, 400, 8), (50, 4, 300, 9), (70, 2, 500, 10)]
    insts = [plse.Instance(g) for g in gs]
    out, rc = plse.solve_batch(insts, jobs, lockstep=True)
    assert rc == plse.PLSE_OK
    for g, job, r in zip(gs, jobs, out):
        assert r["status"] == 0, r["detail"]
        same(r, alone(plse, g, job))
    ref = oracle_mod.Instance(gs[2]).solve(*jobs[2])
    assert out[2]["score"] == ref["score"] and np.array_equal(out[2]["best_grid"], ref["best_grid"])
    assert out[2]["walks"] == ref["stats"]
    for G in insts:
        G.close()


def test_autotune_picks_knobs_without_changing_results(plse, oracle_mod):
    import torch
    from _gpu import dev, empty, host
    grid = inputs.random_insertion(40, 0.5, 31)
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    P = I.init_population(200, 4)
    flags = plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR

    def run():
        out = empty(P.shape, torch.uint8)
        st = empty((P.shape[0], 7), torch.int64)
        G.local_search(dev(P), out, P.shape[0], 3, 2, 600, 9, flags, None, None, st)
        G.sync()
        return host(out), host(st)

    before = run()
    lanes, walks, place, rate = G.autotune(200, probe_iters=100)
    assert lanes in (16, 32, 64, 128) and place in (0, 1, 2) and rate > 0
    assert G.autotune(200, probe_iters=100)[:3] == (lanes, walks, place)     # cached
    after = run()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    So, _, _ = I.tabu_walk(P[0], 3, 2, 1, 600, 9)
    So, _, _ = I.tabu_walk(So, 3, 2, 2, 2 * I.nv, 9)
    So, _ = I.repair(So)
    assert np.array_equal(after[0][0], So)
    G.close()


def test_batch_multistart_both_modes(plse, oracle_mod):
    """A multi-start (one instance, several seeds) in concurrent and in lockstep
    mode; each run equals plse_solve alone."""
    g = inputs.random_insertion(40, 0.6, 77)
    jobs = [(96, 4, 300, 1 + k) for k in range(6)]
    insts = [plse.Instance(g) for _ in jobs]
    out, rc = plse.solve_batch(insts, jobs)
    assert rc == plse.PLSE_OK
    for job, r in zip(jobs, out):
        same(r, alone(plse, g, job))
    out, rc = plse.solve_batch(insts, jobs, lockstep=True)
    assert rc == plse.PLSE_OK
    for job, r in zip(jobs, out):
        same(r, alone(plse, g, job))
    for G in insts:
        G.close()
