"""Serving (continuous batching, ba_submit / ba_poll): a cluster's result is
the same alone and in the mix.

Two flights are cut into sliding windows (the last 25 % of a window reused
by the next, the first half of that overlap fixed, warm start on the device
from the previous window).  Each flight is solved once window by window with
ba_run, and once through the serving scheduler with both flights' windows in
flight at the same time.  Every window's final state must agree bit for bit.
"""
import time

import ctypes

import numpy as np
import pytest

import oracle as O
import scenegen as sg
from helpers import compare_steps

pytestmark = pytest.mark.gpu

ITERS = 6


def _flight(seed, pts_per_cam=120):
    fl = sg.flight(seed, n_strips=2, per_strip=12, pts_per_cam=pts_per_cam)
    plan = sg.window_plan(seed, fl["n_cams"], m_lo=8, m_hi=12)
    wins = [sg.window_cluster(fl, s, e, nf) for (s, e, nf) in plan]
    return wins


def _create(ctx, wins, w, prev_id):
    c, cams, pts = wins[w]
    if w == 0:
        return ctx.create_cluster(c)
    _, pc, pp = wins[w - 1]
    cm, pm = sg.warm_maps(pc, pp, cams, pts)
    return ctx.create_cluster(c, warm_from=prev_id, warm_cam_map=cm, warm_pt_map=pm)


@pytest.mark.parametrize("precision,pts_per_cam", [("mixed", 120), ("fp64", 120), ("mixed", 800), ("fp64", 800)])
def test_serving_results_equal_alone(precision, pts_per_cam):
    """At 800 points per image the last windows hold points seen only by
    their fixed images, whole chunks of them (chunks with nothing to reduce)."""
    import paper_2511_06152_gb300 as ba
    prec = ba.BA_MIXED if precision == "mixed" else ba.BA_FP64
    flights = [_flight(9101, pts_per_cam), _flight(9102, pts_per_cam)]
    assert all(len(w) >= 2 for w in flights)

    alone = []
    with ba.Context(precision=prec) as ctx:
        for wins in flights:
            prev, states = None, []
            for w in range(len(wins)):
                cid = _create(ctx, wins, w, prev)
                ctx.run(cid, ITERS, trace=False)
                states.append(ctx.get_state(cid))
                prev = cid
            alone.append(states)

    mixed = [[None] * len(w) for w in flights]
    with ba.Context(precision=prec, n_slots=8) as ctx:
        nxt = [0, 0]
        prev = [None, None]
        tickets = {}
        deadline = time.time() + 120
        while any(nxt[f] < len(flights[f]) for f in range(2)) or tickets:
            assert time.time() < deadline, "serving did not finish"
            for f in range(2):
                if nxt[f] < len(flights[f]) and not any(v[0] == f for v in tickets.values()):
                    cid = _create(ctx, flights[f], nxt[f], prev[f])
                    tickets[ctx.submit(cid, ITERS)] = (f, nxt[f], cid)
            for t in list(tickets):
                r = ctx.poll(t)
                if r is None:
                    continue
                f, w, cid = tickets.pop(t)
                assert r["status"] == 0 and r["iters"] == ITERS
                mixed[f][w] = ctx.get_state(cid)
                prev[f] = cid
                nxt[f] += 1
            time.sleep(0.001)

    for f in range(2):
        for w in range(len(flights[f])):
            for a, b in zip(alone[f][w], mixed[f][w]):
                assert np.array_equal(a, b), (f, w)


def test_serving_rejects_double_submit_and_reports_latency():
    import paper_2511_06152_gb300 as ba
    wins = _flight(9103)
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        cid = _create(ctx, wins, 0, None)
        t = ctx.submit(cid, 1000)  # long enough to still be running at the second submit
        try:
            t2 = ctx.submit(cid, 3)
        except ba.BAError:
            t2 = None
        assert t2 is None, ("second submit accepted", ctx.poll(t), ctx.L.ba_last_error(ctx.h))
        r = None
        for _ in range(10000):
            r = ctx.poll(t)
            if r is not None:
                break
            time.sleep(0.001)
        assert r is not None and r["iters"] == 1000 and r["latency_ms"] > 0
        with pytest.raises(ba.BAError):
            ctx.poll(t)  # a ticket is consumed by the poll that returns it


def test_serving_ftol_stops_at_the_first_small_accepted_step():
    """ba_solve_opts.ftol: the ticket ends after the first accepted step, other
    than the first iteration, whose decrease F_before - F_after is at most
    ftol * F_before; the served state equals ba_run for that many iterations
    on the same cluster, bit for bit."""
    import paper_2511_06152_gb300 as ba
    wins = _flight(9104)
    ftol, cap = 1e-3, 100
    with ba.Context(precision=ba.BA_MIXED, n_slots=4) as ctx:
        c0 = _create(ctx, wins, 0, None)
        t = ctx.submit(c0, cap, ftol=ftol)
        r = None
        for _ in range(20000):
            r = ctx.poll(t)
            if r is not None:
                break
            time.sleep(0.001)
        assert r is not None and r["status"] == 0
        assert 2 <= r["iters"] < cap
        served = ctx.get_state(c0)
        c1 = _create(ctx, wins, 0, None)
        tr = ctx.run(c1, r["iters"])
        for a, b in zip(served, ctx.get_state(c1)):
            assert np.array_equal(a, b)
        small = [i for i in range(1, len(tr))
                 if tr[i]["accepted"] and tr[i]["F_before"] - tr[i]["F_after"] <= ftol * tr[i]["F_before"]]
        assert small and small[0] == r["iters"] - 1
        with pytest.raises(ba.BAError):
            ctx.submit(c1, 5, ftol=-1.0)
        with pytest.raises(ba.BAError):
            ctx.submit(c1, 5, ftol=float("nan"))


def test_warm_start_after_create_equals_warm_create():
    """ba_warm_start on an existing cluster gives the same state and result as
    creating the cluster with warm_from."""
    import paper_2511_06152_gb300 as ba
    wins = _flight(9104)
    (c0, _, _), (c1, cams1, pts1) = wins[0], wins[1]
    cm, pm = sg.warm_maps(wins[0][1], wins[0][2], cams1, pts1)
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        a0 = ctx.create_cluster(c0)
        ctx.run(a0, ITERS, trace=False)
        a = ctx.create_cluster(c1, warm_from=a0, warm_cam_map=cm, warm_pt_map=pm)
        b = ctx.create_cluster(c1)
        ctx.warm_start(b, a0, cm, pm)
        for u, v in zip(ctx.get_state(a), ctx.get_state(b)):
            assert np.array_equal(u, v)
        ta, tb = ctx.run(a, ITERS), ctx.run(b, ITERS)
        assert ta == tb
        for u, v in zip(ctx.get_state(a), ctx.get_state(b)):
            assert np.array_equal(u, v)


def test_creation_in_threads_while_serving_equals_alone():
    """Windows are created on worker threads while other windows are being
    solved (creation uploads on its own stream, the scheduler's rounds run
    without the API lock); warm start and submit follow each flight's
    previous window.  Every window's final state equals the one of the same
    sequence run alone."""
    from concurrent.futures import ThreadPoolExecutor
    import paper_2511_06152_gb300 as ba
    flights = [_flight(9111 + f) for f in range(4)]

    def maps(f, w):
        _, pc, pp = flights[f][w - 1]
        _, cams, pts = flights[f][w]
        return sg.warm_maps(pc, pp, cams, pts)

    alone = []
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        for f, wins in enumerate(flights):
            prev, states = None, []
            for w in range(len(wins)):
                cid = ctx.create_cluster(wins[w][0])
                if w:
                    ctx.warm_start(cid, prev, *maps(f, w))
                ctx.run(cid, ITERS, trace=False)
                states.append(ctx.get_state(cid))
                prev = cid
            alone.append(states)

    got = [[None] * len(w) for w in flights]
    with ba.Context(precision=ba.BA_MIXED, n_slots=8) as ctx, ThreadPoolExecutor(4) as ex:
        futs = [[ex.submit(ctx.create_cluster, wins[w][0]) for w in range(len(wins))] for wins in flights]
        nxt, prev, live = [0] * len(flights), [None] * len(flights), {}
        deadline = time.time() + 120
        while any(nxt[f] < len(flights[f]) for f in range(len(flights))) or live:
            assert time.time() < deadline, "serving did not finish"
            for f in range(len(flights)):
                w = nxt[f]
                if f in live or w >= len(flights[f]) or not futs[f][w].done():
                    continue
                cid = futs[f][w].result()
                if w:
                    ctx.warm_start(cid, prev[f], *maps(f, w))
                live[f] = (w, cid, ctx.submit(cid, ITERS))
            for f in list(live):
                w, cid, t = live[f]
                r = ctx.poll(t)
                if r is None:
                    continue
                assert r["status"] == 0 and r["iters"] == ITERS
                del live[f]
                got[f][w] = ctx.get_state(cid)
                if prev[f] is not None:
                    ctx.destroy_cluster(prev[f])
                prev[f] = cid
                nxt[f] += 1
            time.sleep(0.0005)
    for f in range(len(flights)):
        for w in range(len(flights[f])):
            for a, b in zip(alone[f][w], got[f][w]):
                assert np.array_equal(a, b), (f, w)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_transition_matches_oracle(precision):
    """Eq. 8 on the device equals the oracle's weighted pose average for every
    free overlap image; every other image keeps its pose."""
    import oracle as O
    import paper_2511_06152_gb300 as ba
    wins = _flight(9121)
    (c0, cams0, pts0), (c1, cams1, pts1) = wins[0], wins[1]
    cm, pm = sg.warm_maps(cams0, pts0, cams1, pts1)
    with ba.Context(precision=ba.BA_MIXED if precision == "mixed" else ba.BA_FP64) as ctx:
        a = ctx.create_cluster(c0)
        ctx.run(a, ITERS, trace=False)
        b = ctx.create_cluster(c1, warm_from=a, warm_cam_map=cm, warm_pt_map=pm)
        ctx.run(b, ITERS, trace=False)
        Ra, Ta, _ = ctx.get_state(a)
        Rb, Tb, _ = ctx.get_state(b)
        ctx.transition(b, a, cm)
        R2, T2, _ = ctx.get_state(b)
    wa = np.bincount(c0["obs_cam"], minlength=c0["n_cams"])
    wb = np.bincount(c1["obs_cam"], minlength=c1["n_cams"])
    blended = 0
    for k in range(c1["n_cams"]):
        m = cm[k]
        if m < 0 or c1["fixed"][k]:
            assert np.array_equal(R2[k], Rb[k]) and np.array_equal(T2[k], Tb[k])
            continue
        R, T = O.transition(Ra[m], Ta[m], float(wa[m]), Rb[k], Tb[k], float(wb[k]))
        np.testing.assert_allclose(R2[k].reshape(3, 3), R, atol=1e-13)
        np.testing.assert_allclose(T2[k], T, rtol=0, atol=1e-9)
        blended += 1
    assert blended >= 1


def test_creation_during_batch_solve_equals_sequential():
    """A batch is solved on one thread while other clusters are created on
    worker threads (the batch's device run holds no lock); both groups end in
    the states of the same work done one call after another, and the batch's
    clusters are in service until the solve returns."""
    from concurrent.futures import ThreadPoolExecutor
    import paper_2511_06152_gb300 as ba
    group_a = [sg.tiny_cluster(7100 + i, 2, 8, 1500) for i in range(6)]
    group_b = [sg.tiny_cluster(7200 + i, 2, 7, 1200) for i in range(6)]
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        ida = [ctx.create_cluster(s) for s in group_a]
        ctx.solve_batch(ida, 8)
        ref_a = [ctx.get_state(c) for c in ida]
        idb = [ctx.create_cluster(s) for s in group_b]
        ctx.solve_batch(idb, 8)
        ref_b = [ctx.get_state(c) for c in idb]
    with ba.Context(precision=ba.BA_MIXED) as ctx, ThreadPoolExecutor(4) as ex:
        ida = [ctx.create_cluster(s) for s in group_a]
        solving = ex.submit(ctx.solve_batch, ida, 8)
        idb = list(ex.map(ctx.create_cluster, group_b))
        res = solving.result()
        assert all(r["status"] == 0 for r in res)
        ctx.solve_batch(idb, 8)
        for cid, ref in zip(ida, ref_a):
            for x, y in zip(ctx.get_state(cid), ref):
                assert np.array_equal(x, y)
        for cid, ref in zip(idb, ref_b):
            for x, y in zip(ctx.get_state(cid), ref):
                assert np.array_equal(x, y)


def test_get_state_batch_equals_get_state():
    """One batched read-back returns, cluster by cluster, exactly what
    get_state returns (R, T of the current buffer, X in the caller's order)."""
    import paper_2511_06152_gb300 as ba
    scenes = [sg.tiny_cluster(7300 + i, 2, 6 + i, 900 + 100 * i) for i in range(5)]
    for prec in (ba.BA_MIXED, ba.BA_FP64):
        with ba.Context(precision=prec) as ctx:
            ids = [ctx.create_cluster(s) for s in scenes]
            ctx.solve_batch(ids[:3], 4)  # some clusters moved, some still at their initial state
            got = ctx.get_state_batch(ids)
            for cid, (R, T, X) in zip(ids, got):
                R1, T1, X1 = ctx.get_state(cid)
                assert np.array_equal(R, R1) and np.array_equal(T, T1) and np.array_equal(X, X1)


def test_get_state_batch_in_groups_equals_get_state():
    """Three clusters of 500,000 points (36 MB of state, more than one 32 MiB
    group of the batched read-back) come back exactly as get_state returns
    them."""
    import paper_2511_06152_gb300 as ba
    scenes = [sg.tiny_cluster(7400 + i, 2, 8, 500_000) for i in range(3)]
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        ids = [ctx.create_cluster(s) for s in scenes]
        ctx.solve_batch(ids, 2)
        got = ctx.get_state_batch(ids)
        for cid, (R, T, X) in zip(ids, got):
            R1, T1, X1 = ctx.get_state(cid)
            assert np.array_equal(R, R1) and np.array_equal(T, T1) and np.array_equal(X, X1)


def test_warm_start_carries_the_damping_and_matches_the_oracle():
    """The next window starts from the previous window's poses, points and
    damping (mu, nu) on the device; the oracle, seeded with the same state
    and damping, takes the same FP64 steps (relative 1e-10).  A reset
    restores the warm-started state and damping."""
    import paper_2511_06152_gb300 as ba
    wins = _flight(9105)
    (c0, cams0, pts0), (c1, cams1, pts1) = wins[0], wins[1]
    cm, pm = sg.warm_maps(cams0, pts0, cams1, pts1)
    with ba.Context(precision=ba.BA_FP64) as ctx:
        a = ctx.create_cluster(c0)
        tr = ctx.run(a, ITERS)
        mu, nu = tr[-1]["mu"], tr[-1]["nu"]
        assert mu != 1e-4  # the previous window moved its damping
        Ra, Ta, Xa = ctx.get_state(a)
        b = ctx.create_cluster(c1)
        ctx.warm_start(b, a, cm, pm)
        seed = dict(c1, R0=np.array(c1["R0"]).reshape(-1, 9).copy(), T0=np.array(c1["T0"]).copy(),
                    X0=np.array(c1["X0"]).copy())
        seed["R0"][cm >= 0] = Ra[cm[cm >= 0]]
        seed["T0"][cm >= 0] = Ta[cm[cm >= 0]]
        seed["X0"][pm >= 0] = Xa[pm[pm >= 0]]
        for u, v in zip(ctx.get_state(b), (seed["R0"], seed["T0"], seed["X0"])):
            assert np.array_equal(u, v)
        P, S = O.Problem(seed), O.State(seed, mu0=mu)
        S.nu = ctypes.c_double(nu)
        first = ctx.solve_step(b)
        assert first["mu_used"] == mu
        ctx.reset(b)  # the warm-started state and damping come back
        for u, v in zip(ctx.get_state(b), (seed["R0"], seed["T0"], seed["X0"])):
            assert np.array_equal(u, v)
        n = compare_steps(ctx, b, O, P, S, ITERS)
        assert n >= 4, n


def test_hbm_budget_admission_waits_for_memory_and_keeps_results():
    """A context whose device-memory budget holds only some of the windows:
    creating one more returns BA_ERR_BUDGET while the others hold memory,
    succeeds once a finished window has been freed, and every window's result
    equals the one computed without a budget."""
    import paper_2511_06152_gb300 as ba
    wins = _flight(9106)[:3]
    ref = []
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        for c, _, _ in wins:
            cid = ctx.create_cluster(c)
            ctx.run(cid, ITERS, trace=False)
            ref.append(ctx.get_state(cid))
        arena = [ctx.cluster_info(cid)["arena_bytes"] for cid in list(ctx.sizes)]
    with ba.Context(precision=ba.BA_MIXED) as probe:  # memory of the first window and the serving slots
        cid = probe.create_cluster(wins[0][0])
        t = probe.submit(cid, ITERS)
        while probe.poll(t) is None:
            time.sleep(0.001)
        base = probe.memory_in_use()
    # room for windows 0 and 1 (and the slot table) but not for window 2 as
    # well; once window 0 is freed, windows 1 and 2 fit
    budget = base + arena[1] + arena[2] - min(arena[0], arena[2]) // 2
    assert budget < base + arena[1] + arena[2] and budget - base + arena[0] >= arena[1] + arena[2]
    with ba.Context(precision=ba.BA_MIXED, hbm_budget_bytes=budget) as ctx:
        c0 = ctx.create_cluster(wins[0][0])
        t0 = ctx.submit(c0, ITERS)
        c1 = ctx.create_cluster(wins[1][0])
        with pytest.raises(ba.BAError) as ei:
            ctx.create_cluster(wins[2][0])
        assert ei.value.status == ba.BA_ERR_BUDGET
        t1 = ctx.submit(c1, ITERS)
        got = {}
        for cid, t in ((c0, t0), (c1, t1)):
            r = None
            while r is None:
                r = ctx.poll(t)
                time.sleep(0.001)
            assert r["status"] == 0 and r["iters"] == ITERS
            got[cid] = ctx.get_state(cid)
        ctx.destroy_cluster(c0)  # a completion frees memory: the waiting window is admitted
        c2 = ctx.create_cluster(wins[2][0])
        t2 = ctx.submit(c2, ITERS)
        r = None
        while r is None:
            r = ctx.poll(t2)
            time.sleep(0.001)
        got[c2] = ctx.get_state(c2)
        for cid, rf in zip((c0, c1, c2), ref):
            for u, v in zip(got[cid], rf):
                assert np.array_equal(u, v)


def test_streamed_batches_equal_sequential():
    """Batches streamed as a caller feeding windows continuously runs them:
    batch k+1 is created on worker threads while batch k is solved and read
    back on another thread (neither holds the context's lock while the device
    works); every state equals that of the same calls made one after another."""
    from concurrent.futures import ThreadPoolExecutor
    import paper_2511_06152_gb300 as ba
    groups = [[sg.tiny_cluster(7400 + 10 * g + i, 2, 6 + i % 3, 1000 + 200 * i) for i in range(5)] for g in range(3)]
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        ref = []
        for grp in groups:
            ids = [ctx.create_cluster(s) for s in grp]
            ctx.solve_batch(ids, 6)
            ref.append(ctx.get_state_batch(ids))
    with ba.Context(precision=ba.BA_MIXED) as ctx, ThreadPoolExecutor(4) as pool, ThreadPoolExecutor(1) as solver:
        def solve_read(ids):
            ctx.solve_batch(ids, 6)
            return ctx.get_state_batch(ids)
        cur = list(pool.map(ctx.create_cluster, groups[0]))
        got = []
        for k in range(len(groups)):
            fut = solver.submit(solve_read, cur)
            nxt = list(pool.map(ctx.create_cluster, groups[k + 1])) if k + 1 < len(groups) else None
            got.append(fut.result())
            cur = nxt
    for g_ref, g_got in zip(ref, got):
        for a, b in zip(g_ref, g_got):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)


def test_get_state_batch_refuses_a_cluster_in_service():
    """ba_get_state_batch runs without the context's lock and keeps its
    clusters in service meanwhile, so it refuses one that the serving
    scheduler is running (nothing is written) and still reads the others."""
    import paper_2511_06152_gb300 as ba
    sa, sb = sg.tiny_cluster(7501, 2, 8, 2000), sg.tiny_cluster(7502, 2, 6, 800)
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        a, b = ctx.create_cluster(sa), ctx.create_cluster(sb)
        before = ctx.get_state_batch([b])[0]
        t = ctx.submit(a, 400)  # hundreds of rounds: still running when the read comes
        with pytest.raises(ba.BAError) as e:
            ctx.get_state_batch([b, a])
        assert e.value.status == ba.BA_ERR_INVALID
        for x, y in zip(ctx.get_state_batch([b])[0], before):
            assert np.array_equal(x, y)
        while ctx.poll(t) is None:
            time.sleep(0.002)
        R, T, X = ctx.get_state_batch([a])[0]
        assert np.all(np.isfinite(R)) and np.all(np.isfinite(T)) and np.all(np.isfinite(X))
