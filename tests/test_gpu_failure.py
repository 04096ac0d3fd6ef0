"""Failure handling on the GPU without a fault: the bounded staging wait.

The mixed-precision linearise+Schur kernel stages each chunk with the copy
engine and waits for it on an mbarrier with a time limit.  With
BA_FLAG_INJECT_COPY_TIMEOUT the kernel waits on a barrier that nothing
completes (1 ms limit) instead, so the expired-wait path runs: the copies it
issued are waited for, the cluster's step status becomes BA_ERR_TIMEOUT, the
step is rejected (mu <- mu nu), the state does not change and the call
returns.  A context without the flag then solves the same cluster normally.
"""
import time

import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ba():
    import paper_2511_06152_gb300 as m
    m.lib()
    return m


def test_expired_copy_wait_rejects_the_step_and_keeps_the_state(ba):
    c = sg.cluster_c1()
    with ba.Context(precision=ba.BA_MIXED, flags=ba.BA_FLAG_INJECT_COPY_TIMEOUT) as ctx:
        cid = ctx.create_cluster(c)
        before = ctx.get_state(cid)
        t0 = time.perf_counter()
        st = ctx.solve_step(cid)
        assert time.perf_counter() - t0 < 10.0
        assert st["status"] == ba.BA_ERR_TIMEOUT and st["accepted"] == 0
        assert st["mu_used"] == 1e-4 and st["mu"] == 2e-4 and st["nu"] == 4.0
        for a, b in zip(ctx.get_state(cid), before):
            assert np.array_equal(a, b)
        tr = ctx.run(cid, 3)  # every iteration of a graph launch gives up the same way
        assert [t["status"] for t in tr] == [ba.BA_ERR_TIMEOUT] * 3
        assert [t["accepted"] for t in tr] == [0, 0, 0]
        assert tr[-1]["mu"] == pytest.approx(2e-4 * 4 * 8 * 16)
        for a, b in zip(ctx.get_state(cid), before):
            assert np.array_equal(a, b)
    with ba.Context(precision=ba.BA_MIXED) as ctx:  # the device is still usable
        cid = ctx.create_cluster(c)
        st = ctx.solve_step(cid)
        assert st["status"] == 0 and st["accepted"] == 1


def test_expired_copy_wait_in_a_batch_and_in_serving(ba):
    scenes = sg.batch_c3(replica=3, n_clusters=3, scale=0.1)
    with ba.Context(precision=ba.BA_MIXED, flags=ba.BA_FLAG_INJECT_COPY_TIMEOUT) as ctx:
        ids = [ctx.create_cluster(s) for s in scenes]
        res = ctx.solve_batch(ids, 2)
        assert [r["status"] for r in res] == [ba.BA_ERR_TIMEOUT] * 3
        assert [r["accepted"] for r in res] == [0, 0, 0]
        t = ctx.submit(ids[0], 2)
        deadline = time.perf_counter() + 30.0
        r = None
        while r is None and time.perf_counter() < deadline:
            r = ctx.poll(t)
            time.sleep(0.001)
        assert r is not None and r["status"] == ba.BA_ERR_TIMEOUT and r["iters"] == 2
