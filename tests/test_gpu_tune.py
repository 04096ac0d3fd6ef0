"""Autotuned launch shapes on the GPU: tuned parameters keep FP64 step
parity with the oracle (1e-10) and batch = alone bit for bit, the large
block's panel width keeps parity too, a batch split into any number of
concurrent launch chains gives the one-chain results bit for bit, and
ba_autotune returns a valid choice that is no slower than the defaults on the
batch it measured."""
import numpy as np
import pytest

import oracle as O
import scenegen as sg
from helpers import compare_steps

pytestmark = pytest.mark.gpu

TUNED_FP64 = dict(chunk_tiles=4, lin_ctas_per_sm=2, back_ctas_per_sm=4, factor_nb=4, factor_threads=256,
                  big_panel_w=8, batch_chains=3)
TUNED_MIXED = dict(TUNED_FP64, chunk_tiles=8, factor_nb=16, factor_threads=384)


@pytest.fixture(scope="module")
def ba():
    import paper_2511_06152_gb300 as m
    m.lib()
    return m


def test_tuned_parameters_keep_fp64_parity(ba):
    c = sg.cluster_c1()
    P, S = O.Problem(c), O.State(c)
    with ba.Context(precision=ba.BA_FP64, tune_table=None) as ctx:
        ctx.set_tune(**TUNED_FP64)
        assert {k: ctx.get_tune()[k] for k in TUNED_FP64} == TUNED_FP64
        cid = ctx.create_cluster(c)
        info = ctx.cluster_info(cid)
        assert info["n_chunks"] == -(-info["n_tiles"] // 4)  # chunks of four tiles
        assert compare_steps(ctx, cid, O, P, S, sg.ITERS["c1"]) >= 10


def test_tuned_large_block_panel_keeps_parity(ba):
    c = sg.tiny_cluster(5151, 4, 10, 3000, fixed=(0, 11))
    P, S = O.Problem(c), O.State(c)
    with ba.Context(precision=ba.BA_FP64, tune_table=None) as ctx:
        ctx.set_tune(big_panel_w=8)
        cid = ctx.create_cluster(c)
        assert compare_steps(ctx, cid, O, P, S, 8) >= 8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tuned_batch_equals_alone_bitwise(ba, precision):
    prec = ba.BA_FP64 if precision == "fp64" else ba.BA_MIXED
    scenes = sg.batch_c3(replica=11, n_clusters=5, scale=0.1)
    with ba.Context(precision=prec, tune_table=None) as ctx:
        ctx.set_tune(**(TUNED_FP64 if precision == "fp64" else TUNED_MIXED))
        ids = [ctx.create_cluster(s) for s in scenes]
        alone = []
        for i in ids:
            ctx.run(i, 4, trace=False)
            alone.append(ctx.get_state(i))
            ctx.reset(i)
        ctx.solve_batch(ids, 4)
        for i, a in zip(ids, alone):
            for u, v in zip(ctx.get_state(i), a):
                assert np.array_equal(u, v)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_launch_chains_do_not_change_results(ba, precision):
    # seven batch clusters and one with more than 32 free images (the
    # global-memory solver), as one chain, three chains and eight chains
    prec = ba.BA_FP64 if precision == "fp64" else ba.BA_MIXED
    scenes = sg.batch_c3(replica=13, n_clusters=7, scale=0.1) + [sg.tiny_cluster(5151, 4, 10, 3000, fixed=(0, 11))]
    with ba.Context(precision=prec, tune_table=None) as ctx:
        ids = [ctx.create_cluster(s) for s in scenes]
        ref = None
        for k in (1, 3, 8):
            ctx.set_tune(batch_chains=k)
            ctx.reset_batch(ids)
            res = ctx.solve_batch(ids, 4, trace=True)
            states = [ctx.get_state(i) for i in ids]
            if ref is None:
                ref = (res, states)
                continue
            for a, b in zip(states, ref[1]):
                for u, v in zip(a, b):
                    assert np.array_equal(u, v)
            assert res == ref[0]


def test_autotune_returns_a_valid_choice(ba):
    scenes = sg.batch_c3(replica=12, n_clusters=6, scale=0.1)
    with ba.Context(precision=ba.BA_MIXED, tune_table=None) as ctx:
        t = ctx.autotune(scenes, 2)
        assert 4 <= t["chunk_tiles"] <= 16 and t["factor_threads"] in (256, 384, 512)
        assert 0 < t["ms_tuned"] <= t["ms_default"]
        assert {k: v for k, v in ctx.get_tune().items() if not k.startswith("ms")} == \
            {k: v for k, v in t.items() if not k.startswith("ms")}
        assert ctx.memory_in_use() < 64 << 20  # the tuning clusters are gone
        cid = ctx.create_cluster(scenes[0])
        tr = ctx.run(cid, 3)
        assert all(x["status"] == 0 for x in tr)


def test_set_tune_rejects_out_of_range(ba):
    with ba.Context(precision=ba.BA_MIXED, tune_table=None) as ctx:
        for bad in (dict(chunk_tiles=17), dict(factor_threads=300), dict(big_panel_w=3), dict(lin_ctas_per_sm=0),
                    dict(batch_chains=0), dict(batch_chains=9)):
            with pytest.raises(ba.BAError) as ei:
                ctx.set_tune(**bad)
            assert ei.value.status == ba.BA_ERR_INVALID
