"""The double-float factorisation of the small reduced camera systems (up to
32 free images, one CTA in shared memory): the mixed path's factor.

Under BA_FLAG_SMALL_DF_FACTOR the binary64 path uses it too, so that its
steps can be held to the oracle at the binary64 parity bar (1e-10 per step on
the state, F, the decision and the damping): the refinement against the
binary64 S removes the factor's rounding.  Panel widths from 3 (ragged last
panel) to 32 (one warp's diagonal block), a system that is not positive
definite until mu has grown (through subnormal binary64 pivots, which the
power-of-two equilibration brings into range), and the mixed path's decisions
against the binary64 path's.
"""
import pytest

import oracle as O
import scenegen as sg
from helpers import compare_steps, fp64_step_parity
from test_gpu_parity import unobserved_camera_cluster

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ba():
    import paper_2511_06152_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("nb", [3, 8, 16, 32])
def test_df_factor_keeps_fp64_parity_c1(ba, nb):
    c = sg.cluster_c1()
    P, S = O.Problem(c), O.State(c)
    with ba.Context(precision=ba.BA_FP64, flags=ba.BA_FLAG_SMALL_DF_FACTOR, tune_table=None) as ctx:
        ctx.set_tune(factor_nb=nb)
        cid = ctx.create_cluster(c)
        assert ctx.cluster_info(cid)["n_free"] <= 32
        assert compare_steps(ctx, cid, O, P, S, sg.ITERS["c1"]) >= 10


@pytest.mark.parametrize("seed,strips,per,pts", [(31, 2, 4, 400), (32, 3, 7, 900), (33, 4, 8, 1500)])
def test_df_factor_keeps_fp64_parity_small_clusters(ba, seed, strips, per, pts):
    c = sg.tiny_cluster(seed, strips, per, pts)
    assert fp64_step_parity(ba, O, c, 6, flags=ba.BA_FLAG_SMALL_DF_FACTOR) >= 4


def test_df_factor_not_positive_definite_matches_oracle(ba):
    """Rejections while the unobserved image's block mu * 1e-6 underflows to
    0, then steps whose pivot is a subnormal binary64 number: the same status,
    decisions, damping and states as the oracle."""
    c = unobserved_camera_cluster()
    n = fp64_step_parity(ba, O, c, 8, flags=ba.BA_FLAG_SMALL_DF_FACTOR)
    assert n == 8


@pytest.mark.parametrize("nb", [3, 8, 16, 32])
def test_mixed_decisions_follow_fp64_for_every_panel_width(ba, nb):
    c = sg.cluster_c1()
    with ba.Context(precision=ba.BA_MIXED, tune_table=None) as cm, ba.Context(precision=ba.BA_FP64) as cd:
        cm.set_tune(factor_nb=nb)
        a, b = cm.create_cluster(c), cd.create_cluster(c)
        tm, td = cm.run(a, 10), cd.run(b, 10)
    for x, y in zip(tm, td):
        assert x["accepted"] == y["accepted"]
        assert x["F_after"] == pytest.approx(y["F_after"], rel=1e-6)
