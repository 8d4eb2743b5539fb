"""OPIM-style early stop (imm_run_opim) through the C ABI: seeds, the
collections' sizes, both coverages, both confidence bounds and the stop
round equal the oracle's opim_run bit for bit, on IC and LT graphs and on a
graph whose second collection holds bitmap-stored giant sets."""
import numpy as np
import pytest

import graphgen
from gpu_common import oracle_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def imm():
    import torch
    assert torch.cuda.is_available()
    from paper_2411_09473_gb300 import imm as mod
    return mod


def same(imm, g, k, eps, ell, seed):
    ctx = imm.imm_create(device=0)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    seeds, st = imm.imm_run_opim(ctx, g.model, k, eps, ell, seed)
    want, ost = oracle_for(g).opim_run(k, eps, ell, seed)
    assert np.array_equal(seeds, want)
    assert (st.rounds, st.stopped_early, st.i_max) == (ost.rounds, ost.stopped_early, ost.i_max)
    assert st.theta_max == ost.theta_max and st.theta_0 == ost.theta_0 and st.alpha == ost.alpha
    for i in range(st.rounds):
        assert st.sets_i[i] == ost.sets_i[i]
        assert st.cov1_i[i] == ost.cov1_i[i] and st.cov2_i[i] == ost.cov2_i[i], i
        assert st.upper_i[i] == ost.upper_i[i] and st.lower_i[i] == ost.lower_i[i], i
    # the context keeps R1: the plain stream under the seed
    assert imm.imm_stream_size(ctx)[0] == st.sets_i[st.rounds - 1]
    imm.imm_destroy(ctx)
    return st


def test_opim_ic_weighted_cascade(imm):
    g = graphgen.plain_workload("ic_wc_4k").graph
    for (k, eps, seed) in [(10, 0.5, 1), (5, 0.2, 9), (20, 0.3, 4), (1, 0.1, 3)]:
        same(imm, g, k, eps, 1.0, seed)


def test_opim_lt(imm):
    g = graphgen.make_graph(20000, 160000, 3, graphgen.LT, "inv_indeg")
    for (k, eps, seed) in [(10, 0.3, 2), (50, 0.2, 5)]:
        same(imm, g, k, eps, 1.0, seed)


def test_opim_giant_bitmap_sets(imm):
    # high edge probabilities: giant sets, stored as bitmaps in both collections
    g = graphgen.make_graph(8192, 65536, 21, graphgen.IC, "uniform", pmax=0.6)
    st = same(imm, g, 10, 0.2, 1.0, 7)
    assert st.cov2_i[st.rounds - 1] > 0


def test_opim_full_workloads_equal_oracle_runs(imm):
    """lt_4m and ic_u1_256k at full size: every field of the oracle's stored
    OPIM run (tests/golden/opim.json)."""
    from gpu_common import graph_digest, load_golden
    gold = load_golden("opim")
    for rec in gold["runs"]:
        w = graphgen.plain_workload(rec["workload"])
        g = w.graph
        assert graph_digest(g) == rec["graph_sha256"]
        ctx = imm.imm_create(device=0)
        imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
        seeds, st = imm.imm_run_opim(ctx, g.model, w.k, w.epsilon, w.ell, w.seed)
        r = st.rounds
        assert [int(x) for x in seeds] == rec["seeds"] and r == rec["rounds"] and st.i_max == rec["i_max"]
        assert [int(st.sets_i[i]) for i in range(r)] == rec["sets_i"]
        assert [int(st.cov1_i[i]) for i in range(r)] == rec["cov1_i"]
        assert [int(st.cov2_i[i]) for i in range(r)] == rec["cov2_i"]
        assert [float(st.upper_i[i]).hex() for i in range(r)] == rec["upper_hex"]
        assert [float(st.lower_i[i]).hex() for i in range(r)] == rec["lower_hex"]
        assert float(st.alpha).hex() == rec["alpha_hex"] and st.stopped_early == rec["stopped_early"]
        imm.imm_destroy(ctx)
