"""Tuning knobs change speed, never results: batched runs under opposite
tunings (cluster vs one-CTA selection, candidate argmax on vs off, large vs
small sampling batches) are identical and equal the oracle; the autotuner
keeps one of its candidates, applies it to the graph contexts and leaves the
results unchanged; solo runs under other thresholds equal the oracle."""
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


def load(imm, g):
    ctx = imm.imm_create(device=0)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    return ctx


def same(a, b):
    assert a.rounds == b.rounds and a.theta == b.theta and a.lb == b.lb
    assert a.num_sets == b.num_sets and a.covered == b.covered
    for i in range(a.rounds):
        assert a.covered_i[i] == b.covered_i[i] and a.sets_i[i] == b.sets_i[i]


def test_batch_results_do_not_depend_on_the_tuning(imm):
    b = graphgen.batch_workload(count=12, max_log_n=15.0)
    ctxs = [load(imm, g) for g in b.graphs]
    queries = [(ctxs[q.graph_id], q.k, q.epsilon, q.ell, q.seed) for q in b.queries]
    runs = []
    for knobs in (dict(cluster_min_n=0, select_cand=1, batch_sets=1 << 22),
                  dict(cluster_min_n=0xFFFFFFFF, select_cand=0, batch_sets=1024)):
        for c in ctxs:
            imm.imm_set_tuning(c, **knobs)
        runs.append(imm.imm_run_batch(queries))
    (sa, ta, ua), (sb, tb, ub) = runs
    assert ua == ub == [0] * len(queries)
    for i in range(len(queries)):
        assert np.array_equal(sa[i], sb[i]), i
        same(ta[i], tb[i])
    for i in (0, 1, 5):
        q = b.queries[i]
        want, ost = oracle_for(b.graphs[q.graph_id]).run(q.k, q.epsilon, q.ell, q.seed)
        assert np.array_equal(sa[i], want)
        same(ta[i], ost)


def test_autotuner_keeps_a_candidate_and_the_results(imm):
    b = graphgen.batch_workload(count=10, max_log_n=15.0)
    ctxs = [load(imm, g) for g in b.graphs]
    queries = [(ctxs[q.graph_id], q.k, q.epsilon, q.ell, q.seed) for q in b.queries]
    s0, t0, u0 = imm.imm_run_batch(queries)
    best, table = imm.imm_autotune_batch(queries, reps=1)
    assert len(table) == imm.IMM_TUNE_CANDIDATES and all(ms > 0 for _, ms in table)
    assert best in [c for c, _ in table]
    assert min(ms for _, ms in table) == dict((tuple(c.items()), ms) for c, ms in table)[tuple(best.items())]
    for c in ctxs:
        assert imm.imm_get_tuning(c) == best
    s1, t1, u1 = imm.imm_run_batch(queries)
    assert u0 == u1 == [0] * len(queries)
    for i in range(len(queries)):
        assert np.array_equal(s0[i], s1[i])
        same(t0[i], t1[i])


def test_solo_results_do_not_depend_on_the_tuning(imm):
    g = graphgen.make_graph(30000, 300000, 4, graphgen.IC, "uniform", pmax=0.12)
    want, ost = oracle_for(g).run(20, 0.4, 1.0, 5)
    for knobs in (dict(select_cta_max_n=0, group_min_mean=1, batch_sets=700),
                  dict(select_cta_max_n=1 << 20, group_min_mean=1 << 30, select_cand=0)):
        ctx = load(imm, g)
        imm.imm_set_tuning(ctx, **knobs)
        seeds, st = imm.imm_run(ctx, g.model, 20, 0.4, 1.0, 5)
        assert np.array_equal(seeds, want), knobs
        same(st, ost)
        imm.imm_destroy(ctx)
