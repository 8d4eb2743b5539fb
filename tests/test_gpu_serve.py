"""Served IMM (continuous batching): queries submitted at different times,
while others are in flight, each return exactly their solo imm_run result."""
import time

import numpy as np
import pytest

import graphgen
from gpu_common import assert_run_equals_golden, graph_digest, load_golden

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


def test_served_results_equal_solo_runs(imm):
    graphs = [graphgen.make_graph(4096, 32768, 1, graphgen.IC, "inv_indeg"),
              graphgen.make_graph(6000, 60000, 2, graphgen.LT, "inv_indeg"),
              graphgen.make_graph(20000, 160000, 3, graphgen.IC, "inv_indeg")]
    ctxs = [load(imm, g) for g in graphs]
    srv = imm.imm_server_create(ctxs, memory_budget_bytes=8 << 30, max_active=16)
    rng = np.random.default_rng(0)
    queries = []
    for i in range(24):
        gid = int(rng.integers(0, 3))
        queries.append((gid, int(rng.integers(1, 40)), float(rng.uniform(0.2, 0.5)), 1.0, 1000 + i))
    ids = {}
    for i, q in enumerate(queries):
        ids[imm.imm_server_submit(srv, *q)] = q
        if i % 6 == 5:
            time.sleep(0.02)  # later submissions join waves already in flight
    got = {}
    deadline = time.time() + 300
    while len(got) < len(queries) and time.time() < deadline:
        for (qid, status, lat, qms) in imm.imm_server_poll(srv):
            assert status == 0, status
            assert lat >= qms >= 0
            q = ids[qid]
            got[qid] = imm.imm_server_take(srv, qid, q[1])
        time.sleep(0.005)
    assert len(got) == len(queries)
    info = imm.imm_server_info(srv)
    assert info["status"] == 0 and info["active"] == 0 and info["pending"] == 0
    imm.imm_server_destroy(srv)
    for qid, (seeds, st) in got.items():
        gid, k, eps, ell, seed = ids[qid]
        s2, st2 = imm.imm_run(ctxs[gid], graphs[gid].model, k, eps, ell, seed)
        assert np.array_equal(seeds, s2)
        assert st.theta == st2.theta and st.lb == st2.lb and st.covered == st2.covered


def test_served_rejects_bad_queries(imm):
    g = graphgen.make_graph(1024, 8192, 5, graphgen.IC, "inv_indeg")
    ctx = load(imm, g)
    srv = imm.imm_server_create([ctx])
    with pytest.raises(imm.ImmError):
        imm.imm_server_submit(srv, 1, 5, 0.5, 1.0, 1)      # no graph 1
    with pytest.raises(imm.ImmError):
        imm.imm_server_submit(srv, 0, 0, 0.5, 1.0, 1)      # k = 0
    with pytest.raises(imm.ImmError):
        imm.imm_server_take(srv, 12345, 5)                 # unknown id
    imm.imm_server_destroy(srv)


def test_served_memory_bound_admission_still_drains(imm):
    # a budget smaller than one query's working set: admission is memory-bound
    # throughout, idle workers are reclaimed, and every query still completes
    g = graphgen.make_graph(20000, 160000, 3, graphgen.IC, "inv_indeg")
    ctx = load(imm, g)
    srv = imm.imm_server_create([ctx], memory_budget_bytes=16 << 20, max_active=4)
    qs = [(0, 10 + i, 0.3 + 0.01 * i, 1.0, 500 + i) for i in range(12)]
    ids = {imm.imm_server_submit(srv, *q): q for q in qs}
    got = {}
    deadline = time.time() + 300
    while len(got) < len(qs) and time.time() < deadline:
        for (qid, status, _, _) in imm.imm_server_poll(srv):
            got[qid] = (status, imm.imm_server_take(srv, qid, ids[qid][1]) if status == 0 else None)
        time.sleep(0.005)
    assert len(got) == len(qs)
    imm.imm_server_destroy(srv)
    for qid, (status, res) in got.items():
        assert status == 0, status
        gid, k, eps, ell, seed = ids[qid]
        s2, _ = imm.imm_run(ctx, g.model, k, eps, ell, seed)
        assert np.array_equal(res[0], s2)


def test_served_stream_equals_oracle_runs(imm):
    """The first queries of the served workload (8 resident R-MAT graphs of
    2^16..2^20 vertices, Poisson arrivals at 200/s, k 10..200, eps 0.1..0.5),
    replayed at their arrival times against a server with the benchmark's
    settings: every result equals the oracle's own run of the query, stored by
    tests/golden/make_golden.py."""
    gold = load_golden("served")
    graphs = graphgen.served_graphs()
    for g, rec in zip(graphs, gold["graphs"]):
        assert graph_digest(g) == rec["graph_sha256"]
    ctxs = [load(imm, g) for g in graphs]
    qs = graphgen.served_queries()[: gold["queries"]]
    srv = imm.imm_server_create(ctxs, memory_budget_bytes=96 << 30, max_active=128)
    ids, got = {}, {}
    t0 = time.perf_counter()
    i = 0
    deadline = t0 + 600
    while len(got) < len(qs) and time.perf_counter() < deadline:
        now = time.perf_counter() - t0
        while i < len(qs) and qs[i].arrival_s <= now:
            q = qs[i]
            ids[imm.imm_server_submit(srv, q.graph_id, q.k, q.epsilon, q.ell, q.seed)] = i
            i += 1
        for (qid, status, _, _) in imm.imm_server_poll(srv):
            assert status == 0, status
            j = ids[qid]
            got[j] = imm.imm_server_take(srv, qid, qs[j].k)
        time.sleep(0.001)
    assert len(got) == len(qs)
    imm.imm_server_destroy(srv)
    for j, q in enumerate(qs):
        rec = gold["results"][j]
        assert (q.graph_id, q.k, q.epsilon.hex(), q.seed) == (rec["graph_id"], rec["k"], rec["epsilon_hex"],
                                                               rec["seed"]), j
        seeds, st = got[j]
        assert_run_equals_golden(seeds, st, rec, f"query {j}")
    for c in ctxs:
        imm.imm_destroy(c)


def test_served_shared_streams_equal_oracle_runs(imm):
    """Prefix-stable stream sharing: queries on the same graph with the same
    rng seed (and different k and epsilon) reuse the resident stream of the
    previous one, and each still equals the oracle's run of it alone."""
    from gpu_common import oracle_for
    graphs = [graphgen.make_graph(4096, 32768, 1, graphgen.IC, "inv_indeg"),
              graphgen.make_graph(6000, 60000, 2, graphgen.LT, "inv_indeg")]
    ctxs = [load(imm, g) for g in graphs]
    srv = imm.imm_server_create(ctxs, memory_budget_bytes=8 << 30, max_active=4, share_streams=True)
    # (graph, k, eps, seed, reuses): one query at a time, so each graph has one
    # idle worker; a query with that worker's seed reuses its stream, one with
    # another seed replaces it
    plan = [(0, 10, 0.5, 11, False), (0, 5, 0.3, 11, True), (0, 20, 0.45, 11, True), (0, 10, 0.5, 12, False),
            (0, 10, 0.5, 11, False), (1, 25, 0.4, 13, False), (1, 10, 0.2, 13, True), (1, 40, 0.5, 13, True)]
    for (gid, k, eps, seed, reuses) in plan:
        qid = imm.imm_server_submit(srv, gid, k, eps, 1.0, seed)
        got = None
        deadline = time.time() + 120
        while got is None and time.time() < deadline:
            for (cid, status, _, _) in imm.imm_server_poll(srv):
                assert cid == qid and status == 0
                got = imm.imm_server_take(srv, qid, k)
            time.sleep(0.002)
        assert got is not None
        seeds, st = got
        g = graphs[gid]
        o = oracle_for(g)
        want, ost = o.run(k, eps, 1.0, seed)
        assert np.array_equal(seeds, want), (gid, k, eps, seed)
        assert st.rounds == ost.rounds and st.theta == ost.theta and st.lb == ost.lb
        assert st.num_sets == ost.num_sets and st.covered == ost.covered and st.members == o.num_members
        for i in range(st.rounds):
            assert st.covered_i[i] == ost.covered_i[i] and st.sets_i[i] == ost.sets_i[i]
        assert (st.reused_sets > 0) == reuses, (gid, k, eps, seed, st.reused_sets)
    imm.imm_server_destroy(srv)
