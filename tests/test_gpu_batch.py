"""Batched IMM (many queries in one engine run): every query's seeds, theta
ladder, LB and theta equal its solo imm_run, and the oracle's on small
cases."""
import numpy as np
import pytest

import graphgen
from gpu_common import assert_run_equals_golden, graph_digest, load_golden, oracle_for

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


def same_run(a, b):
    assert a.rounds == b.rounds and a.stopped_early == b.stopped_early
    for i in range(a.rounds):
        assert a.theta_i[i] == b.theta_i[i] and a.covered_i[i] == b.covered_i[i] and a.sets_i[i] == b.sets_i[i]
    assert a.lb == b.lb and a.theta == b.theta and a.num_sets == b.num_sets and a.covered == b.covered


def test_batch_equals_solo_runs(imm):
    b = graphgen.batch_workload(count=10, max_log_n=14.0)
    ctxs = [load(imm, g) for g in b.graphs]
    queries = [(ctxs[q.graph_id], q.k, q.epsilon, q.ell, q.seed) for q in b.queries]
    seeds, stats, status = imm.imm_run_batch(queries)
    assert status == [0] * len(queries)
    for i, q in enumerate(b.queries):
        g = b.graphs[q.graph_id]
        solo = load(imm, g)
        s2, st2 = imm.imm_run(solo, g.model, q.k, q.epsilon, q.ell, q.seed)
        assert np.array_equal(seeds[i], s2), i
        same_run(stats[i], st2)
    # and the oracle on the first two
    for i in range(2):
        q = b.queries[i]
        g = b.graphs[q.graph_id]
        want, ost = oracle_for(g).run(q.k, q.epsilon, q.ell, q.seed)
        assert np.array_equal(seeds[i], want)
        same_run(stats[i], ost)


def test_batch_shared_graph_and_order_independence(imm):
    # several queries on one graph, submitted in two orders: same answers
    g = graphgen.make_graph(4096, 32768, 9, graphgen.IC, "inv_indeg")
    ctx = load(imm, g)
    qs = [(ctx, 10, 0.5, 1.0, 1), (ctx, 5, 0.3, 1.0, 2), (ctx, 20, 0.4, 1.0, 3), (ctx, 10, 0.5, 1.0, 4)]
    a, sa, _ = imm.imm_run_batch(qs)
    b, sb, _ = imm.imm_run_batch(list(reversed(qs)))
    for i in range(len(qs)):
        assert np.array_equal(a[i], b[len(qs) - 1 - i])
        same_run(sa[i], sb[len(qs) - 1 - i])
    # the graph context's own stream is untouched by the batch
    assert imm.imm_stream_size(ctx) == (0, 0)


def test_batch_rejects_bad_queries(imm):
    g = graphgen.make_graph(1024, 8192, 2, graphgen.IC, "inv_indeg")
    ctx = load(imm, g)
    with pytest.raises(imm.ImmError):
        imm.imm_run_batch([(ctx, 0, 0.5, 1.0, 1)])
    with pytest.raises(imm.ImmError):
        imm.imm_run_batch([(ctx, 5, 1.5, 1.0, 1)])


def test_batch64_equals_oracle_runs(imm):
    """The batched workload at its full size (64 instances, n up to 2^18,
    IC/LT alternating, k 5..100, eps 0.1..0.5): every instance equals the
    oracle's own run of it, stored by tests/golden/make_golden.py."""
    gold = load_golden("batch64")
    b = graphgen.batch_workload(count=gold["count"], max_log_n=gold["max_log_n"])
    ctxs = [load(imm, g) for g in b.graphs]
    queries = [(ctxs[q.graph_id], q.k, q.epsilon, q.ell, q.seed) for q in b.queries]
    seeds, stats, status = imm.imm_run_batch(queries)
    assert status == [0] * len(queries)
    for i, q in enumerate(b.queries):
        rec = gold["instances"][i]
        g = b.graphs[q.graph_id]
        assert graph_digest(g) == rec["graph_sha256"], i
        assert (q.k, q.epsilon.hex(), q.seed) == (rec["k"], rec["epsilon_hex"], rec["seed"]), i
        assert_run_equals_golden(seeds[i], stats[i], rec, f"instance {i}")
    for c in ctxs:
        imm.imm_destroy(c)


_FORCED = r"""
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import numpy as np
import graphgen
from gpu_common import oracle_for
from paper_2411_09473_gb300 import imm
b = graphgen.batch_workload(count=12, max_log_n=14.0)
ctxs = []
for g in b.graphs:
    c = imm.imm_create(device=0)
    imm.imm_load_graph(c, g.n, g.m, g.row, g.src, g.weight, g.model)
    ctxs.append(c)
seeds, stats, status = imm.imm_run_batch([(ctxs[q.graph_id], q.k, q.epsilon, q.ell, q.seed) for q in b.queries])
assert status == [0] * len(b.queries), status
for i, q in enumerate(b.queries):
    g = b.graphs[q.graph_id]
    o = oracle_for(g)
    want, ost = o.run(q.k, q.epsilon, q.ell, q.seed)
    assert np.array_equal(seeds[i], want), i
    st = stats[i]
    assert st.theta == ost.theta and st.covered == ost.covered and st.lb == ost.lb and st.num_sets == ost.num_sets
print("forced ok")
"""


@pytest.mark.parametrize("min_n", ["0", "4294967295"])
def test_batch_selection_teams_forced(min_n):
    """Every instance selects with a cluster of CTAs (min_n = 0), or every one
    with a single CTA: both equal the oracle's runs (a fresh process, since
    the threshold is read once)."""
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    code = _FORCED.format(root=os.path.dirname(here), tests=here)
    env = dict(os.environ, IMM_SELECT_CLUSTER_MIN_N=min_n)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "forced ok" in r.stdout, r.stderr[-3000:]
