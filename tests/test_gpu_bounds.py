"""The bounds-checked build (-DIMM_BOUNDS_CHECK) on the paths the parity tests
cover: IC on the weighted-cascade workload, fuzzed dense graphs, giant sets
through both large-set paths (bitmap- and list-stored), LT walks of every
length (lane path, per-walk tables, bitmap slots), a small batch with both selection teams, and OPIM.  Every index
check passes (a failed one returns an error) and every result equals the
oracle's.  Each case runs in a process of its own that loads the checked
library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

PRELUDE = r"""
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import numpy as np
import graphgen
from gpu_common import oracle_for, assert_same_stream
from paper_2411_09473_gb300 import imm
assert imm.imm_build_flags() & imm.IMM_BUILD_BOUNDS_CHECK


def load(g):
    c = imm.imm_create(device=0)
    imm.imm_load_graph(c, g.n, g.m, g.row, g.src, g.weight, g.model)
    return c


def run_equal(g, k, eps, seed):
    c = load(g)
    seeds, st = imm.imm_run(c, g.model, k, eps, 1.0, seed)
    want, ost = oracle_for(g).run(k, eps, 1.0, seed)
    assert np.array_equal(seeds, want) and st.theta == ost.theta and st.covered == ost.covered
    imm.imm_destroy(c)


def stream_equal(g, theta, seed, ks):
    c = load(g)
    imm.imm_sample(c, g.model, theta, seed)
    o = oracle_for(g)
    o.sample(theta, seed)
    off, mem = imm.imm_get_sets(c, 0, theta)
    ooff, omem = o.arena()
    assert_same_stream(off, mem, ooff, omem)
    for k in ks:
        s1, c1 = imm.imm_select(c, k)
        s2, c2 = o.select(k)
        assert np.array_equal(s1, s2) and c1 == c2
    imm.imm_destroy(c)
"""

CASES = {
    "ic_wc": "run_equal(graphgen.plain_workload('ic_wc_4k').graph, 10, 0.5, 1)",
    "fuzz": """
for gs in range(3):
    g = graphgen.make_graph(3000 + 500 * gs, 30000, 40 + gs, graphgen.IC, 'uniform', pmax=0.25)
    stream_equal(g, 1500, gs + 1, (1, 7, 30))
""",
    "giant_cta": "stream_equal(graphgen.make_graph(20000, 160000, 13, graphgen.IC, 'uniform', pmax=0.5), 700, 3, (1, 40))",
    "giant_group": "stream_equal(graphgen.make_graph(20000, 160000, 13, graphgen.IC, 'uniform', pmax=0.5), 700, 3, (1, 40))",
    "lt": """
stream_equal(graphgen.make_graph(20000, 160000, 3, graphgen.LT, 'inv_indeg'), 4000, 5, (1, 25))
n = 600
row = np.arange(n + 1, dtype=np.uint64)
src = np.array([(v + 1) % n for v in range(n)], dtype=np.uint32)
stream_equal(graphgen.Graph(n=n, row=row, src=src, weight=np.ones(n, dtype=np.float32), model=graphgen.LT), 50, 2, (3,))
from test_gpu_parity import chain_graph
stream_equal(chain_graph([900, 1500, 1800] * 10), 3000, 8, (1, 20))
""",
    "batch_opim": """
b = graphgen.batch_workload(count=8, max_log_n=15.0)
ctxs = [load(g) for g in b.graphs]
qs = [(ctxs[q.graph_id], q.k, q.epsilon, q.ell, q.seed) for q in b.queries]
for cmin in (0, 0xFFFFFFFF):
    for c in ctxs:
        imm.imm_set_tuning(c, cluster_min_n=cmin)
    seeds, stats, status = imm.imm_run_batch(qs)
    assert status == [0] * len(qs)
    for i, q in enumerate(b.queries):
        want, ost = oracle_for(b.graphs[q.graph_id]).run(q.k, q.epsilon, q.ell, q.seed)
        assert np.array_equal(seeds[i], want) and stats[i].theta == ost.theta
g = graphgen.plain_workload('ic_wc_4k').graph
c = load(g)
seeds, st = imm.imm_run_opim(c, g.model, 10, 0.3, 1.0, 2)
want, ost = oracle_for(g).opim_run(10, 0.3, 1.0, 2)
assert np.array_equal(seeds, want) and st.rounds == ost.rounds
""",
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_bounds_checked_build(case):
    code = PRELUDE.format(root=ROOT, tests=HERE) + CASES[case] + "\nprint('case ok')\n"
    env = dict(os.environ, IMM_LIBRARY_VARIANT="bounds")
    if case == "giant_cta":
        env["IMM_IC_LARGE"] = "cta"
    if case == "giant_group":
        env["IMM_IC_LARGE"] = "group"
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "case ok" in r.stdout, r.stderr[-3000:]
