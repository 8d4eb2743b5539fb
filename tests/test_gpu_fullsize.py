"""Full-size workloads through the C ABI, in the launch configuration the
benchmark times.

IC, R-MAT 2^20 vertices / 2^24 edges, p ~ U[0, 0.1], k=50, eps=0.13: the
oracle's complete run takes about two hours on one core and 43 GB of host
memory, so its results are stored (tests/golden/ic_u01_1m.json, written by
tests/golden/make_golden.py, which calls only the oracle): the seed sequence,
the theta ladder with per-round coverage, LB, theta, stream size, coverage,
total members and a digest of the occurrence counts must all be equal.  On
top of that, sampled set ids are recomputed one by one by the oracle (giant
and small sets), and the ladder is re-derived from the GPU's own coverage.

LT, R-MAT 2^22 vertices / 2^26 edges, w = 1/indeg, k=100, eps=0.5: small
enough for the oracle to run in full, so every set, count and seed is
compared."""
import math

import numpy as np
import pytest

import graphgen
import oracle
from gpu_common import (assert_run_equals_golden, assert_same_stream, counts_digest, graph_digest, load_golden,
                        oracle_for)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def imm():
    import torch
    assert torch.cuda.is_available()
    from paper_2411_09473_gb300 import imm as mod
    return mod


def check_ladder(st, n, k, eps, ell):
    prm = oracle.theta_params(n, k, eps, ell)
    assert st.lambda_prime == prm["lambda_prime"] and st.lambda_star == prm["lambda_star"]
    eps_p = math.sqrt(2.0) * eps
    lb = 1.0
    for i in range(1, st.rounds + 1):
        x = math.ldexp(float(n), -i)
        assert st.theta_i[i - 1] == math.ceil(prm["lambda_prime"] / x)
        assert st.sets_i[i - 1] == st.theta_i[i - 1]
        nF = float(n) * float(st.covered_i[i - 1]) / float(st.sets_i[i - 1])
        hit = nF >= (1.0 + eps_p) * x
        assert hit == (i == st.rounds and st.stopped_early == 1)
        if hit:
            lb = nF / (1.0 + eps_p)
    assert st.lb == lb
    assert st.theta == math.ceil(prm["lambda_star"] / lb)
    assert st.num_sets == max(st.theta, st.sets_i[st.rounds - 1])


def test_ic_1m_full_run_sampled_parity(imm):
    w = graphgen.plain_workload("ic_u01_1m")
    g = w.graph
    ctx = imm.imm_create(device=0)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    seeds, st = imm.imm_run(ctx, g.model, w.k, w.epsilon, w.ell, w.seed)
    check_ladder(st, g.n, w.k, w.epsilon, w.ell)
    assert len(set(seeds.tolist())) == w.k
    cnt = imm.imm_get_counts(ctx, g.n)
    assert int(cnt.astype(np.uint64).sum()) == st.members
    # the first pick is the argmax of the counts, lowest id on ties
    assert seeds[0] == int(np.argmax(cnt))
    # the oracle's complete run, stored
    rec = load_golden("ic_u01_1m")
    assert graph_digest(g) == rec["graph_sha256"]
    assert_run_equals_golden(seeds, st, rec, "ic_u01_1m")
    assert counts_digest(cnt) == rec["counts_sha256"] and int(cnt.max()) == rec["counts_max"]
    # sampled set ids, recomputed one by one by the oracle
    o = oracle_for(g)
    rng = np.random.default_rng(2)
    ids = rng.choice(st.num_sets, 400, replace=False)
    checked_big = 0
    for s in ids:
        s = int(s)
        got = imm.imm_get_set(ctx, s, g.n)
        if len(got) > 1000:
            if checked_big >= 25:
                continue
            checked_big += 1
        want = o.sample_one(w.seed, s)
        assert np.array_equal(got, want), s
    assert checked_big >= 5
    imm.imm_destroy(ctx)


def test_lt_4m_full_run_full_parity(imm):
    w = graphgen.plain_workload("lt_4m")
    g = w.graph
    ctx = imm.imm_create(device=0)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    seeds, st = imm.imm_run(ctx, g.model, w.k, w.epsilon, w.ell, w.seed)
    check_ladder(st, g.n, w.k, w.epsilon, w.ell)
    o = oracle_for(g)
    want, ost = o.run(w.k, w.epsilon, w.ell, w.seed)
    assert np.array_equal(seeds, want)
    assert st.theta == ost.theta and st.num_sets == ost.num_sets and st.covered == ost.covered
    assert st.lb == ost.lb
    assert np.array_equal(imm.imm_get_counts(ctx, g.n), o.counts())
    goff, gmem = imm.imm_get_sets(ctx, 0, st.num_sets)
    ooff, omem = o.arena()
    assert_same_stream(goff, gmem, ooff, omem)
    imm.imm_destroy(ctx)


def test_ic_u1_256k_full_run_equals_oracle(imm):
    """The paper's IC weight law (p ~ U[0, 1]) on R-MAT 2^18 / 2^22, k=50,
    eps=0.5: every field of the oracle's stored run, the occurrence counts,
    and every set of a sample of ids."""
    w = graphgen.plain_workload("ic_u1_256k")
    g = w.graph
    rec = load_golden("ic_u1_256k")
    assert graph_digest(g) == rec["graph_sha256"]
    ctx = imm.imm_create(device=0)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    seeds, st = imm.imm_run(ctx, g.model, w.k, w.epsilon, w.ell, w.seed)
    assert_run_equals_golden(seeds, st, rec, "ic_u1_256k")
    cnt = imm.imm_get_counts(ctx, g.n)
    assert counts_digest(cnt) == rec["counts_sha256"]
    o = oracle_for(g)
    for s in np.random.default_rng(6).choice(st.num_sets, 40, replace=False):
        assert np.array_equal(imm.imm_get_set(ctx, int(s), g.n), o.sample_one(w.seed, int(s))), int(s)
    imm.imm_destroy(ctx)
