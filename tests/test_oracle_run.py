"""Pins for the oracle's IMM driver (Alg. 1 with Tang et al.'s theta control):
the recorded ladder, stopping round, LB and theta are re-derived from the
per-round coverage the driver reports, and the final seeds equal a plain
greedy over the final set stream."""
import math

import numpy as np

import graphgen
import oracle


def check_run(g, k, eps, ell, seed):
    o = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
    seeds, st = o.run(k, eps, ell, seed)
    prm = oracle.theta_params(g.n, k, eps, ell)
    n = g.n
    eps_p = math.sqrt(2.0) * eps
    lb = 1.0
    for i in range(1, st.rounds + 1):
        x = n / 2.0 ** i
        assert st.theta_i[i - 1] == math.ceil(prm["lambda_prime"] / x)
        assert st.sets_i[i - 1] == st.theta_i[i - 1]      # stream grows exactly to theta_i
        nF = n * st.covered_i[i - 1] / st.sets_i[i - 1]
        hit = nF >= (1.0 + eps_p) * x
        assert hit == (i == st.rounds and st.stopped_early == 1)
        if hit:
            lb = nF / (1.0 + eps_p)
    if not st.stopped_early:
        assert st.rounds == prm["rounds"]
    assert math.isclose(st.lb, lb, rel_tol=0, abs_tol=0)
    assert st.theta == math.ceil(prm["lambda_star"] / lb)
    assert st.num_sets == max(st.theta, st.sets_i[st.rounds - 1] if st.rounds else 0)
    # final selection = greedy over the final stream
    off, mem = o.arena()
    s2, c2 = oracle.select_sets(n, off, mem, k)
    assert np.array_equal(seeds, s2) and st.covered == c2
    return seeds, st


def test_run_small_weighted_cascade():
    g = graphgen.make_graph(4096, 32768, 1, graphgen.IC, "inv_indeg")
    seeds, st = check_run(g, 10, 0.5, 1.0, 1)
    assert len(set(seeds.tolist())) == 10
    assert st.stopped_early == 1


def test_run_small_lt():
    g = graphgen.make_graph(2048, 16384, 7, graphgen.LT, "inv_indeg")
    check_run(g, 8, 0.5, 1.0, 7)


def test_run_tiny_no_early_stop():
    # a graph with no edges: every set is a singleton, coverage stays near k/n,
    # so the LB test never fires and LB stays 1
    n = 64
    row = np.zeros(n + 1, dtype=np.uint64)
    g = graphgen.Graph(n=n, row=row, src=np.zeros(0, dtype=np.uint32),
                       weight=np.zeros(0, dtype=np.float32), model=graphgen.IC)
    seeds, st = check_run(g, 2, 0.5, 1.0, 3)
    assert st.stopped_early == 0 and st.lb == 1.0


def test_run_is_deterministic():
    g = graphgen.make_graph(1024, 8192, 2, graphgen.IC, "inv_indeg")
    a = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
    s1, st1 = a.run(5, 0.4, 1.0, 99)
    s2, st2 = a.run(5, 0.4, 1.0, 99)
    assert np.array_equal(s1, s2) and st1.theta == st2.theta and st1.covered == st2.covered


def test_fresh_final_stream():
    # Chen 2018's correction: the estimation ladder is unchanged, and the final
    # selection runs on exactly theta fresh sets, which are the sets an
    # independent sampler draws under the second key.  Catches a missing reset
    # (stream longer than theta or reusing old sets), a wrong key, and any
    # change to the estimation phase.
    for model, seed in ((graphgen.IC, 11), (graphgen.LT, 12)):
        g = graphgen.make_graph(1500, 12000, seed, model, "inv_indeg")
        k, eps, ell = 6, 0.5, 1.0
        plain = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
        s0, st0 = plain.run(k, eps, ell, seed)
        fresh = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
        s1, st1 = fresh.run(k, eps, ell, seed, fresh_final=True)
        for f in ("rounds", "stopped_early", "lb", "theta", "lambda_prime", "lambda_star"):
            assert getattr(st1, f) == getattr(st0, f), f
        for i in range(st0.rounds):
            assert st1.theta_i[i] == st0.theta_i[i]
            assert st1.covered_i[i] == st0.covered_i[i]
            assert st1.sets_i[i] == st0.sets_i[i]
        assert st1.num_sets == st1.theta and fresh.num_sets == st1.theta
        indep = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
        indep.sample(st1.theta, seed ^ oracle.FRESH_KEY)
        off1, mem1 = fresh.arena()
        off2, mem2 = indep.arena()
        assert np.array_equal(off1, off2) and np.array_equal(mem1, mem2)
        s2, c2 = oracle.select_sets(g.n, off2, mem2, k)
        assert np.array_equal(s1, s2) and st1.covered == c2
        # the fresh stream shares no set with the estimation stream's prefix
        off0, mem0 = plain.arena()
        same = sum(np.array_equal(mem0[off0[i]:off0[i + 1]], mem1[off1[i]:off1[i + 1]]) for i in range(200))
        assert same < 200
