"""The stored oracle results under tests/golden/ (written by
tests/golden/make_golden.py) are the oracle's: cheap entries are recomputed
here by the oracle and must match field by field, and every entry's theta
ladder obeys Alg. 1's stopping rule with the oracle's own theta constants."""
import json
import math
import os

import numpy as np
import pytest

import graphgen
import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name + ".json")) as f:
        return json.load(f)


def check_ladder(rec, n, k, eps, ell):
    prm = oracle.theta_params(n, k, eps, ell)
    assert float(prm["lambda_prime"]).hex() == rec["lambda_prime_hex"]
    assert float(prm["lambda_star"]).hex() == rec["lambda_star_hex"]
    eps_p = math.sqrt(2.0) * eps
    lb = 1.0
    for i in range(1, rec["rounds"] + 1):
        x = math.ldexp(float(n), -i)
        assert rec["theta_i"][i - 1] == math.ceil(prm["lambda_prime"] / x) == rec["sets_i"][i - 1]
        nF = float(n) * rec["covered_i"][i - 1] / rec["sets_i"][i - 1]
        hit = nF >= (1.0 + eps_p) * x
        assert hit == (i == rec["rounds"] and rec["stopped_early"] == 1)
        if hit:
            lb = nF / (1.0 + eps_p)
    assert float(lb).hex() == rec["lb_hex"]
    assert rec["theta"] == math.ceil(prm["lambda_star"] / lb)
    assert rec["num_sets"] == max(rec["theta"], rec["sets_i"][-1] if rec["sets_i"] else 0)
    assert len(rec["seeds"]) == k and len(set(rec["seeds"])) == k


def same_as_run(rec, seeds, st, o=None):
    r = st.rounds
    assert [int(x) for x in seeds] == rec["seeds"]
    assert r == rec["rounds"] and [int(st.covered_i[i]) for i in range(r)] == rec["covered_i"]
    assert float(st.lb).hex() == rec["lb_hex"] and st.theta == rec["theta"]
    assert st.num_sets == rec["num_sets"] and st.covered == rec["covered"]
    if o is not None:
        assert o.num_members == rec["members"]


@pytest.mark.parametrize("name", ["ic_wc_4k", "lt_4m", "ic_u1_256k", "ic_u01_1m"])
def test_plain_golden_ladders(name):
    p = graphgen.PLAIN[name]
    if not os.path.exists(os.path.join(HERE, name + ".json")):
        pytest.skip(f"{name}.json not written")
    rec = load(name)
    assert (rec["n"], rec["m"], rec["k"], rec["seed"]) == (p["n"], p["m"], p["k"], p["seed"])
    check_ladder(rec, p["n"], p["k"], p["epsilon"], p["ell"])
    assert rec["counts_sum"] == rec["members"]


def test_plain_golden_recomputed_small():
    w = graphgen.plain_workload("ic_wc_4k")
    g = w.graph
    rec = load("ic_wc_4k")
    o = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
    seeds, st = o.run(w.k, w.epsilon, w.ell, w.seed)
    same_as_run(rec, seeds, st, o)
    import hashlib
    assert hashlib.sha256(o.counts().astype("<u4").tobytes()).hexdigest() == rec["counts_sha256"]


def test_batch_golden():
    gold = load("batch64")
    assert len(gold["instances"]) == gold["count"] == 64
    b = graphgen.batch_workload(count=64, max_log_n=gold["max_log_n"])
    cheap = 0
    for i, (q, rec) in enumerate(zip(b.queries, gold["instances"])):
        g = b.graphs[q.graph_id]
        assert (g.n, g.m, q.k, q.epsilon.hex(), q.seed) == (rec["n"], rec["m"], rec["k"], rec["epsilon_hex"],
                                                              rec["seed"])
        check_ladder(rec, g.n, q.k, q.epsilon, q.ell)
        if rec["oracle_seconds"] < 0.3 and cheap < 6:
            cheap += 1
            o = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
            seeds, st = o.run(q.k, q.epsilon, q.ell, q.seed)
            same_as_run(rec, seeds, st, o)
    assert cheap >= 3


def test_served_golden():
    gold = load("served")
    qs = graphgen.served_queries()[: gold["queries"]]
    assert len(gold["results"]) == len(qs)
    ns = [r["n"] for r in gold["graphs"]]
    assert ns == [int(round(2.0 ** (16.0 + 4.0 * j / 7))) for j in range(8)]
    cheap = 0
    gs = None
    for q, rec in zip(qs, gold["results"]):
        assert (q.graph_id, q.k, q.epsilon.hex(), q.seed) == (rec["graph_id"], rec["k"], rec["epsilon_hex"],
                                                               rec["seed"])
        check_ladder(rec, ns[q.graph_id], q.k, q.epsilon, q.ell)
        if rec["oracle_seconds"] < 0.5 and q.graph_id <= 1 and cheap < 2:
            if gs is None:
                gs = graphgen.served_graphs(count=8)
            g = gs[q.graph_id]
            cheap += 1
            seeds, st = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model).run(q.k, q.epsilon, q.ell, q.seed)
            same_as_run(rec, seeds, st)
    assert cheap >= 1


def test_opim_golden_bounds_and_stop_rule():
    gold = load("opim")
    for rec in gold["runs"]:
        p = graphgen.PLAIN[rec["workload"]]
        prm = oracle.opim_params(p["n"], p["k"], p["epsilon"], p["ell"])
        assert rec["i_max"] == prm["i_max"] and rec["theta_max_hex"] == float(prm["theta_max"]).hex()
        t0 = math.ceil(prm["theta_0"])
        r = rec["rounds"]
        assert rec["sets_i"] == [t0 << i for i in range(r)]
        target = 1.0 - 1.0 / math.e - p["epsilon"]
        for i in range(r):
            up, low = oracle.opim_bounds(p["n"], p["k"], prm["a1"], prm["a2"], rec["sets_i"][i], rec["cov1_i"][i],
                                         rec["cov2_i"][i])
            assert (float(up).hex(), float(low).hex()) == (rec["upper_hex"][i], rec["lower_hex"][i])
            assert (low / up >= target) == (i == r - 1) or (i == r - 1 == rec["i_max"] - 1)
        assert len(rec["seeds"]) == p["k"] == len(set(rec["seeds"]))
