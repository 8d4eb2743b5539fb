"""Pins for the oracle's OPIM-style early stop (Sec. VI cites OPIM, Tang et
al. SIGMOD 2018; the oracle follows its OPIM-C procedure).

The bounds are pinned against the truth they bound: on a 6-vertex graph the
spread of every seed set is computed exactly by enumerating live-edge worlds,
so the lower bound must stay below the exact spread and the upper bound above
the exact optimum over many independent RR collections, and both must come
close to the truth when the collections are large.  theta_max is pinned to
Tang et al.'s lambda* (the oracle's already pinned IMM bound) at the same
confidence, divided by k."""
import itertools
import math

import numpy as np
import pytest

import graphgen
import oracle
from test_oracle_sampling import TINY_EDGES, TINY_P, csr_from_edges, exact_sigma_ic

N = 6


@pytest.fixture(scope="module")
def tiny():
    row, src, w = csr_from_edges(N, TINY_EDGES, TINY_P)
    o = oracle.Oracle(N, row, src, w, oracle.IC)
    thr = o.thresholds()
    sig = {}
    for r in (1, 2):
        for S in itertools.combinations(range(N), r):
            sig[S] = exact_sigma_ic(N, row, src, thr, list(S))
    return row, src, w, sig


def hits(off, mem, S):
    """Sets of the collection that contain a member of S."""
    inS = np.zeros(N, dtype=bool)
    inS[list(S)] = True
    flag = inS[mem.astype(np.int64)].astype(np.int64)
    c = np.concatenate([[0], np.cumsum(flag)])
    off = off.astype(np.int64)
    return int(np.count_nonzero(c[off[1:]] - c[off[:-1]]))


def test_theta_max_is_lambda_star_over_k():
    for (n, k, eps, ell) in [(4096, 10, 0.5, 1.0), (1 << 20, 50, 0.13, 1.0), (262144, 7, 0.3, 2.0)]:
        op = oracle.opim_params(n, k, eps, ell)
        # Tang et al.'s lambda* uses ell' ln n + ln 2 where OPIM uses ln(6 / delta),
        # delta = n^-ell: pick the IMM ell whose ell' gives the same confidence term
        ln_n = math.log(n)
        ell_imm = (math.log(3.0) + ell * ln_n) / (ln_n + math.log(2.0))
        lam = oracle.theta_params(n, k, eps, ell_imm)["lambda_star"]
        assert abs(op["theta_max"] * k / lam - 1.0) < 1e-12
        assert abs(op["theta_0"] * n / (eps * eps * k) / op["theta_max"] - 1.0) < 1e-12
        assert op["i_max"] == max(1, math.ceil(math.log2(n / (eps * eps * k))))
        assert abs(op["a1"] - op["a2"] - op["lnC"]) < 1e-9
        assert abs(math.exp(-op["a2"]) * 3 * op["i_max"] / op["delta"] - 1.0) < 1e-9


@pytest.mark.parametrize("S", [(0,), (3,), (1, 4), (2, 5)])
def test_lower_bound_holds_and_is_tight(tiny, S):
    row, src, w, sig = tiny
    k = len(S)
    prm = oracle.opim_params(N, k, 0.5, 3.0)
    o = oracle.Oracle(N, row, src, w, oracle.IC)
    for theta, trials in ((300, 150), (20000, 3)):
        lows = []
        for t in range(trials):
            o.reset()
            o.sample(theta, 1000 + t)
            off, mem = o.arena()
            _, low = oracle.opim_bounds(N, k, prm["a1"], prm["a2"], theta, 0, hits(off, mem, S))
            lows.append(low)
        assert max(lows) <= sig[S], (max(lows), sig[S])
        if theta == 20000:
            assert min(lows) >= 0.9 * sig[S], (min(lows), sig[S])


@pytest.mark.parametrize("k", [1, 2])
def test_upper_bound_holds_and_is_tight(tiny, k):
    row, src, w, sig = tiny
    opt = max(v for S, v in sig.items() if len(S) == k)
    prm = oracle.opim_params(N, k, 0.5, 3.0)
    o = oracle.Oracle(N, row, src, w, oracle.IC)
    ratio = 1.0 - (1.0 - 1.0 / k) ** k
    for theta, trials in ((300, 150), (20000, 3)):
        ups = []
        for t in range(trials):
            o.reset()
            o.sample(theta, 5000 + t)
            _, cov1 = o.select(k)
            up, _ = oracle.opim_bounds(N, k, prm["a1"], prm["a2"], theta, cov1, 0)
            ups.append(up)
        assert min(ups) >= opt, (min(ups), opt)
        if theta == 20000:
            assert max(ups) <= 1.15 * opt / ratio, (max(ups), opt)


def test_run_collections_and_stop_rule():
    w = graphgen.plain_workload("ic_wc_4k")
    g = w.graph
    for (k, eps, seed) in [(10, 0.5, 1), (5, 0.2, 9), (20, 0.3, 4)]:
        o = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
        seeds, st = o.opim_run(k, eps, 1.0, seed)
        prm = oracle.opim_params(g.n, k, eps, 1.0)
        assert st.i_max == prm["i_max"] and st.theta_max == prm["theta_max"]
        r = st.rounds
        t0 = math.ceil(prm["theta_0"])
        assert [st.sets_i[i] for i in range(r)] == [t0 << i for i in range(r)]
        theta = st.sets_i[r - 1]
        # R1: the plain stream under the seed, and the greedy over it
        off, mem = o.arena()
        ref = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
        ref.sample(theta, seed)
        roff, rmem = ref.arena()
        assert np.array_equal(off, roff) and np.array_equal(mem, rmem)
        gs, gcov = oracle.select_sets(g.n, off, mem, k)
        assert np.array_equal(gs, seeds) and gcov == st.cov1_i[r - 1]
        # R2: an independent stream under seed ^ OPIM_KEY
        ref2 = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
        ref2.sample(theta, seed ^ oracle.OPIM_KEY)
        off2, mem2 = ref2.arena()
        inS = np.zeros(g.n, dtype=bool)
        inS[seeds] = True
        flag = np.concatenate([[0], np.cumsum(inS[mem2.astype(np.int64)])])
        o2 = off2.astype(np.int64)
        assert int(np.count_nonzero(flag[o2[1:]] - flag[o2[:-1]])) == st.cov2_i[r - 1]
        up, low = oracle.opim_bounds(g.n, k, prm["a1"], prm["a2"], theta, st.cov1_i[r - 1], st.cov2_i[r - 1])
        assert (up, low) == (st.upper_i[r - 1], st.lower_i[r - 1]) and st.alpha == low / up
        target = 1.0 - 1.0 / math.e - eps
        for i in range(r - 1):
            assert st.lower_i[i] / st.upper_i[i] < target
        assert st.alpha >= target or r == st.i_max
        assert st.stopped_early == (1 if r < st.i_max else 0)


def test_run_meets_its_guarantee_on_exact_spreads(tiny):
    row, src, w, sig = tiny
    for k in (1, 2):
        opt = max(v for S, v in sig.items() if len(S) == k)
        for seed in range(6):
            o = oracle.Oracle(N, row, src, w, oracle.IC)
            seeds, st = o.opim_run(k, 0.3, 3.0, 40 + seed)
            S = tuple(sorted(int(x) for x in seeds))
            assert sig[S] >= (1.0 - 1.0 / math.e - 0.3) * opt
            # the reported bounds bracket the truth
            assert st.lower_i[st.rounds - 1] <= sig[S] and st.upper_i[st.rounds - 1] >= opt


def test_upper_bound_covers_a_suboptimal_greedy():
    """Max coverage where the greedy is not optimal: vertex 2 occurs in most
    RR sets, so the greedy takes it first and covers 5 of 6 sets with k = 2,
    while {0, 1} covers all 6.  With no sampling slack (a1 = 0) the upper
    bound on the optimum must still be at least the optimum's coverage."""
    sets = [[0, 2], [0, 2], [1, 2], [1, 2], [0], [1]]
    off = np.array([0] + list(np.cumsum([len(s) for s in sets])), dtype=np.uint64)
    mem = np.array([v for s in sets for v in s], dtype=np.uint32)
    seeds, cov = oracle.select_sets(3, off, mem, 2)
    assert seeds[0] == 2 and cov == 5
    up, _ = oracle.opim_bounds(3, 2, 0.0, 1.0, len(sets), cov, 0)
    assert up >= 3.0 * 6 / len(sets)
