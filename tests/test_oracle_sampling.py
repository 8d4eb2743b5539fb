"""Pins for the oracle's RRR-set sampling (Alg. 3; IC and LT of Sec. II-A).

The strongest pin is the RIS identity of Reverse Influence Sampling: for any
seed set S, n * Pr[S hits a random RRR set] equals the expected spread
sigma(S).  On tiny graphs sigma(S) is computed exactly by enumerating every
live-edge world, independently of the sampler."""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

import oracle

Q = float(1 << 24)


def csr_from_edges(n, edges, weights):
    """Transposed CSR (grouped by head v, tails ascending) + weights in that order."""
    order = sorted(range(len(edges)), key=lambda i: (edges[i][1], edges[i][0]))
    row = np.zeros(n + 1, dtype=np.uint64)
    for (u, v) in edges:
        row[v + 1] += 1
    row = np.cumsum(row).astype(np.uint64)
    src = np.array([edges[i][0] for i in order], dtype=np.uint32)
    w = np.array([weights[i] for i in order], dtype=np.float32)
    return row, src, w


def forward_reach(n, live_edges, S):
    adj = [[] for _ in range(n)]
    for (u, v) in live_edges:
        adj[u].append(v)
    seen = set(S)
    stack = list(S)
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return len(seen)


def exact_sigma_ic(n, row, src, thr, S):
    """Sum over all 2^m worlds of P(world) * |reach of S| (edge live w.p. thr/2^24)."""
    m = len(src)
    heads = np.repeat(np.arange(n), np.diff(row.astype(np.int64)))
    p = [t / Q for t in thr]
    total = 0.0
    for mask in range(1 << m):
        pr = 1.0
        live = []
        for e in range(m):
            if mask >> e & 1:
                pr *= p[e]
                live.append((int(src[e]), int(heads[e])))
            else:
                pr *= 1.0 - p[e]
        if pr:
            total += pr * forward_reach(n, live, S)
    return total


def exact_sigma_lt(n, row, src, cthr, S):
    """LT as live-edge worlds (Kempe et al.): each head keeps at most one in-edge,
    edge j w.p. (cthr_j - cthr_{j-1}) / 2^24, none with the remaining mass."""
    choices = []
    for v in range(n):
        lo, hi = int(row[v]), int(row[v + 1])
        opts = []
        prev = 0
        for e in range(lo, hi):
            opts.append(((int(src[e]), v), (int(cthr[e]) - prev) / Q))
            prev = int(cthr[e])
        opts.append((None, (Q - prev) / Q))
        choices.append(opts)
    total = 0.0
    for combo in itertools.product(*choices):
        pr = 1.0
        live = []
        for (edge, q) in combo:
            pr *= q
            if edge is not None:
                live.append(edge)
        if pr:
            total += pr * forward_reach(n, live, S)
    return total


def hit_fraction(off, mem, S):
    S = set(S)
    hits = 0
    for s in range(len(off) - 1):
        if any(int(x) in S for x in mem[off[s]:off[s + 1]]):
            hits += 1
    return hits / (len(off) - 1)


TINY_EDGES = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 3), (1, 4), (0, 5), (4, 1)]
TINY_P = [0.6, 0.35, 0.8, 0.5, 0.25, 0.9, 0.4, 0.7, 0.15, 0.55]


@pytest.mark.parametrize("S", [[0], [3], [1, 4], [5], [2, 3]])
def test_ris_identity_ic_exact_enumeration(S):
    n = 6
    row, src, w = csr_from_edges(n, TINY_EDGES, TINY_P)
    o = oracle.Oracle(n, row, src, w, oracle.IC)
    thr = o.thresholds()
    sigma = exact_sigma_ic(n, row, src, thr, S)
    theta = 60000
    o.sample(theta, seed=77)
    off, mem = o.arena()
    f = hit_fraction(off, mem, S)
    se = n * math.sqrt(max(f * (1 - f), 1e-12) / theta)
    assert abs(n * f - sigma) <= 5 * se, (n * f, sigma, se)


def lt_weights(n, edges):
    # each head splits 0.85 of its mass over its in-edges (0.15 left for "none")
    indeg = [0] * n
    for (_, v) in edges:
        indeg[v] += 1
    return [0.85 / indeg[v] for (_, v) in edges]


@pytest.mark.parametrize("S", [[0], [3], [1, 4], [2, 5]])
def test_ris_identity_lt_exact_enumeration(S):
    n = 6
    w_in = lt_weights(n, TINY_EDGES)
    row, src, w = csr_from_edges(n, TINY_EDGES, w_in)
    o = oracle.Oracle(n, row, src, w, oracle.LT)
    cthr = o.thresholds()
    sigma = exact_sigma_lt(n, row, src, cthr, S)
    theta = 60000
    o.sample(theta, seed=91)
    off, mem = o.arena()
    f = hit_fraction(off, mem, S)
    se = n * math.sqrt(max(f * (1 - f), 1e-12) / theta)
    assert abs(n * f - sigma) <= 5 * se, (n * f, sigma, se)


def random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    edges = set()
    while len(edges) < m:
        u, v = rng.integers(0, n, 2)
        if u != v:
            edges.add((int(u), int(v)))
    return sorted(edges)


def test_p1_sets_are_reverse_reachable_closures():
    # p = 1 on every edge: each RRR set is exactly the set of vertices that can
    # reach the root (textbook reverse BFS, scipy's breadth_first_order on G^T)
    n, m = 300, 700
    edges = random_graph(n, m, 1)
    row, src, w = csr_from_edges(n, edges, [1.0] * m)
    o = oracle.Oracle(n, row, src, w, oracle.IC)
    o.sample(200, seed=5)
    gt = sp.csr_matrix((np.ones(m), ([v for (_, v) in edges], [u for (u, _) in edges])), shape=(n, n))
    for s in range(200):
        got = o.get_set(s)
        r = oracle.root(5, s, n)
        want = np.sort(csgraph.breadth_first_order(gt, r, directed=True, return_predecessors=False))
        assert np.array_equal(got, want)


def test_p0_sets_are_singleton_roots():
    n, m = 50, 200
    edges = random_graph(n, m, 2)
    row, src, w = csr_from_edges(n, edges, [0.0] * m)
    o = oracle.Oracle(n, row, src, w, oracle.IC)
    o.sample(500, seed=3)
    off, mem = o.arena()
    assert np.all(np.diff(off.astype(np.int64)) == 1)
    roots = np.array([oracle.root(3, s, n) for s in range(500)])
    assert np.array_equal(mem, roots)
    assert np.array_equal(o.counts(), np.bincount(roots, minlength=n).astype(np.uint32))


def test_ic_sets_equal_live_edge_closures():
    # every member reaches the root through live edges, and every vertex that
    # does is a member: recompute the closure from the coins alone
    n, m = 80, 400
    edges = random_graph(n, m, 3)
    rng = np.random.default_rng(4)
    ps = rng.uniform(0.05, 0.6, m).tolist()
    row, src, w = csr_from_edges(n, edges, ps)
    o = oracle.Oracle(n, row, src, w, oracle.IC)
    thr = o.thresholds()
    seed = 1234567890123
    o.sample(300, seed=seed)
    for s in range(300):
        r = oracle.root(seed, s, n)
        seen = {r}
        stack = [r]
        while stack:
            v = stack.pop()
            for e in range(int(row[v]), int(row[v + 1])):
                u = int(src[e])
                if u not in seen and oracle.ic_live(seed, s, e, int(thr[e])):
                    seen.add(u)
                    stack.append(u)
        assert np.array_equal(o.get_set(s), np.array(sorted(seen), dtype=np.uint32))


def test_counts_equal_occurrences():
    # Alg. 3 lines after the BFS: counter[v] = number of sets containing v
    n, m = 120, 600
    edges = random_graph(n, m, 5)
    row, src, w = csr_from_edges(n, edges, [0.2] * m)
    o = oracle.Oracle(n, row, src, w, oracle.IC)
    o.sample(1000, seed=8)
    off, mem = o.arena()
    assert np.array_equal(o.counts(), np.bincount(mem, minlength=n).astype(np.uint32))
    # members of a set are distinct and the root comes first
    for s in range(1000):
        part = mem[off[s]:off[s + 1]]
        assert len(set(part.tolist())) == len(part)
        assert part[0] == oracle.root(8, s, n)


def test_lt_directed_cycle_covers_everything():
    # w = 1 on a directed cycle: each vertex keeps its only in-edge, the walk
    # goes all the way round and stops at the root
    n = 37
    edges = [(i, (i + 1) % n) for i in range(n)]
    row, src, w = csr_from_edges(n, edges, [1.0] * n)
    o = oracle.Oracle(n, row, src, w, oracle.LT)
    o.sample(50, seed=2)
    for s in range(50):
        assert np.array_equal(o.get_set(s), np.arange(n, dtype=np.uint32))


def test_lt_directed_path_closed_form():
    # path 0 -> 1 -> ... -> n-1 with w = 1: the set of root r is {0..r}
    n = 41
    edges = [(i, i + 1) for i in range(n - 1)]
    row, src, w = csr_from_edges(n, edges, [1.0] * (n - 1))
    o = oracle.Oracle(n, row, src, w, oracle.LT)
    o.sample(60, seed=6)
    for s in range(60):
        r = oracle.root(6, s, n)
        assert np.array_equal(o.get_set(s), np.arange(r + 1, dtype=np.uint32))


def test_lt_pick_frequencies_match_weights():
    # a head with in-weights (0.2, 0.3, 0.1) and 0.4 for "none": the walk's first
    # step from it lands on each tail with the weight's probability
    n = 4
    edges = [(1, 0), (2, 0), (3, 0)]
    row, src, w = csr_from_edges(n, edges, [0.2, 0.3, 0.1])
    o = oracle.Oracle(n, row, src, w, oracle.LT)
    o.sample(80000, seed=12)
    off, mem = o.arena()
    tally = np.zeros(4)
    rooted = 0
    for s in range(len(off) - 1):
        part = mem[off[s]:off[s + 1]]
        if part[0] != 0:
            continue
        rooted += 1
        tally[part[1] if len(part) > 1 else 0] += 1
    probs = np.array([0.4, 0.2, 0.3, 0.1])
    for j in range(4):
        sd = math.sqrt(rooted * probs[j] * (1 - probs[j]))
        assert abs(tally[j] - rooted * probs[j]) < 5 * sd


def test_lt_rejects_overweight_heads():
    n = 3
    edges = [(1, 0), (2, 0)]
    row, src, w = csr_from_edges(n, edges, [0.7, 0.5])
    with pytest.raises(ValueError):
        oracle.Oracle(n, row, src, w, oracle.LT)


def test_invalid_graphs_rejected():
    n = 4
    edges = [(1, 0), (2, 0)]
    row, src, w = csr_from_edges(n, edges, [0.5, 0.5])
    bad_src = src.copy()
    bad_src[0] = 9
    with pytest.raises(ValueError):
        oracle.Oracle(n, row, bad_src, w, oracle.IC)
    bad_w = w.copy()
    bad_w[1] = np.float32("nan")
    with pytest.raises(ValueError):
        oracle.Oracle(n, row, src, bad_w, oracle.IC)
    bad_row = row.copy()
    bad_row[1], bad_row[2] = 2, 1
    with pytest.raises(ValueError):
        oracle.Oracle(n, bad_row, src, w, oracle.IC)


def test_stream_extension_is_prefix_stable():
    # Alg. 1 appends to the existing RRRsets: sampling to theta1 then theta2
    # gives the same sets as sampling to theta2 at once
    n, m = 100, 500
    edges = random_graph(n, m, 9)
    row, src, w = csr_from_edges(n, edges, [0.3] * m)
    a = oracle.Oracle(n, row, src, w, oracle.IC)
    a.sample(100, seed=4)
    a.sample(250, seed=4)
    b = oracle.Oracle(n, row, src, w, oracle.IC)
    b.sample(250, seed=4)
    oa, ma = a.arena()
    ob, mb = b.arena()
    assert np.array_equal(oa, ob) and np.array_equal(ma, mb)
    assert np.array_equal(a.counts(), b.counts())
