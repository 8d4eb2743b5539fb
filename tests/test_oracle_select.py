"""Pins for the oracle's greedy selection (Alg. 2, Find_Most_Influential_Set):
hand-traced fixtures, a from-scratch recount greedy, and brute-force optimum
max coverage with the (1 - 1/e) guarantee."""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "greedy_hand_traced.txt")


def _cases():
    cases = []
    cur = None
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "case":
            cur = dict(name=tok[1], n=int(tok[2].split("=")[1]), k=int(tok[3].split("=")[1]), sets=[])
            cases.append(cur)
        elif tok[0] == "set":
            cur["sets"].append([int(x) for x in tok[1:]])
        elif tok[0] == "expect":
            kv = dict(t.split("=") for t in tok[1:])
            cur["seeds"] = [int(x) for x in kv["seeds"].split(",")]
            cur["covered"] = int(kv["covered"])
            cur["opt"] = int(kv["opt"])
    return cases


def to_arena(sets):
    off = np.zeros(len(sets) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(s) for s in sets])
    mem = np.array([x for s in sets for x in s], dtype=np.uint32)
    return off, mem


def brute_force_opt(n, sets, k):
    best = 0
    for S in itertools.combinations(range(n), k):
        Sset = set(S)
        best = max(best, sum(1 for s in sets if Sset & set(s)))
    return best


def recount_greedy(n, sets, k):
    """Greedy that recomputes every marginal gain from scratch each round."""
    picked = []
    alive = [set(s) for s in sets]
    covered = 0
    for _ in range(k):
        gains = [0] * n
        for s in alive:
            for v in s:
                gains[v] += 1
        best = None
        for v in range(n):
            if v in picked:
                continue
            if best is None or gains[v] > gains[best]:
                best = v
        picked.append(best)
        keep = [s for s in alive if best not in s]
        covered += len(alive) - len(keep)
        alive = keep
    return picked, covered


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_traced_fixtures(case):
    off, mem = to_arena(case["sets"])
    seeds, cov = oracle.select_sets(case["n"], off, mem, case["k"])
    assert seeds.tolist() == case["seeds"]
    assert cov == case["covered"]
    assert brute_force_opt(case["n"], case["sets"], case["k"]) == case["opt"]


@pytest.mark.parametrize("trial", range(12))
def test_random_set_systems_vs_recount_and_optimum(trial):
    rng = np.random.default_rng(100 + trial)
    n = int(rng.integers(4, 10))
    nsets = int(rng.integers(1, 30))
    sets = []
    for _ in range(nsets):
        size = int(rng.integers(1, n + 1))
        sets.append(sorted(rng.choice(n, size=size, replace=False).tolist()))
    k = int(rng.integers(1, min(n, 4) + 1))
    off, mem = to_arena(sets)
    seeds, cov = oracle.select_sets(n, off, mem, k)
    want_seeds, want_cov = recount_greedy(n, sets, k)
    assert seeds.tolist() == want_seeds
    assert cov == want_cov
    opt = brute_force_opt(n, sets, k)
    assert cov >= (1.0 - 1.0 / np.e) * opt - 1e-9
    assert cov <= opt


def test_k_equals_n_and_empty_system():
    seeds, cov = oracle.select_sets(4, np.zeros(1, dtype=np.uint64), np.zeros(0, dtype=np.uint32), 4)
    assert seeds.tolist() == [0, 1, 2, 3] and cov == 0
    with pytest.raises(ValueError):
        oracle.select_sets(4, np.zeros(1, dtype=np.uint64), np.zeros(0, dtype=np.uint32), 5)
    with pytest.raises(ValueError):
        oracle.select_sets(4, np.zeros(1, dtype=np.uint64), np.zeros(0, dtype=np.uint32), 0)
