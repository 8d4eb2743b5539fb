"""Helpers shared by the GPU parity tests (not collected as tests)."""
import numpy as np

import graphgen
import oracle


def canonical_sets(off, mem):
    """Per-set sorted member lists as a flat array (set order kept)."""
    off = off.astype(np.int64)
    out = mem.copy()
    sizes = np.diff(off)
    set_of = np.repeat(np.arange(len(sizes)), sizes)
    order = np.lexsort((mem, set_of))
    out = mem[order]
    return off, out


def assert_same_stream(gpu_off, gpu_mem, orc_off, orc_mem):
    assert np.array_equal(gpu_off.astype(np.int64), orc_off.astype(np.int64)), "set sizes differ"
    _, a = canonical_sets(gpu_off, gpu_mem)
    _, b = canonical_sets(orc_off, orc_mem)
    if not np.array_equal(a, b):
        off = gpu_off.astype(np.int64)
        bad = np.nonzero(a != b)[0][0]
        s = int(np.searchsorted(off, bad, side="right") - 1)
        raise AssertionError(f"first differing set id {s}")


def edges_to_graph(n, edges, weights, model):
    order = sorted(range(len(edges)), key=lambda i: (edges[i][1], edges[i][0]))
    row = np.zeros(n + 1, dtype=np.uint64)
    for (u, v) in edges:
        row[v + 1] += 1
    row = np.cumsum(row).astype(np.uint64)
    src = np.array([edges[i][0] for i in order], dtype=np.uint32)
    w = np.array([weights[i] for i in order], dtype=np.float32)
    return graphgen.Graph(n=n, row=row, src=src, weight=w, model=model)


def oracle_for(g):
    return oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)


def load_golden(name):
    """Stored oracle results written by tests/golden/make_golden.py."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name + ".json")) as f:
        return json.load(f)


def graph_digest(g) -> str:
    import hashlib
    h = hashlib.sha256()
    for a in (g.row.astype("<u8"), g.src.astype("<u4"), g.weight.astype("<f4")):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def counts_digest(cnt) -> str:
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(np.asarray(cnt).astype("<u4")).tobytes()).hexdigest()


def assert_run_equals_golden(seeds, st, rec, what=""):
    """Every field of one IMM run (Alg. 1) against the oracle's stored run:
    seeds in pick order, the theta ladder with per-round coverage, LB, theta,
    stream size, coverage, total members, lambda' and lambda* (bit for bit)."""
    assert [int(x) for x in seeds] == rec["seeds"], what
    assert st.rounds == rec["rounds"] and st.stopped_early == rec["stopped_early"], what
    r = st.rounds
    assert [int(st.theta_i[i]) for i in range(r)] == rec["theta_i"], what
    assert [int(st.covered_i[i]) for i in range(r)] == rec["covered_i"], what
    assert [int(st.sets_i[i]) for i in range(r)] == rec["sets_i"], what
    assert float(st.lb).hex() == rec["lb_hex"], what
    assert st.theta == rec["theta"] and st.num_sets == rec["num_sets"], what
    assert st.covered == rec["covered"] and st.members == rec["members"], what
    assert float(st.lambda_prime).hex() == rec["lambda_prime_hex"], what
    assert float(st.lambda_star).hex() == rec["lambda_star_hex"], what
