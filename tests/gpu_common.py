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
