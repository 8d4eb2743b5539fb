"""The seeded input generator: R-MAT in transposed CSR, weights, workloads."""
import numpy as np

import graphgen


def test_rmat_shape_and_invariants():
    row, src = graphgen.rmat(4096, 32768, 1)
    assert row.dtype == np.uint64 and src.dtype == np.uint32
    assert row[0] == 0 and row[-1] == 32768 and np.all(np.diff(row.astype(np.int64)) >= 0)
    assert src.max() < 4096
    heads = np.repeat(np.arange(4096), np.diff(row.astype(np.int64)))
    assert not np.any(heads == src)                          # no self-loops
    keys = src.astype(np.uint64) << np.uint64(32) | heads.astype(np.uint64)
    assert len(np.unique(keys)) == 32768                      # duplicates merged
    for v in range(0, 4096, 97):                              # tails ascending per head
        part = src[row[v]:row[v + 1]]
        assert np.all(np.diff(part.astype(np.int64)) > 0)


def test_rmat_deterministic_and_seeded():
    a = graphgen.rmat(1000, 5000, 3)
    b = graphgen.rmat(1000, 5000, 3)
    c = graphgen.rmat(1000, 5000, 4)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])
    assert not np.array_equal(a[1], c[1])


def test_rmat_skew():
    # quadrant a = 0.57: low ids are hubs (in-degree of vertex 0 far above mean)
    row, src = graphgen.rmat(1 << 14, 1 << 18, 2)
    indeg = np.diff(row.astype(np.int64))
    assert indeg[0] > 20 * indeg.mean()


def test_weights():
    row, src = graphgen.rmat(512, 4096, 5)
    w = graphgen.weights_inv_indeg(row)
    indeg = np.diff(row.astype(np.int64))
    heads = np.repeat(np.arange(512), indeg)
    assert np.array_equal(w, (np.float32(1.0) / indeg[heads].astype(np.float32)))
    u = graphgen.weights_uniform(4096, 0.1, 5)
    assert u.dtype == np.float32 and u.min() >= 0 and u.max() < 0.1
    assert abs(u.mean() - 0.05) < 0.005


def test_workload_generators():
    qs = graphgen.served_queries(count=500)
    t = np.array([q.arrival_s for q in qs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(qs) / t[-1] - 200.0) < 40.0               # ~200 req/s
    assert all(10 <= q.k <= 200 and 0.1 <= q.epsilon <= 0.5 for q in qs)
    b = graphgen.batch_workload(count=6, max_log_n=12)
    assert len(b.graphs) == 6 and all(1024 <= g.n <= 4096 for g in b.graphs)
