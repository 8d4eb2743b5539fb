"""GPU path vs the oracle, element by element, through the C ABI.

Integer work is compared bit for bit: every RRR set (as a sorted member list
per set id), the per-vertex occurrence counts, the seed sequence, covered
counts, the theta ladder, LB and theta.  Sizes span several tiles, ragged
tails, the warp path, the CTA path (shared-memory and global bitmaps), the
LT long-walk path, staging overflow with resampling, and degenerate graphs."""
import numpy as np
import pytest

import graphgen
import oracle
from gpu_common import assert_same_stream, edges_to_graph, oracle_for

pytestmark = pytest.mark.gpu

IC, LT = graphgen.IC, graphgen.LT


@pytest.fixture(params=["cta", "group"])
def large_path(request, monkeypatch):
    """IC sets that outgrow a warp go one per CTA, or 64 at a time through the
    whole-GPU multi-source BFS; both must give the oracle's sets."""
    monkeypatch.setenv("IMM_IC_LARGE", request.param)
    return request.param


@pytest.fixture(scope="module")
def imm():
    import torch
    assert torch.cuda.is_available()
    from paper_2411_09473_gb300 import imm as mod
    return mod


def new_ctx(imm, g):
    ctx = imm.imm_create(device=0)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    return ctx


def check_stream(imm, ctx, g, theta, seed, o=None):
    imm.imm_sample(ctx, g.model, theta, seed)
    if o is None:
        o = oracle_for(g)
    o.sample(theta, seed)
    goff, gmem = imm.imm_get_sets(ctx, 0, theta)
    ooff, omem = o.arena()
    assert_same_stream(goff, gmem, ooff, omem)
    assert np.array_equal(imm.imm_get_counts(ctx, g.n), o.counts())
    return o


def rand_graph(n, m, seed, model, p=None):
    rng = np.random.default_rng(seed)
    edges = set()
    while len(edges) < m:
        u, v = (int(x) for x in rng.integers(0, n, 2))
        if u != v:
            edges.add((u, v))
    edges = sorted(edges)
    if model == IC:
        w = rng.uniform(0, 1, m) if p is None else np.full(m, p)
    else:
        indeg = np.bincount([v for (_, v) in edges], minlength=n)
        w = [0.9 / indeg[v] for (_, v) in edges]
    return edges_to_graph(n, edges, list(w), model)


# ---------------------------------------------------------------------------
# sampling
# ---------------------------------------------------------------------------

def test_ic_weighted_cascade_all_sets(imm):
    g = graphgen.plain_workload("ic_wc_4k").graph
    ctx = new_ctx(imm, g)
    check_stream(imm, ctx, g, 6000, 1)


def test_lt_rmat_all_sets(imm):
    g = graphgen.make_graph(4096, 32768, 3, LT, "inv_indeg")
    ctx = new_ctx(imm, g)
    check_stream(imm, ctx, g, 20000, 3)


@pytest.mark.parametrize("case", range(8))
def test_fuzz_small_graphs(imm, case):
    rng = np.random.default_rng(1000 + case)
    n = int(rng.integers(3, 700))
    m = int(rng.integers(0, min(n * (n - 1), 6 * n)))
    model = IC if case % 2 == 0 else LT
    g = rand_graph(n, m, case, model)
    ctx = new_ctx(imm, g)
    seed = int(rng.integers(0, 2**63))
    check_stream(imm, ctx, g, int(rng.integers(1, 3000)), seed)


@pytest.mark.parametrize("case", range(6))
def test_fuzz_ic_large_sets_both_paths(imm, large_path, case):
    # random IC graphs dense enough for many sets past the warp's 512
    # members: n not a multiple of 32, groups of a handful of sets, sets of
    # a few hundred members next to sets of most of the graph
    rng = np.random.default_rng(2000 + case)
    n = int(rng.integers(300, 3000))
    m = int(rng.integers(3 * n, 10 * n))
    g = rand_graph(n, m, 50 + case, IC)
    ctx = new_ctx(imm, g)
    seed = int(rng.integers(0, 2**63))
    check_stream(imm, ctx, g, int(rng.integers(200, 1500)), seed)


@pytest.mark.parametrize("n,m,gseed,pmax", [(3000, 24000, 11, 0.3), (1 << 14, 1 << 17, 12, 0.1),
                                            (5000, 20000, 13, 1.0)])
def test_ic_rmat_giant_sets(imm, large_path, n, m, gseed, pmax):
    # high edge probabilities: many sets outgrow a warp and go to the CTA path
    g = graphgen.make_graph(n, m, gseed, IC, "uniform", pmax=pmax)
    ctx = new_ctx(imm, g)
    o = check_stream(imm, ctx, g, 1500, gseed)
    # sets above n/32 members are stored as bitmaps: selection must see them
    for k in (1, 5, 40):
        seeds, cov = imm.imm_select(ctx, k)
        want, wcov = o.select(k)
        assert np.array_equal(seeds, want) and cov == wcov


def test_ic_p1_closures_and_star_hub(imm, large_path):
    # star: vertex 0 has 5000 in-neighbours, all with p = 1; every set rooted at 0
    # is the whole star (CTA path), the others are {leaf}
    n = 5001
    edges = [(i, 0) for i in range(1, n)]
    g = edges_to_graph(n, edges, [1.0] * (n - 1), IC)
    ctx = new_ctx(imm, g)
    check_stream(imm, ctx, g, 30000, 8)


def test_edgeless_and_p0_graphs(imm):
    n = 777
    g = graphgen.Graph(n=n, row=np.zeros(n + 1, dtype=np.uint64), src=np.zeros(0, dtype=np.uint32),
                       weight=np.zeros(0, dtype=np.float32), model=IC)
    ctx = new_ctx(imm, g)
    check_stream(imm, ctx, g, 2000, 5)
    g0 = rand_graph(300, 1500, 4, IC, p=0.0)
    ctx = new_ctx(imm, g0)
    check_stream(imm, ctx, g0, 1000, 6)
    gl = graphgen.Graph(n=n, row=np.zeros(n + 1, dtype=np.uint64), src=np.zeros(0, dtype=np.uint32),
                        weight=np.zeros(0, dtype=np.float32), model=LT)
    ctx = new_ctx(imm, gl)
    check_stream(imm, ctx, gl, 2000, 5)


def test_lt_long_walks(imm):
    # directed path and cycle with w = 1: walks far longer than the per-lane
    # path capacity take the long-walk path
    n = 3000
    path = edges_to_graph(n, [(i, i + 1) for i in range(n - 1)], [1.0] * (n - 1), LT)
    ctx = new_ctx(imm, path)
    check_stream(imm, ctx, path, 400, 2)
    cyc = edges_to_graph(1000, [(i, (i + 1) % 1000) for i in range(1000)], [1.0] * 1000, LT)
    ctx = new_ctx(imm, cyc)
    check_stream(imm, ctx, cyc, 300, 3)


def chain_graph(lengths, w_back1=0.7, w_back2=0.3):
    """Disjoint chains; position p of a chain has in-edges from p - 1
    (w_back1) and p - 2 (w_back2), so a reverse walk from p runs back to the
    chain's start with a random length of about p / 1.3 steps."""
    edges, w = [], []
    base = 0
    for L in lengths:
        for p in range(1, L):
            edges.append((base + p - 1, base + p))
            w.append(w_back1 if p > 1 else 1.0)
            if p > 1:
                edges.append((base + p - 2, base + p))
                w.append(w_back2)
        base += L
    return edges_to_graph(base, edges, w, LT)


def test_lt_walks_of_every_length(imm):
    # n = 42,000 (bitmaps of 1,313 words): walks up to 160 steps on the lane
    # path, up to 1,024 with per-walk tables, longer ones on the bitmap slots
    # (lists up to 1,313 members, bitmaps beyond)
    g = chain_graph([900, 1500, 1800] * 10)
    ctx = new_ctx(imm, g)
    o = check_stream(imm, ctx, g, 3000, 8)
    off, _ = imm.imm_get_sets(ctx, 0, 3000, members=False)
    lens = np.diff(off.astype(np.int64))
    assert (lens > 1024).any() and ((lens > 160) & (lens <= 1024)).sum() > 1000 and (lens > 1313).any()
    for k in (1, 20):
        s1, c1 = imm.imm_select(ctx, k)
        s2, c2 = o.select(k)
        assert np.array_equal(s1, s2) and c1 == c2


def test_lt_guide_layouts_and_misses(imm):
    """Heads of 65,535 and 70,000 in-edges (the two guide entry layouts, j
    relative or absolute), uneven weights with "none" mass (guide misses and
    threshold scans), and tails of in-degree 2..300 (degrees inside and past
    the 7-bit field of the absolute layout)."""
    rng = np.random.default_rng(12)
    H1, H2 = 0, 1                     # heads of 70,000 and 65,535 in-edges
    n = 72000
    edges, w = [], []
    for u in range(2, 70002):
        edges.append((u, H1))
    w += list(rng.uniform(0, 1, 70000) * (0.9 / 35000.0))       # ~0.9 in all, uneven
    for u in range(2, 65537):
        edges.append((u, H2))
    w += list(rng.uniform(0, 1, 65535) * (0.95 / 32767.5))
    for u in range(2, n):
        # every tail gets back to a head, and some have many in-edges
        extra = 300 if u % 97 == 0 else 0
        srcs = [H1, H2] + [int(x) for x in rng.integers(2, n, extra)]
        srcs = sorted(set(srcs) - {u})
        ww = rng.uniform(0.1, 1, len(srcs))
        ww = ww / ww.sum() * 0.97
        edges += [(t, u) for t in srcs]
        w += list(ww)
    g = edges_to_graph(n, edges, [float(x) for x in w], LT)
    ctx = new_ctx(imm, g)
    o = check_stream(imm, ctx, g, 4000, 13)
    for k in (1, 10):
        s1, c1 = imm.imm_select(ctx, k)
        s2, c2 = o.select(k)
        assert np.array_equal(s1, s2) and c1 == c2


def test_stream_extension_is_prefix_stable(imm, large_path):
    g = graphgen.make_graph(2048, 16384, 21, IC, "uniform", pmax=0.2)
    a = new_ctx(imm, g)
    imm.imm_sample(a, IC, 100, 9)
    imm.imm_sample(a, IC, 2500, 9)
    b = new_ctx(imm, g)
    imm.imm_sample(b, IC, 2500, 9)
    oa, ma = imm.imm_get_sets(a, 0, 2500)
    ob, mb = imm.imm_get_sets(b, 0, 2500)
    assert_same_stream(oa, ma, ob, mb)
    assert np.array_equal(imm.imm_get_counts(a, g.n), imm.imm_get_counts(b, g.n))


def test_ic_global_bitmap_path(imm, large_path):
    # n = 2^21: the n-bit visited bitmap no longer fits in shared memory, so the
    # CTA path keeps it in a per-CTA global slot; compare sampled set ids
    n, m = 1 << 21, 1 << 23
    g = graphgen.make_graph(n, m, 31, IC, "uniform", pmax=0.1)
    ctx = new_ctx(imm, g)
    theta = 1200
    imm.imm_sample(ctx, IC, theta, 31)
    off, mem = imm.imm_get_sets(ctx, 0, theta)
    sizes = np.diff(off.astype(np.int64))
    big = np.nonzero(sizes > 512)[0]
    assert len(big) > 10
    o = oracle_for(g)
    rng = np.random.default_rng(0)
    ids = list(big[:12]) + list(rng.choice(theta, 40, replace=False))
    for s in ids:
        want = o.sample_one(31, int(s))
        got = np.sort(mem[off[s]:off[s + 1]])
        assert np.array_equal(got, want), s


def test_ic_large_output_overflow_resamples(imm, large_path, monkeypatch):
    # an output buffer of three bitmaps: most large sets fail their
    # reservation and are resampled by later (smaller) batches; the stream
    # must still be the oracle's, set for set
    g = graphgen.make_graph(1 << 13, 1 << 16, 43, IC, "uniform", pmax=0.25)
    words = (g.n + 31) // 32
    monkeypatch.setenv("IMM_BIG_CAP_WORDS", str(3 * words))
    ctx = new_ctx(imm, g)
    check_stream(imm, ctx, g, 700, 43)
    off, _ = imm.imm_get_sets(ctx, 0, 700)
    assert (np.diff(off.astype(np.int64)) > 512).sum() > 50


def test_ic_group_ragged_groups_lists_and_bitmaps(imm, monkeypatch):
    monkeypatch.setenv("IMM_IC_LARGE", "group")
    # R-MAT with giant sets over several batches: groups of 64 and ragged
    # last groups
    g = graphgen.make_graph(1 << 13, 1 << 16, 41, IC, "uniform", pmax=0.25)
    ctx = new_ctx(imm, g)
    imm.imm_sample(ctx, IC, 300, 41)
    check_stream(imm, ctx, g, 2600, 41)
    off, _ = imm.imm_get_sets(ctx, 0, 2600)
    assert (np.diff(off.astype(np.int64)) > 512).sum() > 130
    # disjoint directed cycles with p = 1 in n = 2^15: a set rooted on a cycle
    # is the whole cycle (one BFS level per member), stored as a list below
    # n/32 = 1024 members and as a bitmap above; sparse random edges elsewhere
    n = 1 << 15
    lens = [300, 600, 900, 1500, 3000]
    edges, base = [], 0
    for ln in lens:
        edges += [(base + i, base + (i + 1) % ln) for i in range(ln)]
        base += ln
    weights = [1.0] * len(edges)
    rng = np.random.default_rng(5)
    extra = set()
    while len(extra) < 20000:
        u, v = (int(x) for x in rng.integers(base, n, 2))
        if u != v:
            extra.add((u, v))
    edges += sorted(extra)
    weights += list(rng.uniform(0, 0.3, len(extra)))
    cyc = edges_to_graph(n, edges, weights, IC)
    ctx = new_ctx(imm, cyc)
    check_stream(imm, ctx, cyc, 1500, 7)
    off, _ = imm.imm_get_sets(ctx, 0, 1500)
    sizes = set(np.diff(off.astype(np.int64)).tolist())
    assert set(lens) <= sizes


# ---------------------------------------------------------------------------
# selection and the IMM driver
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("model,k", [(IC, 10), (IC, 64), (LT, 25)])
def test_select_matches_oracle(imm, model, k):
    g = graphgen.make_graph(4096, 32768, 41, model, "inv_indeg")
    ctx = new_ctx(imm, g)
    o = check_stream(imm, ctx, g, 8000, 41)
    seeds, cov = imm.imm_select(ctx, k)
    want, wcov = o.select(k)
    assert np.array_equal(seeds, want) and cov == wcov


@pytest.mark.parametrize("mode", ["decrement", "rebuild"])
def test_select_decrement_equals_rebuild(imm, monkeypatch, mode):
    # the counter update of every round forced to one form (Sec. IV-C's
    # adaptive update only picks the cheaper of two that give the same
    # counts): seeds and coverage must be the oracle's either way, with
    # bitmap-stored giant sets (IC) and short list-stored walks (LT)
    monkeypatch.setenv("IMM_SELECT_MODE", mode)
    for g, theta, seed in ((graphgen.make_graph(1 << 13, 1 << 16, 61, IC, "uniform", pmax=0.25), 1200, 61),
                           (graphgen.make_graph(1 << 12, 1 << 15, 62, LT, "inv_indeg"), 3000, 62)):
        ctx = new_ctx(imm, g)
        o = check_stream(imm, ctx, g, theta, seed)
        for k in (1, 7, 60):
            seeds, cov = imm.imm_select(ctx, k)
            want, wcov = o.select(k)
            assert np.array_equal(seeds, want) and cov == wcov


def test_select_k_equals_n_and_empty_stream(imm):
    g = rand_graph(40, 120, 5, IC)
    ctx = new_ctx(imm, g)
    seeds, cov = imm.imm_select(ctx, 40)                 # no sets at all
    assert seeds.tolist() == list(range(40)) and cov == 0
    o = check_stream(imm, ctx, g, 500, 77)
    seeds, cov = imm.imm_select(ctx, 40)
    want, wcov = o.select(40)
    assert np.array_equal(seeds, want) and cov == wcov == 500


def check_run(imm, g, k, eps, ell, seed, fresh_final=False):
    ctx = new_ctx(imm, g)
    if fresh_final:
        seeds, st = imm.imm_run_ex(ctx, g.model, k, eps, ell, seed, imm.IMM_RUN_FRESH_FINAL)
    else:
        seeds, st = imm.imm_run(ctx, g.model, k, eps, ell, seed)
    o = oracle_for(g)
    want, ost = o.run(k, eps, ell, seed, fresh_final=fresh_final)
    assert np.array_equal(seeds, want)
    assert st.rounds == ost.rounds and st.stopped_early == ost.stopped_early
    for i in range(st.rounds):
        assert st.theta_i[i] == ost.theta_i[i]
        assert st.covered_i[i] == ost.covered_i[i]
        assert st.sets_i[i] == ost.sets_i[i]
    assert st.lb == ost.lb and st.theta == ost.theta
    assert st.num_sets == ost.num_sets and st.covered == ost.covered
    assert st.lambda_prime == ost.lambda_prime and st.lambda_star == ost.lambda_star
    assert np.array_equal(imm.imm_get_counts(ctx, g.n), o.counts())
    goff, gmem = imm.imm_get_sets(ctx, 0, st.num_sets)
    ooff, omem = o.arena()
    assert_same_stream(goff, gmem, ooff, omem)
    return st


def test_run_ic_weighted_cascade_4k(imm):
    w = graphgen.plain_workload("ic_wc_4k")
    check_run(imm, w.graph, w.k, w.epsilon, w.ell, w.seed)


@pytest.mark.parametrize("model", [IC, LT])
def test_run_fresh_final_stream(imm, model):
    # the final selection on exactly theta fresh sets under the second key
    g = graphgen.make_graph(3000, 30000, 17, model, "inv_indeg")
    st = check_run(imm, g, 8, 0.4, 1.0, 17, fresh_final=True)
    assert st.num_sets == st.theta
    ctx = new_ctx(imm, g)
    with pytest.raises(imm.ImmError):
        imm.imm_run_ex(ctx, g.model, 8, 0.4, 1.0, 17, 2)


def test_run_lt_small(imm):
    g = graphgen.make_graph(8192, 65536, 7, LT, "inv_indeg")
    check_run(imm, g, 20, 0.3, 1.0, 7)


def test_run_ic_uniform_small(imm):
    g = graphgen.make_graph(3000, 30000, 8, IC, "uniform", pmax=0.1)
    check_run(imm, g, 7, 0.4, 1.0, 8)


def test_run_no_early_stop(imm):
    n = 64
    g = graphgen.Graph(n=n, row=np.zeros(n + 1, dtype=np.uint64), src=np.zeros(0, dtype=np.uint32),
                       weight=np.zeros(0, dtype=np.float32), model=IC)
    st = check_run(imm, g, 2, 0.5, 1.0, 3)
    assert st.stopped_early == 0 and st.lb == 1.0


# ---------------------------------------------------------------------------
# errors leave the context usable
# ---------------------------------------------------------------------------

def test_errors(imm):
    g = graphgen.make_graph(1024, 8192, 2, IC, "inv_indeg")
    ctx = new_ctx(imm, g)
    with pytest.raises(imm.ImmError) as e:
        imm.imm_sample(ctx, LT, 10, 1)
    assert e.value.code == imm.IMM_EINVAL
    imm.imm_sample(ctx, IC, 10, 1)
    with pytest.raises(imm.ImmError) as e:
        imm.imm_sample(ctx, IC, 20, 2)                # other seed, same stream
    assert e.value.code == imm.IMM_ESTATE
    with pytest.raises(imm.ImmError) as e:
        imm.imm_select(ctx, 0)
    assert e.value.code == imm.IMM_EINVAL
    with pytest.raises(imm.ImmError) as e:
        imm.imm_select(ctx, 1025)
    assert e.value.code == imm.IMM_EINVAL
    bad = g.src.copy()
    bad[5] = 5000
    with pytest.raises(imm.ImmError) as e:
        imm.imm_load_graph(ctx, g.n, g.m, g.row, bad, g.weight, IC)
    assert e.value.code == imm.IMM_EINVAL
    w = g.weight.copy()
    w[0] = np.float32("nan")
    with pytest.raises(imm.ImmError):
        imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, w, IC)
    lt_over = graphgen.make_graph(1024, 8192, 2, LT, "inv_indeg")
    w2 = lt_over.weight * np.float32(1.5)
    with pytest.raises(imm.ImmError):
        imm.imm_load_graph(ctx, g.n, g.m, lt_over.row, lt_over.src, np.minimum(w2, 1), LT)
    # context still usable after the errors
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, IC)
    o = check_stream(imm, ctx, g, 300, 4)
    assert o.num_sets == 300


def test_arena_limit_enomem_then_recovers(imm):
    g = graphgen.make_graph(4096, 32768, 5, IC, "uniform", pmax=0.5)
    ctx = new_ctx(imm, g)
    imm.imm_set_arena_limit(ctx, 1 << 16)
    with pytest.raises(imm.ImmError) as e:
        imm.imm_sample(ctx, IC, 5000, 5)
    assert e.value.code == imm.IMM_ENOMEM
    imm.imm_set_arena_limit(ctx, 0)
    imm.imm_reset_sets(ctx)
    check_stream(imm, ctx, g, 2000, 5)


@pytest.mark.parametrize("seed", [1, 2])
def test_lt_uneven_weights_and_none_mass(imm, seed):
    # per-head weights drawn unevenly, summing to U(0.3, 1.0): exercises the
    # walker's threshold search on ragged cumulative thresholds and on "none"
    rng = np.random.default_rng(50 + seed)
    g0 = graphgen.make_graph(3000, 40000, 60 + seed, LT, "inv_indeg")
    w = np.zeros(g0.m, dtype=np.float32)
    for v in range(g0.n):
        lo, hi = int(g0.row[v]), int(g0.row[v + 1])
        if hi > lo:
            x = rng.exponential(1.0, hi - lo)
            w[lo:hi] = (x / x.sum() * rng.uniform(0.3, 1.0)).astype(np.float32) * np.float32(0.999)
    g = graphgen.Graph(n=g0.n, row=g0.row, src=g0.src, weight=w, model=LT)
    ctx = new_ctx(imm, g)
    o = check_stream(imm, ctx, g, 20000, seed)
    seeds, cov = imm.imm_select(ctx, 30)
    want, wcov = o.select(30)
    assert np.array_equal(seeds, want) and cov == wcov
