"""imm_select_noalloc: selection for callers that cannot allocate device memory
(a plugin inside a framework whose pool owns the GPU, a service with a fixed
footprint).  Its output must equal imm_select's and the oracle's greedy on the
same sets, call after call, although every call reuses the same fixed scratch
array."""
import numpy as np
import pytest

import graphgen
import oracle


def _sets_on_device(imm, ctx, theta):
    import torch
    off, mem = imm.imm_get_sets(ctx, 0, theta)
    d_off = torch.from_numpy(off.astype(np.int64)).cuda()
    d_mem = torch.from_numpy(mem.astype(np.int32)).cuda()
    return off, mem, d_off, d_mem


@pytest.mark.gpu
def test_noalloc_selection_matches_imm_select_twice():
    import torch
    from paper_2411_09473_gb300 import imm

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    cases = [
        (graphgen.make_graph(4096, 32768, 1, graphgen.IC, "inv_indeg"), 4000, 1, 10),
        (graphgen.make_graph(3000, 24000, 11, graphgen.IC, "uniform", pmax=0.3), 1500, 11, 25),
    ]
    for g, theta, seed, k in cases:
        ctx = imm.imm_create(device=0)
        imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
        imm.imm_sample(ctx, g.model, theta, seed)
        want, wcov = imm.imm_select(ctx, k)
        off, mem, d_off, d_mem = _sets_on_device(imm, ctx, theta)
        oseeds, ocov = oracle.select_sets(g.n, off, mem, k)
        assert np.array_equal(oseeds, want) and ocov == wcov
        for _ in range(2):  # the second call sees the first call's leftovers
            d_seeds = torch.full((k,), -1, dtype=torch.int32, device="cuda")
            d_cov = torch.zeros(1, dtype=torch.int64, device="cuda")
            imm.imm_select_noalloc(g.n, theta, d_off, d_mem, k, d_seeds, d_cov)
            torch.cuda.synchronize()
            assert np.array_equal(d_seeds.cpu().numpy().astype(np.uint32), want)
            assert int(d_cov.item()) == wcov
        imm.imm_destroy(ctx)


@pytest.mark.gpu
def test_noalloc_picks_past_full_coverage_on_a_side_stream():
    """k larger than the number of vertices that occur in any set: once every
    set is covered all counts are 0, and the picks continue with the lowest
    unpicked ids (the tie rule of the selection).  One call runs on a new
    stream without a covered output."""
    import torch
    from paper_2411_09473_gb300 import imm

    torch.cuda.set_device(0)
    # p = 1 on a sparse graph: each set is its root's reverse closure, and
    # few vertices occur in any set
    n = 64
    edges = [(i + 1, i) for i in range(0, 20)] + [(40, 41), (42, 41), (50, 51)]
    row = np.zeros(n + 1, dtype=np.uint64)
    for (_, v) in edges:
        row[v + 1] += 1
    row = np.cumsum(row).astype(np.uint64)
    src = np.array([u for (u, v) in sorted(edges, key=lambda e: (e[1], e[0]))], dtype=np.uint32)
    w = np.ones(len(src), dtype=np.float32)
    ctx = imm.imm_create(device=0)
    imm.imm_load_graph(ctx, n, len(src), row, src, w, graphgen.IC)
    theta, k = 40, n
    imm.imm_sample(ctx, graphgen.IC, theta, 7)
    want, wcov = imm.imm_select(ctx, k)
    off, mem, d_off, d_mem = _sets_on_device(imm, ctx, theta)
    assert len(np.unique(mem)) < k
    oseeds, ocov = oracle.select_sets(n, off, mem, k)
    assert np.array_equal(oseeds, want) and ocov == wcov == theta
    side = torch.cuda.Stream()
    for covered in (True, False):
        d_seeds = torch.full((k,), -1, dtype=torch.int32, device="cuda")
        d_cov = torch.zeros(1, dtype=torch.int64, device="cuda") if covered else None
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            imm.imm_select_noalloc(n, theta, d_off, d_mem, k, d_seeds, d_cov, stream=side)
        side.synchronize()
        assert np.array_equal(d_seeds.cpu().numpy().astype(np.uint32), want)
        if covered:
            assert int(d_cov.item()) == theta
    imm.imm_destroy(ctx)


@pytest.mark.gpu
def test_noalloc_member_id_out_of_range_gives_the_error_pattern():
    """A member id >= n is skipped by the kernels (never used as an index) and
    the outputs carry the documented error pattern; the next valid call is
    unaffected."""
    import torch
    from paper_2411_09473_gb300 import imm

    n, k = 100, 3
    off = torch.tensor([0, 2, 4], dtype=torch.int64, device="cuda")
    mem = torch.tensor([1, 2, 3, 100], dtype=torch.int32, device="cuda")
    d_seeds = torch.zeros(k, dtype=torch.int32, device="cuda")
    d_cov = torch.zeros(1, dtype=torch.int64, device="cuda")
    imm.imm_select_noalloc(n, 2, off, mem, k, d_seeds, d_cov)
    torch.cuda.synchronize()
    assert np.all(d_seeds.cpu().numpy().astype(np.uint32) == 0xFFFFFFFF)
    assert int(d_cov.cpu().numpy().view(np.uint64)[0]) == 2 ** 64 - 1
    mem[3] = 99
    imm.imm_select_noalloc(n, 2, off, mem, k, d_seeds, d_cov)
    torch.cuda.synchronize()
    want, wcov = oracle.select_sets(n, off.cpu().numpy(), mem.cpu().numpy(), k)
    assert np.array_equal(d_seeds.cpu().numpy().astype(np.uint32), want) and int(d_cov.item()) == wcov


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    from paper_2411_09473_gb300 import imm

    d_off = torch.zeros(2, dtype=torch.int64, device="cuda")
    d_mem = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_seeds = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(imm.ImmError):
        imm.imm_select_noalloc(imm.IMM_NOALLOC_MAX_N + 1, 1, d_off, d_mem, 4, d_seeds)
    with pytest.raises(imm.ImmError):
        imm.imm_select_noalloc(100, imm.IMM_NOALLOC_MAX_SETS + 1, d_off, d_mem, 4, d_seeds)
    with pytest.raises(imm.ImmError):
        imm.imm_select_noalloc(100, 1, d_off, d_mem, 0, d_seeds)
