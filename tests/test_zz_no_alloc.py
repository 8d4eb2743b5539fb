"""imm_select_noalloc: selection for callers that cannot allocate device memory
(a plugin inside a framework whose pool owns the GPU, a service with a fixed
footprint).  Its output must equal imm_select's on the same sets, call after
call, although every call reuses the same fixed scratch array."""
import numpy as np
import pytest

import graphgen


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
        off, mem = imm.imm_get_sets(ctx, 0, theta)
        d_off = torch.from_numpy(off.astype(np.int64)).cuda()
        d_mem = torch.from_numpy(mem.astype(np.int32)).cuda()
        for _ in range(2):  # the second call sees the first call's leftovers
            d_seeds = torch.full((k,), -1, dtype=torch.int32, device="cuda")
            d_cov = torch.zeros(1, dtype=torch.int64, device="cuda")
            imm.imm_select_noalloc(g.n, theta, d_off, d_mem, k, d_seeds, d_cov)
            torch.cuda.synchronize()
            assert np.array_equal(d_seeds.cpu().numpy().astype(np.uint32), want)
            assert int(d_cov.item()) == wcov
        imm.imm_destroy(ctx)


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
