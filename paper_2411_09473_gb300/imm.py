"""Thin ctypes binding of the C ABI in include/imm.h (same names, argument
marshalling only).  Every step of the IMM hot path runs in the CUDA library;
PyTorch supplies the device memory (its caching allocator, through the
imm_alloc callbacks) and the CUDA stream.

The binding refuses to work without the compiled library: there is no CPU
fallback.  Build it with ``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import _build

IMM_OK, IMM_EINVAL, IMM_ENOMEM, IMM_ECUDA, IMM_ETIMEOUT, IMM_ESTATE = range(6)
IMM_IC, IMM_LT = 0, 1
IMM_MAX_ROUNDS = 64
_NAMES = {0: "IMM_OK", 1: "IMM_EINVAL", 2: "IMM_ENOMEM", 3: "IMM_ECUDA", 4: "IMM_ETIMEOUT", 5: "IMM_ESTATE"}


class ImmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class imm_stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint32),
        ("stopped_early", ctypes.c_uint32),
        ("theta_i", ctypes.c_uint64 * IMM_MAX_ROUNDS),
        ("covered_i", ctypes.c_uint64 * IMM_MAX_ROUNDS),
        ("sets_i", ctypes.c_uint64 * IMM_MAX_ROUNDS),
        ("lb", ctypes.c_double),
        ("theta", ctypes.c_uint64),
        ("num_sets", ctypes.c_uint64),
        ("covered", ctypes.c_uint64),
        ("lambda_prime", ctypes.c_double),
        ("lambda_star", ctypes.c_double),
        ("members", ctypes.c_uint64),
        ("edges_examined", ctypes.c_uint64),
        ("ms_total", ctypes.c_double),
        ("ms_sample", ctypes.c_double),
        ("ms_select", ctypes.c_double),
        ("ms_index", ctypes.c_double),
        ("sample_launches", ctypes.c_uint64),
        ("kernel_launches", ctypes.c_uint64),
        ("sample_edges", ctypes.c_uint64),
        ("sample_members", ctypes.c_uint64),
        ("reused_sets", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        r = self.rounds
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("theta_i", "covered_i", "sets_i")}
        d["theta_i"] = [int(self.theta_i[i]) for i in range(min(r, IMM_MAX_ROUNDS))]
        d["covered_i"] = [int(self.covered_i[i]) for i in range(min(r, IMM_MAX_ROUNDS))]
        d["sets_i"] = [int(self.sets_i[i]) for i in range(min(r, IMM_MAX_ROUNDS))]
        return d


class imm_opim_stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint32),
        ("stopped_early", ctypes.c_uint32),
        ("i_max", ctypes.c_uint32),
        ("sets_i", ctypes.c_uint64 * IMM_MAX_ROUNDS),
        ("cov1_i", ctypes.c_uint64 * IMM_MAX_ROUNDS),
        ("cov2_i", ctypes.c_uint64 * IMM_MAX_ROUNDS),
        ("upper_i", ctypes.c_double * IMM_MAX_ROUNDS),
        ("lower_i", ctypes.c_double * IMM_MAX_ROUNDS),
        ("theta_max", ctypes.c_double),
        ("theta_0", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("ms_sample", ctypes.c_double),
        ("ms_select", ctypes.c_double),
        ("kernel_launches", ctypes.c_uint64),
    ]


IMM_OPIM_KEY = 0xD1B54A32D192ED03


class imm_tuning(ctypes.Structure):
    _fields_ = [("batch_sets", ctypes.c_uint32), ("group_min_mean", ctypes.c_uint32),
                ("select_cta_max_n", ctypes.c_uint32), ("cluster_min_n", ctypes.c_uint32),
                ("select_cand", ctypes.c_uint32), ("solo_cluster", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


IMM_TUNE_CANDIDATES = 12


class imm_server_config(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_uint64), ("max_active", ctypes.c_uint32),
                ("share_streams", ctypes.c_uint32)]


class imm_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double)]


class imm_query(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("k", ctypes.c_uint32), ("epsilon", ctypes.c_double),
                ("ell", ctypes.c_double), ("rng_seed", ctypes.c_uint64)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class imm_alloc(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # IMM_LIBRARY_VARIANT=bounds (tests) loads the bounds-checked build
    path = _build.BOUNDS_LIB_PATH if os.environ.get("IMM_LIBRARY_VARIANT") == "bounds" else _build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: the CUDA library must be built (__graft_entry__.build()); "
                           "there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32, f64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    sig = {
        "imm_create": ([ctypes.POINTER(vp), i32, ctypes.POINTER(imm_alloc), vp], i32),
        "imm_destroy": ([vp], None),
        "imm_last_error": ([vp], ctypes.c_char_p),
        "imm_load_graph": ([vp, u32, u64, vp, vp, vp, i32], i32),
        "imm_load_graph_device": ([vp, u32, u64, vp, vp, vp, i32], i32),
        "imm_sample": ([vp, i32, u64, u64], i32),
        "imm_select": ([vp, u32, vp, ctypes.POINTER(u64)], i32),
        "imm_run": ([vp, i32, u32, f64, f64, u64, vp, ctypes.POINTER(imm_stats)], i32),
        "imm_run_ex": ([vp, i32, u32, f64, f64, u64, u32, vp, ctypes.POINTER(imm_stats)], i32),
        "imm_run_opim": ([vp, i32, u32, f64, f64, u64, vp, ctypes.POINTER(imm_opim_stats)], i32),
        "imm_set_tuning": ([vp, ctypes.POINTER(imm_tuning)], i32),
        "imm_build_flags": ([], i32),
        "imm_get_tuning": ([vp, ctypes.POINTER(imm_tuning)], i32),
        "imm_autotune_batch": ([vp, u32, u32, ctypes.POINTER(imm_tuning), vp, vp], i32),
        "imm_reset_sets": ([vp], i32),
        "imm_stream_size": ([vp, ctypes.POINTER(u64), ctypes.POINTER(u64)], i32),
        "imm_get_set": ([vp, u64, vp, u32, ctypes.POINTER(u32)], i32),
        "imm_get_sets": ([vp, u64, u64, vp, vp, u64], i32),
        "imm_get_counts": ([vp, vp], i32),
        "imm_set_arena_limit": ([vp, u64], i32),
        "imm_select_noalloc": ([u32, u64, vp, vp, u32, vp, vp, vp], i32),
        "imm_run_batch": ([ctypes.POINTER(imm_query), u32, vp, ctypes.POINTER(imm_stats), vp], i32),
        "imm_server_create": ([ctypes.POINTER(vp), ctypes.POINTER(vp), u32, ctypes.POINTER(imm_server_config)], i32),
        "imm_server_submit": ([vp, u32, u32, f64, f64, u64, ctypes.POINTER(u64)], i32),
        "imm_server_poll": ([vp, ctypes.POINTER(imm_completion), u32, ctypes.POINTER(u32)], i32),
        "imm_server_take": ([vp, u64, vp, u32, ctypes.POINTER(imm_stats)], i32),
        "imm_server_info": ([vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64),
                             ctypes.POINTER(u64)], i32),
        "imm_server_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


class _Ctx:
    """Opaque context handle plus the Python objects it must keep alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        try:
            imm_destroy(self)
        except Exception:
            pass


def _check(ctx: Optional[_Ctx], rc: int):
    if rc != IMM_OK:
        msg = _load().imm_last_error(ctx.handle if ctx is not None else None)
        raise ImmError(rc, msg.decode() if msg else "")


def _torch_allocator(device: int, stream_int: int):
    import torch

    def _alloc(user, nbytes, stream):
        # The block belongs to the stream the library names (a batch worker's
        # own stream, not the creating context's): torch's caching allocator
        # only reuses a freed block in that stream's order.
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=device, stream=int(stream or 0))
        except Exception:
            return None

    def _free(user, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_FN(_alloc), _FREE_FN(_free)
    return imm_alloc(a, f, None), (a, f)


def imm_create(device: int = 0, stream=None, allocator: str = "torch") -> _Ctx:
    """Create a context.  stream: a torch.cuda.Stream, an int cudaStream_t, or
    None for torch's current stream; allocator: "torch" (caching allocator) or
    "cuda" (cudaMallocAsync inside the library)."""
    import torch
    lib = _load()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    stream_int = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    keep = [stream]
    alloc_p = None
    if allocator == "torch":
        st, cbs = _torch_allocator(device, stream_int)
        keep += [st, cbs]
        alloc_p = ctypes.pointer(st)
    elif allocator != "cuda":
        raise ValueError(allocator)
    h = ctypes.c_void_p()
    rc = lib.imm_create(ctypes.byref(h), device, alloc_p, ctypes.c_void_p(stream_int))
    if rc != IMM_OK:
        raise ImmError(rc, "imm_create failed")
    return _Ctx(h, keep)


def imm_destroy(ctx: _Ctx) -> None:
    if ctx.handle:
        _load().imm_destroy(ctx.handle)
        ctx.handle = None


def imm_last_error(ctx: _Ctx) -> str:
    return _load().imm_last_error(ctx.handle).decode()


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def imm_load_graph(ctx: _Ctx, n: int, m: int, in_row, in_src, weight, model: int) -> None:
    row = _host(in_row, np.uint64)
    src = _host(in_src if m else np.zeros(1), np.uint32)
    w = _host(weight if m else np.zeros(1), np.float32)
    _check(ctx, _load().imm_load_graph(ctx.handle, n, m, row.ctypes.data, src.ctypes.data, w.ctypes.data, model))


def imm_load_graph_device(ctx: _Ctx, n: int, m: int, d_row, d_src, d_weight, model: int) -> None:
    """Device-pointer variant: torch CUDA tensors (uint64/int64 row, int32 src, float32 weight)."""
    _check(ctx, _load().imm_load_graph_device(ctx.handle, n, m, d_row.data_ptr(), d_src.data_ptr(),
                                              d_weight.data_ptr(), model))


def imm_sample(ctx: _Ctx, model: int, theta: int, rng_seed: int) -> None:
    _check(ctx, _load().imm_sample(ctx.handle, model, theta, rng_seed))


def imm_select(ctx: _Ctx, k: int):
    seeds = np.zeros(max(k, 1), dtype=np.uint32)
    cov = ctypes.c_uint64(0)
    _check(ctx, _load().imm_select(ctx.handle, k, seeds.ctypes.data, ctypes.byref(cov)))
    return seeds[:k], int(cov.value)


def imm_run(ctx: _Ctx, model: int, k: int, epsilon: float, ell: float, rng_seed: int):
    seeds = np.zeros(max(k, 1), dtype=np.uint32)
    st = imm_stats()
    _check(ctx, _load().imm_run(ctx.handle, model, k, epsilon, ell, rng_seed, seeds.ctypes.data, ctypes.byref(st)))
    return seeds[:k], st


IMM_RUN_FRESH_FINAL = 1


def imm_run_ex(ctx: _Ctx, model: int, k: int, epsilon: float, ell: float, rng_seed: int, flags: int):
    seeds = np.zeros(max(k, 1), dtype=np.uint32)
    st = imm_stats()
    _check(ctx, _load().imm_run_ex(ctx.handle, model, k, epsilon, ell, rng_seed, flags, seeds.ctypes.data,
                                   ctypes.byref(st)))
    return seeds[:k], st


def imm_run_opim(ctx: _Ctx, model: int, k: int, epsilon: float, ell: float, rng_seed: int):
    """OPIM-style early stop (OPIM-C): (seeds, imm_opim_stats)."""
    seeds = np.zeros(max(k, 1), dtype=np.uint32)
    st = imm_opim_stats()
    _check(ctx, _load().imm_run_opim(ctx.handle, model, k, epsilon, ell, rng_seed, seeds.ctypes.data,
                                     ctypes.byref(st)))
    return seeds[:k], st


IMM_BUILD_BOUNDS_CHECK = 1


def imm_build_flags() -> int:
    return int(_load().imm_build_flags())


def imm_set_tuning(ctx: _Ctx, **knobs) -> None:
    """Change knobs of the context's tuning (see imm_tuning); speed only."""
    t = imm_tuning()
    _check(ctx, _load().imm_get_tuning(ctx.handle, ctypes.byref(t)))
    for k, v in knobs.items():
        setattr(t, k, v)
    _check(ctx, _load().imm_set_tuning(ctx.handle, ctypes.byref(t)))


def imm_get_tuning(ctx: _Ctx) -> dict:
    t = imm_tuning()
    _check(ctx, _load().imm_get_tuning(ctx.handle, ctypes.byref(t)))
    return t.as_dict()


def imm_autotune_batch(queries, reps: int = 1):
    """Autotune a batch: (best tuning dict, [(candidate dict, mean ms)])."""
    nq = len(queries)
    arr = (imm_query * max(nq, 1))()
    for i, (g, k, eps, ell, seed) in enumerate(queries):
        arr[i] = imm_query(g.handle, k, eps, ell, seed)
    best = imm_tuning()
    times = np.zeros(IMM_TUNE_CANDIDATES, dtype=np.float64)
    cands = (imm_tuning * IMM_TUNE_CANDIDATES)()
    rc = _load().imm_autotune_batch(arr, nq, reps, ctypes.byref(best), times.ctypes.data, cands)
    if rc != IMM_OK:
        raise ImmError(rc, "imm_autotune_batch failed")
    return best.as_dict(), [(cands[i].as_dict(), float(times[i])) for i in range(IMM_TUNE_CANDIDATES)]


def imm_run_batch(queries):
    """queries: list of (graph_ctx, k, epsilon, ell, rng_seed).  Returns
    (seeds per query, imm_stats per query, status per query); raises ImmError
    only when the batch as a whole is rejected."""
    nq = len(queries)
    arr = (imm_query * max(nq, 1))()
    total = 0
    for i, (g, k, eps, ell, seed) in enumerate(queries):
        arr[i] = imm_query(g.handle, k, eps, ell, seed)
        total += k
    seeds = np.zeros(max(total, 1), dtype=np.uint32)
    stats = (imm_stats * max(nq, 1))()
    status = np.zeros(max(nq, 1), dtype=np.int32)
    rc = _load().imm_run_batch(arr, nq, seeds.ctypes.data, stats, status.ctypes.data)
    if rc != IMM_OK:
        _check(queries[0][0] if nq else None, rc)
    out, off = [], 0
    for (_, k, _, _, _) in queries:
        out.append(seeds[off:off + k].copy())
        off += k
    return out, [stats[i] for i in range(nq)], [int(x) for x in status[:nq]]


def imm_reset_sets(ctx: _Ctx) -> None:
    _check(ctx, _load().imm_reset_sets(ctx.handle))


def imm_stream_size(ctx: _Ctx):
    a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(ctx, _load().imm_stream_size(ctx.handle, ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def imm_get_set(ctx: _Ctx, set_id: int, cap: int) -> np.ndarray:
    buf = np.zeros(max(cap, 1), dtype=np.uint32)
    ln = ctypes.c_uint32(0)
    _check(ctx, _load().imm_get_set(ctx.handle, set_id, buf.ctypes.data, cap, ctypes.byref(ln)))
    return buf[: ln.value].copy()


def imm_get_sets(ctx: _Ctx, first: int, count: int, members: bool = True):
    """Sets first .. first+count-1: (offsets relative to the first set,
    members); with members=False only the offsets (a call with cap 0)."""
    lib = _load()
    off = np.zeros(count + 1, dtype=np.uint64)
    rc = lib.imm_get_sets(ctx.handle, first, count, off.ctypes.data, None, 0)
    total = int(off[-1])
    if rc != IMM_OK and total == 0:
        _check(ctx, rc)
    if not members:
        return off, None
    mem = np.zeros(max(total, 1), dtype=np.uint32)
    _check(ctx, lib.imm_get_sets(ctx.handle, first, count, off.ctypes.data, mem.ctypes.data, total))
    return off, mem[:total]


def imm_get_counts(ctx: _Ctx, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint32)
    _check(ctx, _load().imm_get_counts(ctx.handle, out.ctypes.data))
    return out


def imm_set_arena_limit(ctx: _Ctx, nbytes: int) -> None:
    _check(ctx, _load().imm_set_arena_limit(ctx.handle, nbytes))


IMM_NOALLOC_MAX_N = 1 << 20
IMM_NOALLOC_MAX_SETS = 1 << 22
IMM_NOALLOC_MAX_K = 4096


def imm_select_noalloc(n: int, nsets: int, d_off, d_members, k: int, d_seeds_out, d_covered_out=None,
                       stream=None) -> None:
    """Greedy selection over a device-resident set system without any device
    allocation (for callers that cannot allocate).  d_off: CUDA int64 tensor
    [nsets+1]; d_members: CUDA int32 tensor; d_seeds_out: CUDA int32 tensor [k];
    d_covered_out: CUDA int64 tensor [1] or None.  Enqueued on `stream`
    (default: torch's current stream); raises ImmError on a rejected call."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    mem_ptr = d_members.data_ptr() if d_members is not None and d_members.numel() else None
    cov_ptr = d_covered_out.data_ptr() if d_covered_out is not None else None
    rc = _load().imm_select_noalloc(n, nsets, d_off.data_ptr(), mem_ptr, k, d_seeds_out.data_ptr(), cov_ptr,
                                     ctypes.c_void_p(st))
    if rc != IMM_OK:
        raise ImmError(rc, "imm_select_noalloc rejected the call (sizes above the fixed scratch limits, "
                           "bad k, or a NULL pointer)" if rc == IMM_EINVAL else "CUDA error")


class _Server:
    def __init__(self, handle, graphs):
        self.handle = handle
        self._graphs = graphs  # keep the graph contexts alive

    def __del__(self):
        try:
            imm_server_destroy(self)
        except Exception:
            pass


def imm_server_create(graphs, memory_budget_bytes: int = 0, max_active: int = 64,
                      share_streams: bool = False) -> _Server:
    """Continuous-batching server over loaded graph contexts (kept alive by the
    handle); share_streams: prefix-stable reuse of resident streams."""
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle.value if hasattr(g.handle, "value") else g.handle
                                              for g in graphs])
    cfg = imm_server_config(memory_budget_bytes, max_active, 1 if share_streams else 0)
    h = ctypes.c_void_p()
    rc = _load().imm_server_create(ctypes.byref(h), arr, len(graphs), ctypes.byref(cfg))
    if rc != IMM_OK:
        raise ImmError(rc, "imm_server_create failed")
    return _Server(h, list(graphs))


def imm_server_submit(server: _Server, graph: int, k: int, epsilon: float, ell: float, rng_seed: int) -> int:
    qid = ctypes.c_uint64(0)
    rc = _load().imm_server_submit(server.handle, graph, k, epsilon, ell, rng_seed, ctypes.byref(qid))
    if rc != IMM_OK:
        raise ImmError(rc, "imm_server_submit rejected the query")
    return int(qid.value)


def imm_server_poll(server: _Server, cap: int = 1024):
    buf = (imm_completion * cap)()
    n = ctypes.c_uint32(0)
    rc = _load().imm_server_poll(server.handle, buf, cap, ctypes.byref(n))
    if rc != IMM_OK:
        raise ImmError(rc, "imm_server_poll failed")
    return [(int(buf[i].id), int(buf[i].status), float(buf[i].latency_ms), float(buf[i].queue_ms))
            for i in range(n.value)]


def imm_server_take(server: _Server, qid: int, k: int):
    seeds = np.zeros(max(k, 1), dtype=np.uint32)
    st = imm_stats()
    rc = _load().imm_server_take(server.handle, qid, seeds.ctypes.data, k, ctypes.byref(st))
    if rc != IMM_OK:
        raise ImmError(rc, f"imm_server_take({qid}) failed")
    return seeds[:k], st


def imm_server_info(server: _Server):
    a, b, c, d = (ctypes.c_uint64(0) for _ in range(4))
    rc = _load().imm_server_info(server.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
    return dict(pending=int(a.value), active=int(b.value), waves=int(c.value), device_bytes=int(d.value),
                status=rc)


def imm_server_destroy(server: _Server) -> None:
    if server.handle:
        _load().imm_server_destroy(server.handle)
        server.handle = None
