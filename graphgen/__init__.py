"""Seeded synthetic inputs for the IMM hot path.

This package produces the inputs that both the oracle and the CUDA path
consume: R-MAT graphs in transposed CSR (`row`, `src`), fp32 edge weights, and
the per-workload parameters (k, epsilon, ell, seeds, batches, arrival times).
It contains none of the method's arithmetic: no thresholds, coins, RRR sets,
counts or theta math.  The random words come from a counter hash of its own
(see rmat.c), independent of the Philox stream the method draws.

The R-MAT graphs stand in for the SNAP social graphs the paper evaluates on
(EfficientIMM Table I, Sec. V-A); those datasets are not used.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmat.c")
_LIB = os.path.join(_HERE, "_rmat.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile rmat.c into graphgen/_rmat.so (plain C, host only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32, u64, f64, f32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_float
        vp = ctypes.c_void_p
        lib.gg_rmat.argtypes = [u32, u64, f64, f64, f64, u64, vp, vp]
        lib.gg_rmat.restype = ctypes.c_int
        lib.gg_weights_inv_indeg.argtypes = [u32, vp, vp]
        lib.gg_weights_inv_indeg.restype = None
        lib.gg_weights_uniform.argtypes = [u64, f32, u64, vp]
        lib.gg_weights_uniform.restype = None
        lib.gg_uniform_f64.argtypes = [u64, u64, u64, vp]
        lib.gg_uniform_f64.restype = None
        lib.gg_word.argtypes = [u64, u64, u32]
        lib.gg_word.restype = u64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def rmat(n: int, m: int, seed: int, a: float = 0.57, b: float = 0.19, c: float = 0.19):
    """R-MAT graph as transposed CSR: (row uint64[n+1], src uint32[m])."""
    lib = _load()
    row = np.empty(n + 1, dtype=np.uint64)
    src = np.empty(max(m, 1), dtype=np.uint32)
    rc = lib.gg_rmat(n, m, a, b, c, seed, _ptr(row), _ptr(src))
    if rc != 0:
        raise ValueError(f"gg_rmat failed with code {rc} (n={n}, m={m})")
    return row, src[:m]


def weights_inv_indeg(row: np.ndarray) -> np.ndarray:
    """w_e = 1/indeg(head) in fp32 (weighted cascade for IC, uniform LT weights)."""
    lib = _load()
    n = row.shape[0] - 1
    m = int(row[-1])
    w = np.zeros(max(m, 1), dtype=np.float32)
    lib.gg_weights_inv_indeg(n, _ptr(np.ascontiguousarray(row, dtype=np.uint64)), _ptr(w))
    return w[:m]


def weights_uniform(m: int, pmax: float, seed: int) -> np.ndarray:
    """w_e uniform in [0, pmax) as fp32: (u24 * 2^-24) * pmax."""
    lib = _load()
    w = np.empty(max(m, 1), dtype=np.float32)
    lib.gg_weights_uniform(m, ctypes.c_float(pmax), seed, _ptr(w))
    return w[:m]


def uniform_f64(count: int, seed: int, first: int = 0) -> np.ndarray:
    lib = _load()
    out = np.empty(max(count, 1), dtype=np.float64)
    lib.gg_uniform_f64(count, seed, first, _ptr(out))
    return out[:count]


IC, LT = 0, 1


@dataclass
class Graph:
    n: int
    row: np.ndarray
    src: np.ndarray
    weight: np.ndarray
    model: int

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


@dataclass
class Workload:
    """One plain-IMM workload: a graph plus (k, epsilon, ell, rng seed)."""
    name: str
    graph: Graph
    k: int
    epsilon: float
    ell: float
    seed: int
    desc: str = ""


def make_graph(n: int, m: int, graph_seed: int, model: int, weights: str = "inv_indeg",
               pmax: float = 0.1) -> Graph:
    row, src = rmat(n, m, graph_seed)
    if weights == "inv_indeg":
        w = weights_inv_indeg(row)
    elif weights == "uniform":
        w = weights_uniform(m, pmax, graph_seed)
    else:
        raise ValueError(weights)
    return Graph(n=n, row=row, src=src, weight=w, model=model)


# The three plain-IMM workloads (sizes, weight laws, k, epsilon, ell, seed).
PLAIN = {
    "ic_wc_4k": dict(n=1 << 12, m=1 << 15, model=IC, weights="inv_indeg", k=10, epsilon=0.5,
                     ell=1.0, seed=1,
                     desc="IC, R-MAT 4,096 vertices / 32,768 edges, p=1/indeg, k=10, eps=0.5"),
    "ic_u01_1m": dict(n=1 << 20, m=1 << 24, model=IC, weights="uniform", k=50, epsilon=0.13,
                      ell=1.0, seed=2,
                      desc="IC, R-MAT 1,048,576 vertices / 16,777,216 edges, p~U[0,0.1], "
                           "k=50, eps=0.13"),
    "lt_4m": dict(n=1 << 22, m=1 << 26, model=LT, weights="inv_indeg", k=100, epsilon=0.5,
                  ell=1.0, seed=3,
                  desc="LT, R-MAT 4,194,304 vertices / 67,108,864 edges, w=1/indeg, k=100, "
                       "eps=0.5"),
    # the paper's IC weight law (p ~ U[0, 1]) with its k = 50, eps = 0.5
    "ic_u1_256k": dict(n=1 << 18, m=1 << 22, model=IC, weights="uniform", pmax=1.0, k=50, epsilon=0.5,
                       ell=1.0, seed=6,
                       desc="IC, R-MAT 262,144 vertices / 4,194,304 edges, p~U[0,1], k=50, eps=0.5"),
}


def plain_workload(name: str) -> Workload:
    p = PLAIN[name]
    g = make_graph(p["n"], p["m"], p["seed"], p["model"], p["weights"], p.get("pmax", 0.1))
    return Workload(name=name, graph=g, k=p["k"], epsilon=p["epsilon"], ell=p["ell"],
                    seed=p["seed"], desc=p["desc"])


@dataclass
class Query:
    """One IMM query against a graph (batched and served workloads)."""
    graph_id: int
    k: int
    epsilon: float
    ell: float
    seed: int
    arrival_s: float = 0.0


@dataclass
class Batch:
    graphs: list = field(default_factory=list)
    queries: list = field(default_factory=list)


def batch_workload(count: int = 64, batch_seed: int = 4, max_log_n: float = 18.0) -> Batch:
    """Many independent instances of uneven size: n = round(2^U(10, max_log_n)),
    average degree U(8, 32), models alternating IC (1/indeg) / LT (1/indeg),
    k = U{5..100}, epsilon = U(0.1, 0.5); graph seed and rng seed = instance index."""
    u = uniform_f64(4 * count, batch_seed)
    out = Batch()
    for i in range(count):
        n = int(round(2.0 ** (10.0 + (max_log_n - 10.0) * u[4 * i])))
        deg = 8.0 + 24.0 * u[4 * i + 1]
        m = int(round(n * deg))
        k = 5 + int(u[4 * i + 2] * 96)
        eps = 0.1 + 0.4 * u[4 * i + 3]
        model = IC if i % 2 == 0 else LT
        out.graphs.append(make_graph(n, m, i, model, "inv_indeg"))
        out.queries.append(Query(graph_id=i, k=min(k, n), epsilon=eps, ell=1.0, seed=i))
    return out


def served_graphs(log_n_lo: float = 16.0, log_n_hi: float = 20.0, count: int = 8,
                  avg_deg: int = 16):
    """Resident graphs: n log-spaced over 2^16..2^20, average degree 16,
    models alternating IC (1/indeg) / LT (1/indeg); graph seed 100 + j."""
    gs = []
    for j in range(count):
        n = int(round(2.0 ** (log_n_lo + (log_n_hi - log_n_lo) * j / max(count - 1, 1))))
        model = IC if j % 2 == 0 else LT
        gs.append(make_graph(n, n * avg_deg, 100 + j, model, "inv_indeg"))
    return gs


def served_queries(count: int = 10000, rate_per_s: float = 200.0, num_graphs: int = 8,
                   stream_seed: int = 5, k_lo: int = 10, k_hi: int = 200):
    """Poisson arrivals (exponential gaps), uniform graph choice, k = U{k_lo..k_hi},
    epsilon = U(0.1, 0.5), rng seed = query id."""
    u = uniform_f64(4 * count, stream_seed)
    t = 0.0
    qs = []
    for i in range(count):
        t += -math.log1p(-u[4 * i]) / rate_per_s
        gid = min(int(u[4 * i + 1] * num_graphs), num_graphs - 1)
        k = k_lo + min(int(u[4 * i + 2] * (k_hi - k_lo + 1)), k_hi - k_lo)
        eps = 0.1 + 0.4 * u[4 * i + 3]
        qs.append(Query(graph_id=gid, k=k, epsilon=eps, ell=1.0, seed=i, arrival_s=t))
    return qs
