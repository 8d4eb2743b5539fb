"""IMM oracle (plain single-threaded C, loaded with ctypes).

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import or call this package.  The
product path (``paper_2411_09473_gb300``) never imports it, and it imports
nothing from the product path.

Every function follows a passage of EfficientIMM (arXiv 2411.09473) or of
Tang, Shi & Xiao (SIGMOD 2015, the paper's IMM reference); see oracle.c for
the per-function citations and the readings taken where the paper is silent.

Parity status per function (what pins it, tests/test_oracle_*.py):
  philox4x32_10       Random123 known-answer vectors + uniformity chi^2
  root / ic_live      empirical frequencies vs 1/n and thr/2^24 (chi^2, binomial)
  sample (IC)         RIS identity vs exact spread by live-edge enumeration;
                      p=1 closure vs scipy reverse BFS; p=0 singletons;
                      every member reaches the root through live edges
  sample (LT)         RIS identity vs exact spread by LT world enumeration;
                      directed cycle and path closed forms
  select_sets         brute-force optimum (greedy >= (1-1/e) OPT); recount-
                      from-scratch greedy; hand-traced tie-broken fixtures
  theta_params        ln C(n,k) vs exact big-integer binomial; lambda* vs the
                      two concentration bounds it balances; lambda' vs the
                      martingale tail bound it solves; ell' vs n^-ell / 2^ell
  run                 composition of the above; stopping rule checked
                      against theta_params on every round
  run (fresh_final)   same ladder as the plain run; final stream is exactly
                      theta sets equal to an independent sample under the
                      second key; RIS identity of its covered fraction
  opim_params         theta_max * k equals lambda* of Tang et al.'s bound at
                      the same confidence (OPT >= k); i_max against theta ratio
  opim_bounds         lower bound below the exact spread (world enumeration)
                      and upper bound above the exact optimum (brute force)
                      over many independent collections, and both within a
                      stated factor of the truth at large theta
  opim_run            collections double; R1 is the plain stream, R2 the
                      stream under seed ^ OPIM_KEY; stop rule on alpha; the
                      returned set's spread meets 1 - 1/e - eps of OPT
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

OK, EINVAL, ENOMEM = 0, 1, 2
FRESH_KEY = 0x9E3779B97F4A7C15  # key of the fresh final stream: seed ^ FRESH_KEY
IC, LT = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint32),
        ("stopped_early", ctypes.c_uint32),
        ("theta_i", ctypes.c_uint64 * 64),
        ("covered_i", ctypes.c_uint64 * 64),
        ("sets_i", ctypes.c_uint64 * 64),
        ("lb", ctypes.c_double),
        ("theta", ctypes.c_uint64),
        ("num_sets", ctypes.c_uint64),
        ("covered", ctypes.c_uint64),
        ("lambda_prime", ctypes.c_double),
        ("lambda_star", ctypes.c_double),
    ]


class OpimStats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint32),
        ("stopped_early", ctypes.c_uint32),
        ("i_max", ctypes.c_uint32),
        ("sets_i", ctypes.c_uint64 * 64),
        ("cov1_i", ctypes.c_uint64 * 64),
        ("cov2_i", ctypes.c_uint64 * 64),
        ("upper_i", ctypes.c_double * 64),
        ("lower_i", ctypes.c_double * 64),
        ("theta_max", ctypes.c_double),
        ("theta_0", ctypes.c_double),
        ("alpha", ctypes.c_double),
    ]


OPIM_KEY = 0xD1B54A32D192ED03  # key of the second RR collection: seed ^ OPIM_KEY


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u32, u64, i32, f64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "orc_philox4x32_10": ([vp, vp, vp], None),
        "orc_root": ([u64, u64, u32], u32),
        "orc_ic_threshold": ([ctypes.c_float], u32),
        "orc_ic_live": ([u64, u64, u32, u32], i32),
        "orc_lt_draw": ([u64, u64, u32], u32),
        "orc_theta_params": ([u32, u32, f64, f64, vp], None),
        "orc_create": ([u32, u64, vp, vp, vp, i32, ctypes.POINTER(i32)], vp),
        "orc_destroy": ([vp], None),
        "orc_sample": ([vp, u64, u64], i32),
        "orc_reset": ([vp], i32),
        "orc_select_sets": ([u32, u64, vp, vp, u32, vp, ctypes.POINTER(u64)], i32),
        "orc_select": ([vp, u32, vp, ctypes.POINTER(u64)], i32),
        "orc_run": ([vp, u32, f64, f64, u64, vp, ctypes.POINTER(Stats)], i32),
        "orc_run_ex": ([vp, u32, f64, f64, u64, u32, vp, ctypes.POINTER(Stats)], i32),
        "orc_num_sets": ([vp], u64),
        "orc_num_members": ([vp], u64),
        "orc_get_set": ([vp, u64, vp, u32, ctypes.POINTER(u32)], i32),
        "orc_sample_one": ([vp, u64, u64, vp, ctypes.POINTER(u32)], i32),
        "orc_get_counts": ([vp, vp], None),
        "orc_get_arena": ([vp, vp, vp], None),
        "orc_get_thresholds": ([vp, vp], None),
        "orc_opim_params": ([u32, u32, f64, f64, vp], None),
        "orc_opim_bounds": ([u32, u32, f64, f64, u64, u64, u64, vp], None),
        "orc_opim_run": ([vp, u32, f64, f64, u64, vp, ctypes.POINTER(OpimStats)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def root(seed: int, set_id: int, n: int) -> int:
    return int(_load().orc_root(seed, set_id, n))


def ic_threshold(p: float) -> int:
    return int(_load().orc_ic_threshold(ctypes.c_float(p)))


def ic_live(seed: int, set_id: int, e: int, thr: int) -> bool:
    return bool(_load().orc_ic_live(seed, set_id, e, thr))


def lt_draw(seed: int, set_id: int, v: int) -> int:
    return int(_load().orc_lt_draw(seed, set_id, v))


def theta_params(n: int, k: int, eps: float, ell: float) -> dict:
    out = np.zeros(8, dtype=np.float64)
    _load().orc_theta_params(n, k, eps, ell, _p(out))
    return dict(ell_p=out[0], eps_p=out[1], lnC=out[2], lambda_prime=out[3],
                lambda_star=out[4], alpha=out[5], beta=out[6], rounds=int(out[7]))


def opim_params(n: int, k: int, eps: float, ell: float) -> dict:
    """OPIM-C's constants (delta = n^-ell): theta_max, theta_0, i_max, a1, a2."""
    out = np.zeros(7, dtype=np.float64)
    _load().orc_opim_params(n, k, eps, ell, _p(out))
    return dict(delta=out[0], lnC=out[1], theta_max=out[2], theta_0=out[3], i_max=int(out[4]), a1=out[5],
                a2=out[6])


def opim_bounds(n: int, k: int, a1: float, a2: float, theta: int, cov1: int, cov2: int):
    """(upper bound on OPT from R1 coverage, lower bound on the spread of the
    greedy's set from its R2 coverage)."""
    out = np.zeros(2, dtype=np.float64)
    _load().orc_opim_bounds(n, k, a1, a2, theta, cov1, cov2, _p(out))
    return float(out[0]), float(out[1])


def select_sets(n: int, off: np.ndarray, mem: np.ndarray, k: int):
    """Greedy max coverage (Alg. 2) over an explicit set system."""
    off = np.ascontiguousarray(off, dtype=np.uint64)
    mem = np.ascontiguousarray(mem if len(mem) else np.zeros(1), dtype=np.uint32)
    seeds = np.zeros(max(k, 1), dtype=np.uint32)
    cov = ctypes.c_uint64(0)
    rc = _load().orc_select_sets(n, len(off) - 1, _p(off), _p(mem), k, _p(seeds), ctypes.byref(cov))
    if rc != OK:
        raise ValueError(f"orc_select_sets -> {rc}")
    return seeds[:k].copy(), int(cov.value)


class Oracle:
    """Plain IMM over one graph (transposed CSR, per-edge fp32 weights)."""

    def __init__(self, n, row, src, weight, model):
        lib = _load()
        self.n = int(n)
        self._row = np.ascontiguousarray(row, dtype=np.uint64)
        self._src = np.ascontiguousarray(src if len(src) else np.zeros(1), dtype=np.uint32)
        self._w = np.ascontiguousarray(weight if len(weight) else np.zeros(1), dtype=np.float32)
        self.m = int(self._row[-1])
        err = ctypes.c_int(0)
        self._h = lib.orc_create(self.n, self.m, _p(self._row), _p(self._src), _p(self._w), model,
                                 ctypes.byref(err))
        if not self._h:
            raise ValueError(f"orc_create failed with code {err.value}")
        self.model = model

    def close(self):
        if getattr(self, "_h", None):
            _load().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sample(self, theta: int, seed: int) -> None:
        rc = _load().orc_sample(self._h, theta, seed)
        if rc != OK:
            raise ValueError(f"orc_sample -> {rc}")

    def reset(self) -> None:
        _load().orc_reset(self._h)

    def select(self, k: int):
        seeds = np.zeros(k, dtype=np.uint32)
        cov = ctypes.c_uint64(0)
        rc = _load().orc_select(self._h, k, _p(seeds), ctypes.byref(cov))
        if rc != OK:
            raise ValueError(f"orc_select -> {rc}")
        return seeds, int(cov.value)

    def run(self, k: int, eps: float, ell: float, seed: int, fresh_final: bool = False):
        """Alg. 1; fresh_final: the final selection uses a fresh stream of
        exactly theta sets drawn under seed ^ FRESH_KEY (Chen 2018's
        correction of the set reuse)."""
        seeds = np.zeros(k, dtype=np.uint32)
        st = Stats()
        rc = _load().orc_run_ex(self._h, k, eps, ell, seed, 1 if fresh_final else 0, _p(seeds), ctypes.byref(st))
        if rc != OK:
            raise ValueError(f"orc_run -> {rc}")
        return seeds, st

    def opim_run(self, k: int, eps: float, ell: float, seed: int):
        """OPIM-style early stop (OPIM-C of Tang et al. 2018, which Sec. VI
        cites): R1 (key seed) and R2 (key seed ^ OPIM_KEY) double each round
        until the lower / upper bound ratio reaches 1 - 1/e - eps."""
        seeds = np.zeros(k, dtype=np.uint32)
        st = OpimStats()
        rc = _load().orc_opim_run(self._h, k, eps, ell, seed, _p(seeds), ctypes.byref(st))
        if rc != OK:
            raise ValueError(f"orc_opim_run -> {rc}")
        return seeds, st

    @property
    def num_sets(self) -> int:
        return int(_load().orc_num_sets(self._h))

    @property
    def num_members(self) -> int:
        return int(_load().orc_num_members(self._h))

    def get_set(self, set_id: int) -> np.ndarray:
        buf = np.zeros(self.n, dtype=np.uint32)
        ln = ctypes.c_uint32(0)
        rc = _load().orc_get_set(self._h, set_id, _p(buf), self.n, ctypes.byref(ln))
        if rc != OK:
            raise ValueError(f"orc_get_set -> {rc}")
        return buf[: ln.value].copy()

    def sample_one(self, seed: int, set_id: int) -> np.ndarray:
        buf = np.zeros(self.n, dtype=np.uint32)
        ln = ctypes.c_uint32(0)
        _load().orc_sample_one(self._h, seed, set_id, _p(buf), ctypes.byref(ln))
        return buf[: ln.value].copy()

    def counts(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.uint32)
        _load().orc_get_counts(self._h, _p(out))
        return out

    def arena(self):
        off = np.zeros(self.num_sets + 1, dtype=np.uint64)
        mem = np.zeros(max(self.num_members, 1), dtype=np.uint32)
        _load().orc_get_arena(self._h, _p(off), _p(mem))
        return off, mem[: self.num_members]

    def thresholds(self) -> np.ndarray:
        out = np.zeros(max(self.m, 1), dtype=np.uint32)
        _load().orc_get_thresholds(self._h, _p(out))
        return out[: self.m]
