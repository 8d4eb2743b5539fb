"""Write the stored expected values of the full-size parity tests.

Every value written here comes from the oracle (oracle/) run on the seeded
inputs of graphgen/ and from nothing else: this script imports no part of the
CUDA library.  The oracle is single-threaded; the batched and served sets run
several oracle processes side by side (spawned, one query each), which changes
nothing in what each query computes.

    python tests/golden/make_golden.py ic_u01_1m     # ~2 h, ~43 GB RAM, one core
    python tests/golden/make_golden.py batch64       # 64 instances, n up to 2^18
    python tests/golden/make_golden.py served [N]    # the first N served queries
    python tests/golden/make_golden.py opim          # OPIM early stop, LT and U[0,1] IC

Each writes tests/golden/<name>.json.  Floating-point fields are also stored as
float.hex() so that the tests compare them bit for bit.
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402


def graph_digest(g) -> str:
    h = hashlib.sha256()
    for a in (g.row.astype("<u8"), g.src.astype("<u4"), g.weight.astype("<f4")):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def counts_digest(cnt: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(cnt.astype("<u4")).tobytes()).hexdigest()


def run_record(g, k, eps, ell, seed, with_counts=False):
    """One oracle run (Alg. 1) and the fields the tests compare."""
    o = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
    t0 = time.perf_counter()
    seeds, st = o.run(k, eps, ell, seed)
    dt = time.perf_counter() - t0
    r = st.rounds
    rec = dict(
        seeds=[int(x) for x in seeds],
        rounds=int(st.rounds), stopped_early=int(st.stopped_early),
        theta_i=[int(st.theta_i[i]) for i in range(r)],
        covered_i=[int(st.covered_i[i]) for i in range(r)],
        sets_i=[int(st.sets_i[i]) for i in range(r)],
        lb=float(st.lb), lb_hex=float(st.lb).hex(),
        theta=int(st.theta), num_sets=int(st.num_sets), covered=int(st.covered),
        members=int(o.num_members),
        lambda_prime_hex=float(st.lambda_prime).hex(), lambda_star_hex=float(st.lambda_star).hex(),
        oracle_seconds=round(dt, 3),
    )
    if with_counts:
        cnt = o.counts()
        rec.update(counts_sha256=counts_digest(cnt), counts_sum=int(cnt.astype(np.uint64).sum()),
                   counts_max=int(cnt.max()), counts_argmax=int(np.argmax(cnt)))
    o.close()
    return rec


def write(name, obj):
    path = os.path.join(HERE, name + ".json")
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        f.write("{\n")
        keys = list(obj)
        for j, key in enumerate(keys):
            val = obj[key]
            if isinstance(val, list) and val and isinstance(val[0], dict):
                body = "[\n" + ",\n".join("  " + json.dumps(v, separators=(",", ":")) for v in val) + "\n ]"
            else:
                body = json.dumps(val, separators=(",", ":"))
            f.write(f" {json.dumps(key)}: {body}{',' if j + 1 < len(keys) else ''}\n")
        f.write("}\n")
    os.replace(tmp, path)
    print("wrote", path)


def make_plain(name):
    w = graphgen.plain_workload(name)
    g = w.graph
    rec = run_record(g, w.k, w.epsilon, w.ell, w.seed, with_counts=True)
    rec.update(workload=name, desc=w.desc, n=g.n, m=g.m, k=w.k, epsilon=w.epsilon, ell=w.ell,
               seed=w.seed, graph_sha256=graph_digest(g),
               generated_by=f"python tests/golden/make_golden.py {name}")
    write(name, rec)


_CACHE = {}


def _cached(key, make):
    """Inputs regenerated once per worker process."""
    if key not in _CACHE:
        _CACHE[key] = make()
    return _CACHE[key]


def _batch_one(i):
    b = _cached("batch64", lambda: graphgen.batch_workload(count=64, max_log_n=18.0))
    q = b.queries[i]
    g = b.graphs[q.graph_id]
    rec = run_record(g, q.k, q.epsilon, q.ell, q.seed, with_counts=True)
    rec.update(index=i, n=g.n, m=g.m, model=g.model, k=q.k, epsilon=q.epsilon, epsilon_hex=q.epsilon.hex(),
               ell=q.ell, seed=q.seed, graph_sha256=graph_digest(g))
    return rec


def _served_one(i):
    gs = _cached("served_graphs", graphgen.served_graphs)
    q = _cached("served_queries", graphgen.served_queries)[i]
    g = gs[q.graph_id]
    rec = run_record(g, q.k, q.epsilon, q.ell, q.seed)
    rec.update(index=i, graph_id=q.graph_id, k=q.k, epsilon=q.epsilon, epsilon_hex=q.epsilon.hex(),
               ell=q.ell, seed=q.seed)
    return rec


def _opim_one(name):
    w = graphgen.plain_workload(name)
    g = w.graph
    o = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
    t0 = time.perf_counter()
    seeds, st = o.opim_run(w.k, w.epsilon, w.ell, w.seed)
    dt = time.perf_counter() - t0
    r = st.rounds
    return dict(workload=name, k=w.k, epsilon=w.epsilon, ell=w.ell, seed=w.seed, graph_sha256=graph_digest(g),
                seeds=[int(x) for x in seeds], rounds=int(r), stopped_early=int(st.stopped_early),
                i_max=int(st.i_max), sets_i=[int(st.sets_i[i]) for i in range(r)],
                cov1_i=[int(st.cov1_i[i]) for i in range(r)], cov2_i=[int(st.cov2_i[i]) for i in range(r)],
                upper_hex=[float(st.upper_i[i]).hex() for i in range(r)],
                lower_hex=[float(st.lower_i[i]).hex() for i in range(r)],
                alpha_hex=float(st.alpha).hex(), theta_max_hex=float(st.theta_max).hex(),
                theta_0_hex=float(st.theta_0).hex(), oracle_seconds=round(dt, 3))


def _pool_map(fn, items, procs):
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        out = []
        for j, r in enumerate(pool.imap(fn, items, chunksize=1)):
            out.append(r)
            print(f"{j + 1}/{len(items)} done ({r['oracle_seconds']:.1f} s)", flush=True)
        return out


def make_batch(procs):
    recs = _pool_map(_batch_one, list(range(64)), procs)
    write("batch64", dict(workload="batch64", count=64, max_log_n=18.0, batch_seed=4,
                          desc="64 IMM instances: R-MAT n=round(2^U(10,18)), avg degree U(8,32), "
                               "IC/LT alternating with 1/indeg weights, k=U{5..100}, eps=U(0.1,0.5)",
                          generated_by="python tests/golden/make_golden.py batch64",
                          instances=recs))


def make_served(count, procs):
    gs = graphgen.served_graphs()
    recs = _pool_map(_served_one, list(range(count)), procs)
    write("served", dict(workload="served", queries=count, rate_per_s=200.0, stream_seed=5,
                         desc="first queries of the served stream: 8 resident R-MAT graphs of "
                              "2^16..2^20 vertices (avg degree 16, IC/LT alternating, 1/indeg), "
                              "k=U{10..200}, eps=U(0.1,0.5), rng seed = query id",
                         graphs=[dict(n=g.n, m=g.m, model=g.model, graph_sha256=graph_digest(g)) for g in gs],
                         generated_by=f"python tests/golden/make_golden.py served {count}",
                         results=recs))


def make_opim(procs):
    recs = _pool_map(_opim_one, ["lt_4m", "ic_u1_256k"], procs)
    write("opim", dict(workload="opim", desc="OPIM-style early stop (OPIM-C) on the LT and U[0,1] IC workloads",
                       generated_by="python tests/golden/make_golden.py opim", runs=recs))


def main(argv):
    graphgen.build()
    oracle.build()
    what = argv[1] if len(argv) > 1 else ""
    procs = int(os.environ.get("GOLDEN_PROCS", max(1, (os.cpu_count() or 2) - 1)))
    if what in graphgen.PLAIN:
        make_plain(what)
    elif what == "batch64":
        make_batch(procs)
    elif what == "opim":
        make_opim(procs)
    elif what == "served":
        make_served(int(argv[2]) if len(argv) > 2 else 300, procs)
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv)
