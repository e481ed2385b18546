"""Autotuner for the solve kernel's launch mapping.

The solve is compiled in several variants: two kernel forms (owner-mapped
tree sweeps; compact upper levels with incrementally updated strains) and,
for the mixed precision, several numbers of CTAs per SM the compiler is asked
to fit (register budget per thread: 65536 / (128 * CTAs)).  The best one
depends on the tree depth and on how many Newton iterations the workload
takes, so it is measured: every variant runs the same synthetic increments
and the fastest is written to a JSON table that ``DMN`` consults when no
variant is given.  Variant numbers are those of ``dmn_options.solve_variant``:
2, 3, 4 owner-mapped mixed; 12, 13, 14 compact mixed; 0 owner-mapped FP64;
11 compact FP64.

Usage (on a GPU):  python -m paper_2109_14403_gb300.autotune [--K 8] [--points 65536]
"""
from __future__ import annotations

import argparse
import json
import os

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
VARIANTS = {"mixed": (2, 3, 4, 12, 13, 14), "fp64": (0, 11)}


def key(K: int, precision: str) -> str:
    return f"K={int(K)},{precision}"


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(K: int, precision: str, path: str = TABLE) -> int:
    """Variant chosen by the last tuning run (0 = library default)."""
    e = load_table(path).get(key(K, precision))
    return int(e["variant"]) if e else 0


def choose(times: dict) -> int:
    """Fastest variant from {variant: ms_per_step}; ties go to the smaller variant."""
    return min(sorted(times), key=lambda v: (times[v], v))


def tune(K: int = 8, n_points: int = 65536, n_steps: int = 4, warmup: int = 2,
         precision: str = "mixed", path: str = TABLE) -> dict:
    """Time every variant on the K-deep random-walk workload; update the table."""
    import torch

    from . import synthetic as syn
    from .dmn import DMN

    dev = torch.device("cuda", torch.cuda.current_device())
    w, nrm, ph = syn.tree(K)
    deps, theta = syn.random_walk_k8(n_points=n_points, n_incr=warmup + n_steps)
    D = torch.tensor(deps, device=dev)
    T = torch.tensor(theta, device=dev)
    times = {}
    for v in VARIANTS[precision]:
        d = DMN(K, w, nrm, ph, syn.materials(), precision=precision, solve_variant=v)
        s = d.init_state(torch.full((n_points,), syn.THETA_START, dtype=torch.float64, device=dev))
        s2 = torch.empty_like(s)
        out = torch.empty((n_points, 57), dtype=torch.float64, device=dev)
        st = torch.empty(n_points, dtype=torch.int32, device=dev)
        it = torch.empty_like(st)
        for k in range(warmup):
            d.eval(D[k], T[k], 1.0, s, s2, out, st, it)
            s, s2 = s2, s
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(warmup, warmup + n_steps):
            d.eval(D[k], T[k], 1.0, s, s2, out, st, it)
            s, s2 = s2, s
        e1.record()
        torch.cuda.synchronize()
        times[v] = e0.elapsed_time(e1) / n_steps
        d.close()
    best = choose(times)
    table = load_table(path)
    table[key(K, precision)] = {"variant": best, "ms_per_step": times, "points": n_points}
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return table[key(K, precision)]


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--K", type=int, default=8)
    ap.add_argument("--points", type=int, default=65536)
    ap.add_argument("--precision", default="mixed")
    a = ap.parse_args()
    print(json.dumps(tune(a.K, a.points, precision=a.precision)))
