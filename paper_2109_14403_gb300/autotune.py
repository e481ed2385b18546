"""Autotuner for the solve kernel's launch mapping.

The solve is compiled in several variants along two mapping axes and one
resource axis:
  * warps per Gauss point and points per CTA: the owner-mapped and the
    compact form put one point on a CTA of 2^(K-1) threads (four warps at
    K = 8, one point per CTA); the warp form puts one point on one warp and
    four points on a CTA;
  * CTAs per SM the compiler is asked to fit (the register budget per thread,
    65536 / (threads per CTA x CTAs)).
The fastest depends on the tree depth and on how many Newton iterations the
workload takes, so it is measured: every variant runs the same synthetic
increments of one workload, and the fastest is written to a JSON table under
a key of (depth, precision, workload) that ``DMN`` consults when no variant
is given.  Workloads: the random walk of the benchmark ("random_walk"), the
uniaxial ramp that drives the matrix into plastic flow ("plastic") and the
lognormal increment magnitudes of the uneven batch ("uneven").  Variant
numbers are those of ``dmn_options.solve_variant``: 2, 3, 4 owner-mapped
mixed; 12, 13, 14 compact mixed; 22, 23, 24 warp form (mixed, K = 6..8);
0 owner-mapped FP64; 11 compact FP64.  A variant the library rejects for a
configuration is left out of that run.

Usage (on a GPU):  python -m paper_2109_14403_gb300.autotune [--K 8] [--points 65536]
                   [--workload random_walk|plastic|uneven]
"""
from __future__ import annotations

import argparse
import json
import os

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
VARIANTS = {"mixed": (2, 3, 4, 12, 13, 14, 22, 23, 24), "fp64": (0, 11)}
WORKLOADS = ("random_walk", "plastic", "uneven")
# the mapping each variant selects (points per CTA, warps per point at K = 8)
MAPPING = {0: "owner-mapped, 1 point per CTA", 2: "owner-mapped, 1 point per CTA",
           3: "owner-mapped, 1 point per CTA", 4: "owner-mapped, 1 point per CTA",
           11: "compact, 1 point per CTA", 12: "compact, 1 point per CTA",
           13: "compact, 1 point per CTA", 14: "compact, 1 point per CTA",
           22: "warp form, 4 points per CTA, 1 warp per point",
           23: "warp form, 4 points per CTA, 1 warp per point",
           24: "warp form, 4 points per CTA, 1 warp per point"}


def key(K: int, precision: str, workload: str = "random_walk") -> str:
    base = f"K={int(K)},{precision}"
    return base if workload == "random_walk" else f"{base},{workload}"


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(K: int, precision: str, path: str = TABLE, workload: str = "random_walk") -> int:
    """Variant chosen by the last tuning run for this workload, else the
    random walk's, else 0 (the library default)."""
    t = load_table(path)
    e = t.get(key(K, precision, workload)) or t.get(key(K, precision))
    return int(e["variant"]) if e else 0


def choose(times: dict) -> int:
    """Fastest variant from {variant: ms_per_step}; ties go to the smaller variant."""
    return min(sorted(times), key=lambda v: (times[v], v))


def workload_increments(workload: str, K: int, n_points: int, n_incr: int):
    """(deps[n_incr, n, 6], theta[n_incr, n]) of a tuning workload."""
    from . import synthetic as syn
    if workload == "random_walk":
        return syn.random_walk_k8(n_points=n_points, n_incr=n_incr)
    if workload == "plastic":
        return syn.ramp_k4(n_points=n_points, n_incr=n_incr)
    if workload == "uneven":
        _, deps, theta = syn.uneven_batch(n_points=n_points, n_incr=n_incr)
        return deps, theta
    raise ValueError(f"unknown workload {workload!r}")


def tune(K: int = 8, n_points: int = 65536, n_steps: int = 4, warmup: int = 2,
         precision: str = "mixed", path: str = TABLE, workload: str = "random_walk",
         variants=None) -> dict:
    """Time every variant on the workload's increments; update the table."""
    import torch

    from . import synthetic as syn
    from .dmn import DMN

    dev = torch.device("cuda", torch.cuda.current_device())
    w, nrm, ph = syn.tree(K)
    deps, theta = workload_increments(workload, K, n_points, warmup + n_steps)
    D = torch.tensor(deps, device=dev)
    T = torch.tensor(theta, device=dev)
    times = {}
    for v in (variants or VARIANTS[precision]):
        try:
            d = DMN(K, w, nrm, ph, syn.materials(), precision=precision, solve_variant=v)
        except RuntimeError as e:
            if "solve_variant" in str(e):  # not available for this configuration
                continue
            raise
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
    table[key(K, precision, workload)] = {"variant": best, "mapping": MAPPING.get(best, ""),
                                          "ms_per_step": times, "points": n_points,
                                          "workload": workload}
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return table[key(K, precision, workload)]


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--K", type=int, default=8)
    ap.add_argument("--points", type=int, default=65536)
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--workload", default="random_walk", choices=WORKLOADS)
    a = ap.parse_args()
    print(json.dumps(tune(a.K, a.points, precision=a.precision, workload=a.workload)))
