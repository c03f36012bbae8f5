"""Autotuner for the assembly tile extents (wq_plan_set_tiles), per degree.

For each degree it builds a seeded perturbed spline cube, times the FP64 stiffness
assembly for every candidate (t1, t2) that fits in shared memory, and keeps the
fastest. Results are cached as JSON {"p": [t1, t2], ...}; load_tiles() reads the
cache and apply_tiles() sets each plan's tiles from it.
"""
from __future__ import annotations

import json
import os

CANDIDATES = [(8, 2), (8, 4), (12, 4), (16, 2), (16, 4), (24, 2), (24, 4), (32, 2), (32, 4), (16, 6), (12, 6)]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "wq_gb300_tiles.json")


def tune(degrees=(2, 3, 4, 5), n_el: int = 24, reps: int = 3, cache: str | None = DEFAULT_CACHE,
         candidates=CANDIDATES, verbose: bool = False) -> dict:
    import torch

    from . import Plan, WqError
    from wq_synth import perturbed_cube
    best = {}
    for p in degrees:
        patch = perturbed_cube(p, n_el, seed=1605 + 4)
        plan = Plan(p, patch.knots, patch.ctrl)
        out = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
        timings = {}
        for (t1, t2) in candidates:
            plan.set_tiles(t1, t2)
            try:
                plan.stiffness(out=out)
            except WqError:
                continue
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                plan.stiffness(out=out)
            b.record()
            torch.cuda.synchronize()
            timings[(t1, t2)] = a.elapsed_time(b) / reps
        choice = min(timings, key=timings.get)
        best[str(p)] = list(choice)
        if verbose:
            print(f"p={p}: " + ", ".join(f"{k}: {v:.3f} ms" for k, v in sorted(timings.items(), key=lambda x: x[1])))
        plan.close()
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(best, f)
    return best


def load_tiles(cache: str = DEFAULT_CACHE) -> dict:
    if not os.path.exists(cache):
        return {}
    with open(cache) as f:
        return {int(k): tuple(v) for k, v in json.load(f).items()}


def apply_tiles(plans, tiles: dict) -> None:
    for pl in plans:
        if pl.p in tiles:
            pl.set_tiles(*tiles[pl.p])
