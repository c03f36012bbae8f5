"""Autotuner for the assembly tile extents (wq_plan_set_tiles), per degree.

For each degree it builds a seeded perturbed spline cube, times the FP64 stiffness
assembly for every candidate (t1, t2) that fits in shared memory, and keeps the
fastest. Results are cached as a text file of "p t1 t2" lines, the format that
wq_options.tune_cache reads at plan creation; load_tiles() reads the cache and
apply_tiles() sets each plan's tiles from it.
"""
from __future__ import annotations

import os

CANDIDATES = [(8, 2), (8, 4), (12, 4), (16, 2), (16, 4), (24, 2), (24, 4), (32, 2), (32, 4), (16, 6), (12, 6)]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "wq_gb300_tiles.txt")


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
        save_tiles(best, cache)
    return best


def save_tiles(tiles: dict, cache: str = DEFAULT_CACHE) -> None:
    """Write {p: (t1, t2)} as "p t1 t2" lines."""
    d = os.path.dirname(cache)
    if d:
        os.makedirs(d, exist_ok=True)
    with open(cache, "w") as f:
        f.write("# p t1 t2: fused-assembly tile extents per degree\n")
        for p, (t1, t2) in sorted((int(k), v) for k, v in tiles.items()):
            f.write(f"{p} {int(t1)} {int(t2)}\n")


def load_tiles(cache: str = DEFAULT_CACHE) -> dict:
    if not os.path.exists(cache):
        return {}
    out = {}
    with open(cache) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if len(parts) == 3:
                out[int(parts[0])] = (int(parts[1]), int(parts[2]))
    return out


def apply_tiles(plans, tiles: dict) -> None:
    for pl in plans:
        if pl.p in tiles:
            pl.set_tiles(*tiles[pl.p])
