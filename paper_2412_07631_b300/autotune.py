"""Autotuners of the blocking, measured on the GPU and cached.

outer_block: the factorisation's outer block width (the rank of the
tensor-core trailing updates, the paper's block size of the blocked QR of
Sec. 2.1).  A wider block raises the flops per byte of every trailing update
but lengthens the inner panel updates and the T assembly; the best width
depends on the geometry, the precision and the GPU, so it is measured:
each candidate factorises the actual system once (CUDA events) and the
fastest is kept in a JSON cache keyed by geometry, precision and device.

solve_plan: the tile plan of the batched solve (Sec. 2 Eq. 3 for a batch of
sinograms): the rows of the triangular solve's diagonal superblocks (each
applied as one GEMM with its stored inverse: larger blocks mean fewer,
deeper dependent steps but more inverse flops) and the least split-K depth
of the solve's GEMMs (the Q^T sweep's products over all rows and the
triangular solve's products are short and wide; deeper splits mean fewer,
longer CTAs and less partial-sum traffic).  Each candidate solves the given
batch with the given factor (the first, untimed solve builds the inverses
and captures the graphs; the second is timed) and the fastest is cached,
keyed by geometry, precision, batch size and device.

    nb = autotune.outer_block(geom, "tf32")          # tune once, then cached
    F = System(geom, "fp32").factor("tf32", nb_outer=nb)
    F.solve_plan = autotune.solve_plan(F, B)
"""
from __future__ import annotations

import json
import os
import time

DEFAULT_CANDIDATES = (1024, 1536, 2048, 2560)


def cache_path() -> str:
    return os.environ.get("CTQR_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ctqr", "tune.json"))


def _key(geom, precision: str, device: str) -> str:
    return (f"{device}|n{geom.n_side}|v{geom.n_views}|b{geom.n_bins}|pw{geom.pixel_width:g}"
            f"|bw{geom.bin_width:g}|arc{geom.arc_deg:g}|sl{geom.sqrt_lambda:g}|{precision}")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path: str | None = None) -> None:
    path = path or cache_path()
    d = load_cache(path)
    d[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(timings: dict) -> int:
    """The fastest candidate; ties go to the narrower block."""
    return min(timings, key=lambda nb: (timings[nb], nb))


def time_factor(geom, precision: str, nb_outer: int, repeats: int = 1) -> float:
    """Milliseconds of one factorisation (system build excluded), best of repeats."""
    import torch
    import paper_2412_07631_b300 as ct
    storage = "fp64" if precision == "fp64" else "fp32"
    best = float("inf")
    for _ in range(repeats):
        sysg = ct.System(geom, storage)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        F = sysg.factor(precision, nb_outer=nb_outer)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
        F.free()
        sysg.free()
    return best


def outer_block(geom, precision: str = "tf32", candidates=DEFAULT_CANDIDATES, path: str | None = None,
                retune: bool = False, repeats: int = 1, timer=None) -> int:
    """The outer block width for this geometry and precision: from the cache,
    or measured over `candidates` (and cached).  `timer(geom, precision, nb)`
    replaces the GPU timing (for tests of the selection logic)."""
    device = "cpu"
    if timer is None:
        import torch
        device = torch.cuda.get_device_name()
    key = _key(geom, precision, device)
    if not retune:
        hit = load_cache(path).get(key)
        if hit and int(hit.get("nb_outer", 0)) > 0:
            return int(hit["nb_outer"])
    timer = timer or (lambda g, p, nb: time_factor(g, p, nb, repeats))
    timings = {int(nb): float(timer(geom, precision, int(nb))) for nb in candidates}
    nb = pick(timings)
    store(key, {"nb_outer": nb, "ms": {str(k): v for k, v in timings.items()},
                "when": time.strftime("%Y-%m-%dT%H:%M:%S")}, path)
    return nb


DEFAULT_SOLVE_PLANS = ((2048, 256), (1024, 256), (4096, 256), (2048, 512), (2048, 1024), (4096, 1024))


def time_solve(factor, B, plan, max_iter: int = 0, tol: float = 0.0) -> float:
    """Milliseconds of one solve of batch B with `plan` (after one untimed solve)."""
    import torch
    factor.solve_plan = tuple(plan)
    factor.solve(B, max_iter=max_iter, tol=tol, allow_noconv=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    factor.solve(B, max_iter=max_iter, tol=tol, allow_noconv=True)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def solve_plan(factor, B, candidates=DEFAULT_SOLVE_PLANS, path: str | None = None, retune: bool = False,
               max_iter: int = 0, tol: float = 0.0, timer=None) -> tuple[int, int]:
    """(solve_block, solve_split) for this factor's geometry, precision and
    batch size: from the cache, or measured over `candidates` (and cached).
    `timer(factor, B, plan)` replaces the GPU timing (for tests of the
    selection logic).  The factor's plan is left at the choice."""
    device = "cpu"
    if timer is None:
        import torch
        device = torch.cuda.get_device_name()
    key = _key(factor.system.geom, factor.precision, device) + f"|k{int(B.shape[0])}|solve"
    if not retune:
        hit = load_cache(path).get(key)
        if hit and "solve_plan" in hit:
            factor.solve_plan = tuple(int(v) for v in hit["solve_plan"])
            return factor.solve_plan
    timer = timer or (lambda f, b, p: time_solve(f, b, p, max_iter, tol))
    timings = {tuple(int(v) for v in p): float(timer(factor, B, p)) for p in candidates}
    best = min(timings, key=lambda p: (timings[p], p))
    store(key, {"solve_plan": list(best), "ms": {f"{p[0]}x{p[1]}": v for p, v in timings.items()},
                "when": time.strftime("%Y-%m-%dT%H:%M:%S")}, path)
    factor.solve_plan = best
    return best
