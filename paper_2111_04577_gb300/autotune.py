"""Autotuner of the library's launch shapes (x-transform lines per CTA, y-transform
columns, z-solve columns, row-kernel block width).

For one grid and precision it measures, knob by knob, every candidate with
pf_profile on a scratch context and keeps the value that minimises the device
time of the kernels that knob shapes.  Results are cached in a JSON file keyed
by grid and precision, and applied to a Solver with `apply`.  The knobs change
only the tiling, never the arithmetic of a cell, so a tuned context computes
the same numbers as an untuned one.
"""
from __future__ import annotations

import json
import os

from . import binding
from . import workloads as wl

KNOBS = {
    0: ("xfft_pairs", [1, 2, 4, 8], ("rfft_x_fine", "ch_ifftx_finish", "rfft_x_coarse", "irfft_x_coarse")),
    1: ("yfft_cols", [8, 16, 32], ("fft_y_fine", "fft_y_coarse")),
    2: ("zsolve_cols", [16, 32], ("zsolve_pair", "zsolve")),
    3: ("row_block", [64, 128, 256], ("ns_rhs", "div", "correct", "polymer_stage1", "polymer_stage2")),
    4: ("ch_zchunk", [16, 32, 64], ("ch_rhs",)),
    5: ("ch_minb", [2, 3, 4], ("ch_rhs",)),
    6: ("ns_minb", [3, 4], ("ns_rhs",)),
    7: ("g_zchunk", [4, 8, 16], ("ch_G_restrict",)),
    8: ("ns_kz", [4, 8, 16, 32], ("ns_rhs",)),
}

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tuning.json")


def signature(grid: wl.Grid, precision: int) -> str:
    return f"{grid.nx}x{grid.ny}x{grid.nz}/dual{grid.dual}/{'fp64' if precision == binding.PF_FP64 else 'mixed'}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_of(prof, names) -> float:
    return sum(ms for (n, ms, _) in prof if n in names)


def tune(grid: wl.Grid, params: wl.Params, precision: int, phi0=None, steps: int = 3) -> dict:
    """Greedy knob-by-knob search on a scratch context.  Returns {knob_name: value}."""
    s = binding.Solver(grid, params, precision)
    try:
        if phi0 is None:
            phi0 = wl.initial_phi(wl.Workload("tune", grid, params, 1))
        s.load_state(phi0)
        s.profile(1)  # warm: graph-free launches, allocations touched
        best = {}
        for knob, (name, cands, kernels) in KNOBS.items():
            if grid.dim == 2 and name in ("yfft_cols", "ch_zchunk", "ch_minb", "g_zchunk"):
                continue
            timings = {}
            for v in cands:
                try:
                    s.set_tuning(knob, v)
                except binding.PFError:
                    continue  # does not fit this grid
                prof, _ = s.profile(steps)
                timings[v] = _time_of(prof, kernels)
            if timings:
                v = min(timings, key=timings.get)
                s.set_tuning(knob, v)
                best[name] = v
        return best
    finally:
        s.close()


def apply(solver: "binding.Solver", choice: dict) -> None:
    for knob, (name, _, _) in KNOBS.items():
        if name in choice:
            solver.set_tuning(knob, int(choice[name]))


def tuned(grid: wl.Grid, params: wl.Params, precision: int, path: str = DEFAULT_CACHE, phi0=None) -> dict:
    """Cached choice for this grid/precision, tuning on first use."""
    cache = load_cache(path)
    key = signature(grid, precision)
    if key not in cache:
        cache[key] = tune(grid, params, precision, phi0=phi0)
        save_cache(cache, path)
    return cache[key]
