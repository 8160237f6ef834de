"""Orbital-block autotuner for the Horner-stage kernels.

The block width bo (orbitals interleaved per grid point) fixes the memory
layout and the stencil kernel's tile: bo = 2 gives a 32 x 16-point tile per
CTA in the complex64 kernel, bo = 4 a 16 x 16-point tile that shares the
potential and projector lists among more orbitals.  Which is faster depends
on the grid, the stencil order and the number of orbitals, so it is measured:
each candidate runs a few MD steps of the given system with the stage kernel
timed by CUDA events inside libemd, and the fastest is cached in a JSON file
keyed by (grid, order, precision, orbital-count bucket).
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional

from . import emd

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json")


def _key(sysin, precision: int) -> str:
    bucket = 32 if sysin.n_orb <= 32 else 64 if sysin.n_orb <= 64 else 128
    return f"n{sysin.n}-p{sysin.fd_order}-prec{precision}-orb{bucket}"


def _load(path: str) -> Dict[str, dict]:
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def measure_stage_ms(sysin, precision: int, bo: int, steps: int = 2) -> float:
    """Average Horner-stage launch time (ms) for block width bo."""
    sysg = emd.System(sysin, precision, block_orbitals=bo)
    try:
        sysg.propagate(1)
        emd.emd_set_option(sysg.handle, emd.EMD_OPT_PROFILE, 1)
        emd.emd_kernel_stats(sysg.handle)
        sysg.propagate(steps)
        ms, n = emd.emd_kernel_stats(sysg.handle)
        return ms / max(n, 1)
    finally:
        sysg.close()


def best_block_orbitals(sysin, precision: int = emd.EMD_FP32_ORBITALS,
                        candidates: Iterable[int] = (2, 4),
                        cache_path: Optional[str] = DEFAULT_CACHE) -> int:
    key = _key(sysin, precision)
    cache = _load(cache_path) if cache_path else {}
    if key in cache:
        return int(cache[key]["bo"])
    timings = {bo: measure_stage_ms(sysin, precision, bo) for bo in candidates}
    best = min(timings, key=timings.get)
    if cache_path:
        cache[key] = {"bo": best, "stage_ms": {str(k): v for k, v in timings.items()}}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return best
