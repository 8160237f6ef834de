"""Autotuner of the Horner-stage configuration for batched replicas.

Three knobs fix how a system's stage kernel tiles the grid:

* the block width bo (orbitals interleaved per grid point): bo = 4 gives the
  complex64 column kernel a 16 x 16-point tile that shares the potential and
  the projector records among four orbitals, bo = 2 a 32 x 16-point tile,
  bo = 1 the one-point-per-thread L1 kernel;
* the tile variant (EMD_OPT_STAGE_VARIANT) for bo = 2: the column kernel
  (one thread per orbital column and 2 rows), or one thread per point over
  1 or 2 rows (32 x 16 or 32 x 32 points);
* the z-chunk (EMD_OPT_ZCHUNK): planes marched per CTA; shorter chunks give
  more CTAs (small replicas fill more SMs) at the price of restaging 2M halo
  planes per chunk.

Which is fastest depends on the grid, the stencil order and the number of
orbitals, so each candidate runs a few MD steps of the given system timed
with CUDA events, and the fastest whole step is kept in a JSON cache keyed
by (grid, order, precision, orbital-count bucket) with every candidate's
timing, so the choice can be reported.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, List, Optional

from . import emd

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json")


def _key(sysin, precision: int) -> str:
    bucket = 32 if sysin.n_orb <= 32 else 64 if sysin.n_orb <= 64 else 128
    return f"n{sysin.n}-p{sysin.fd_order}-prec{precision}-orb{bucket}"


def candidates(sysin, precision: int) -> List[dict]:
    """The configurations searched for one system."""
    zs = sorted({0, max(8, sysin.n // 4)})
    out = []
    for z in zs:
        out.append(dict(bo=4, variant=0, zchunk=z))
        for v in (0, 2, 3):
            out.append(dict(bo=2, variant=v, zchunk=z))
    out.append(dict(bo=1, variant=0, zchunk=0))
    if precision == emd.EMD_FP64:          # one FP64 kernel per block width
        out = [c for c in out if c["variant"] == 0]
    return out


def _load(path: str) -> Dict[str, dict]:
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def configure(sysg, cfg: dict) -> None:
    """Apply a configuration's options to a system built with its bo."""
    emd.emd_set_option(sysg.handle, emd.EMD_OPT_STAGE_VARIANT, cfg["variant"])
    emd.emd_set_option(sysg.handle, emd.EMD_OPT_ZCHUNK, cfg["zchunk"])


def measure(sysin, precision: int, cfg: dict, steps: int = 2) -> dict:
    """MD-step time and average Horner-stage launch time (ms) of one
    configuration, CUDA events."""
    import torch
    sysg = emd.System(sysin, precision, block_orbitals=cfg["bo"])
    try:
        configure(sysg, cfg)
        sysg.propagate(1)
        emd.emd_set_option(sysg.handle, emd.EMD_OPT_PROFILE, 1)
        emd.emd_kernel_stats(sysg.handle)
        sysg.propagate(1)
        ms, n = emd.emd_kernel_stats(sysg.handle)
        emd.emd_set_option(sysg.handle, emd.EMD_OPT_PROFILE, 0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        sysg.propagate(steps)
        b.record()
        torch.cuda.synchronize()
        return {"step_ms": a.elapsed_time(b) / steps, "stage_ms": ms / max(n, 1)}
    finally:
        sysg.close()


def cfg_name(cfg: dict) -> str:
    return f"bo{cfg['bo']}-v{cfg['variant']}-z{cfg['zchunk']}"


def best_config(sysin, precision: int = emd.EMD_FP32_ORBITALS,
                cands: Optional[Iterable[dict]] = None,
                cache_path: Optional[str] = DEFAULT_CACHE) -> dict:
    """The fastest configuration for sysin's key (measured once per key)."""
    key = _key(sysin, precision)
    cache = _load(cache_path) if cache_path else {}
    if key in cache:
        return dict(cache[key]["best"])
    cands = list(cands) if cands is not None else candidates(sysin, precision)
    timings = {cfg_name(c): measure(sysin, precision, c) for c in cands}
    best = min(cands, key=lambda c: timings[cfg_name(c)]["step_ms"])
    if cache_path:
        cache[key] = {"best": best, "timings": timings}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dict(best)


def best_block_orbitals(sysin, precision: int = emd.EMD_FP32_ORBITALS,
                        cache_path: Optional[str] = DEFAULT_CACHE) -> int:
    """The block width of the best configuration."""
    return int(best_config(sysin, precision, cache_path=cache_path)["bo"])


def report(cache_path: str = DEFAULT_CACHE) -> Dict[str, dict]:
    """Per key: the chosen configuration and every candidate's timings."""
    return _load(cache_path)
