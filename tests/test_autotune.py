"""Stage-configuration autotuner: candidate set, choice and cache logic on the
host (timings are faked; the GPU measurement runs in the batched bench leg
and in tests/test_gpu_batch.py)."""

from paper_0812_2801_gb300 import autotune, emd, inputs


def test_candidates_cover_block_widths_tiles_and_zchunks():
    s = inputs.small_system(n=48, h=0.3, n_atoms=2, seed=1)
    c = autotune.candidates(s, emd.EMD_FP32_ORBITALS)
    assert {x["bo"] for x in c} == {1, 2, 4}
    assert {x["variant"] for x in c if x["bo"] == 2} == {0, 2, 3}
    assert {x["zchunk"] for x in c} == {0, 12}
    c64 = autotune.candidates(s, emd.EMD_FP64)
    assert all(x["variant"] == 0 for x in c64)


def test_picks_the_fastest_step_and_caches_by_key(tmp_path, monkeypatch):
    calls = []

    def fake(sysin, precision, cfg, steps=2):
        calls.append(autotune.cfg_name(cfg))
        step = {4: 0.7, 2: 0.9, 1: 2.0}[cfg["bo"]] - (0.05 if cfg["zchunk"] else 0.0)
        return {"step_ms": step, "stage_ms": step / 10}

    monkeypatch.setattr(autotune, "measure", fake)
    cache = str(tmp_path / "tune.json")
    s = inputs.small_system(n=16, h=0.35, n_atoms=2, seed=1)
    best = autotune.best_config(s, emd.EMD_FP32_ORBITALS, cache_path=cache)
    assert best == {"bo": 4, "variant": 0, "zchunk": 8}
    n_first = len(calls)
    assert n_first == len(autotune.candidates(s, emd.EMD_FP32_ORBITALS))
    # a second system with the same key is answered from the cache
    s2 = inputs.small_system(n=16, h=0.35, n_atoms=2, seed=2)
    assert autotune.best_block_orbitals(s2, emd.EMD_FP32_ORBITALS, cache_path=cache) == 4
    assert len(calls) == n_first
    rep = autotune.report(cache)
    key = next(iter(rep))
    assert rep[key]["best"] == best and len(rep[key]["timings"]) == n_first
    # another grid is measured again
    s3 = inputs.small_system(n=20, h=0.3, n_atoms=2, seed=1)
    autotune.best_config(s3, emd.EMD_FP32_ORBITALS, cache_path=cache)
    assert len(calls) == 2 * n_first
