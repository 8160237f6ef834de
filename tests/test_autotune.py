"""Block-width autotuner: choice and cache logic on the host (the timings
are faked; the GPU measurement itself runs in the batched bench leg)."""

from paper_0812_2801_gb300 import autotune, emd, inputs


def test_picks_the_fastest_and_caches_by_key(tmp_path, monkeypatch):
    calls = []

    def fake(sysin, precision, bo, steps=2):
        calls.append(bo)
        return {2: 0.9, 4: 0.7}[bo]

    monkeypatch.setattr(autotune, "measure_stage_ms", fake)
    cache = str(tmp_path / "tune.json")
    s = inputs.small_system(n=16, h=0.35, n_atoms=2, seed=1)
    assert autotune.best_block_orbitals(s, emd.EMD_FP32_ORBITALS, cache_path=cache) == 4
    assert sorted(calls) == [2, 4]
    # a second system with the same key is answered from the cache
    s2 = inputs.small_system(n=16, h=0.35, n_atoms=2, seed=2)
    assert autotune.best_block_orbitals(s2, emd.EMD_FP32_ORBITALS, cache_path=cache) == 4
    assert len(calls) == 2
    # another grid is measured again
    s3 = inputs.small_system(n=20, h=0.3, n_atoms=2, seed=1)
    autotune.best_block_orbitals(s3, emd.EMD_FP32_ORBITALS, cache_path=cache)
    assert len(calls) == 4
