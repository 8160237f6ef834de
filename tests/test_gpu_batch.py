"""Batched ragged replicas through the C ABI: a batch replays captured CUDA
graphs of 6 MD steps with one branch per replica; every replica must end
bit-identical to the same system stepped on its own, and (FP64) match the
oracle."""
import numpy as np
import pytest

from oracle import emd_oracle as O
from paper_0812_2801_gb300 import emd, inputs

pytestmark = pytest.mark.gpu


def replicas():
    return [inputs.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=3),
            inputs.small_system(n=20, h=0.3, fd_order=6, n_atoms=3, seed=5, n_orb=5),
            inputs.small_system(n=24, h=0.3, fd_order=8, n_atoms=2, seed=7, n_orb=3)]


@pytest.mark.parametrize("prec", [emd.EMD_FP64, emd.EMD_FP32_ORBITALS])
def test_batch_equals_individual_runs(prec):
    sysins = replicas()
    dt, mu = 0.04, 1.0
    solo = []
    for s in sysins:
        g = emd.System(s, prec)
        g.propagate(14, dt=dt, mu=mu)
        g.propagate(9, dt=dt, mu=mu)
        solo.append((g.state()[2], g.forces()))
        g.close()
    gs = [emd.System(s, prec) for s in sysins]
    b = emd.emd_batch_create([g.handle for g in gs])
    emd.emd_batch_propagate(b, 14, dt, mu)     # 2 eager + 2 graph chunks
    emd.emd_batch_propagate(b, 9, dt, mu)      # 1 graph chunk + 3 eager
    got = [(g.state()[2], g.forces()) for g in gs]
    emd.emd_batch_destroy(b)
    for g in gs:
        g.close()
    for (p1, f1), (p2, f2) in zip(solo, got):
        assert np.array_equal(p1, p2)
        assert np.array_equal(f1, f2)


def test_batch_replay_after_a_shifted_history_phase():
    """A call ending in 2 eager steps leaves the position-set parity as it
    was but rotates the three v_Hxc history slots; the next call must not
    replay a graph captured at the other rotation.  Also a plain propagate
    between batch calls, and a changed stage variant."""
    sysins = replicas()
    dt, mu = 0.04, 1.0
    solo = []
    for s in sysins:
        g = emd.System(s, emd.EMD_FP32_ORBITALS)
        g.propagate(14 + 8 + 6 + 1 + 6 + 6, dt=dt, mu=mu)
        solo.append((g.state()[2], g.forces()))
        g.close()
    gs = [emd.System(s, emd.EMD_FP32_ORBITALS) for s in sysins]
    b = emd.emd_batch_create([g.handle for g in gs])
    emd.emd_batch_propagate(b, 14, dt, mu)     # 2 eager + 2 graph chunks
    emd.emd_batch_propagate(b, 8, dt, mu)      # 1 graph chunk + 2 eager
    emd.emd_batch_propagate(b, 6, dt, mu)      # same parity, other history slots
    for g in gs:
        g.propagate(1, dt=dt, mu=mu)           # outside the batch
    emd.emd_batch_propagate(b, 6, dt, mu)
    emd.emd_set_option(gs[0].handle, emd.EMD_OPT_STAGE_VARIANT, 1)
    emd.emd_batch_propagate(b, 6, dt, mu)
    got = [(g.state()[2], g.forces()) for g in gs]
    emd.emd_batch_destroy(b)
    for g in gs:
        g.close()
    for k, ((p1, f1), (p2, f2)) in enumerate(zip(solo, got)):
        if k == 0:   # another kernel for the last 6 steps: same physics
            assert np.max(np.abs(p1 - p2)) < 1e-5 * np.max(np.abs(p1))
        else:
            assert np.array_equal(p1, p2), k
            assert np.array_equal(f1, f2), k


def test_batch_fp64_matches_oracle():
    sysins = replicas()[:2]
    gs = [emd.System(s) for s in sysins]
    b = emd.emd_batch_create([g.handle for g in gs])
    emd.emd_batch_propagate(b, 8, 0.04, 1.0)
    emd.emd_batch_destroy(b)
    for s, g in zip(sysins, gs):
        psi = g.state()[2]
        F = g.forces()
        g.close()
        st = O.run(s, 8, dt=0.04, mu=1.0)
        assert np.max(np.abs(psi - st.psi)) <= 1e-10
        assert np.max(np.abs(F - st.F)) <= 1e-9 * np.max(np.abs(st.F))


def c3_replicas():
    """One replica of each grid of the ragged-replica workload (48^3, 64^3,
    80^3; Si-like, order 8, 2 orbitals per atom)."""
    specs = inputs.replica_specs(32, seed=5)
    out, seen = [], set()
    for i, sp in enumerate(specs):
        if sp["n"] not in seen:
            seen.add(sp["n"])
            out.append(inputs.replica(sp, i))
    return out


CONFIGS = [dict(bo=4, variant=0, zchunk=0), dict(bo=2, variant=2, zchunk=16),
           dict(bo=2, variant=3, zchunk=0), dict(bo=1, variant=0, zchunk=0)]


def test_c3_shapes_every_tuned_configuration_against_oracle_points():
    """H psi of 4 orbitals at sampled points of each replica shape, in every
    configuration the autotuner searches (block width, tile variant,
    z-chunk), against the oracle evaluated point by point."""
    from paper_0812_2801_gb300 import autotune
    for s in c3_replicas():
        tables = O.atom_tables(s.R, s.species, s.n, s.h)
        rng = np.random.default_rng(s.n)
        pts = [tuple(int(v) for v in rng.integers(0, s.n, size=3)) for _ in range(16)]
        pts += [(0, 0, 0), (s.n - 1, s.n - 1, s.n - 1), (0, s.n - 1, s.n // 2)]
        u = s.psi[:4]
        c = O.projections(u, tables, s.species, s.h)
        for cfg in CONFIGS:
            g = emd.System(s, emd.EMD_FP32_ORBITALS, block_orbitals=cfg["bo"])
            autotune.configure(g, cfg)
            pot = emd.emd_get_potentials(g.handle, s.n)
            hu = emd.emd_apply_hamiltonian(g.handle, u)
            g.close()
            v_eff = pot["v_loc"] + pot["v_h"] + pot["v_xc"]
            ref = O.hamiltonian_at_points(u, v_eff, c, s.R, s.species, s.h, s.fd_order, pts,
                                          list(range(4)))
            got = np.array([[hu[a, z, y, x] for (z, y, x) in pts] for a in range(4)])
            assert np.max(np.abs(got - ref)) < 2e-5 * np.max(np.abs(ref)), (s.n, cfg)


def test_c3_shapes_batch_with_mixed_configurations_equals_solo_runs():
    """The three replica shapes, each in a different configuration, stepped as
    one batch (eager warm-up, then graph chunks) equal the same systems
    stepped alone, bit for bit."""
    from paper_0812_2801_gb300 import autotune
    sysins = c3_replicas()
    cfgs = CONFIGS[:len(sysins)]
    dt, mu = sysins[0].dt, sysins[0].mu
    solo = []
    for s, cfg in zip(sysins, cfgs):
        g = emd.System(s, emd.EMD_FP32_ORBITALS, block_orbitals=cfg["bo"])
        autotune.configure(g, cfg)
        g.propagate(8, dt=dt, mu=mu)
        solo.append(g.state()[2])
        g.close()
    gs = []
    for s, cfg in zip(sysins, cfgs):
        g = emd.System(s, emd.EMD_FP32_ORBITALS, block_orbitals=cfg["bo"])
        autotune.configure(g, cfg)
        gs.append(g)
    b = emd.emd_batch_create([g.handle for g in gs])
    emd.emd_batch_propagate(b, 8, dt, mu)
    got = [g.state()[2] for g in gs]
    emd.emd_batch_destroy(b)
    for g in gs:
        g.close()
    for p1, p2 in zip(solo, got):
        assert np.array_equal(p1, p2)
