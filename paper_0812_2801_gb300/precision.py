"""Energy conservation of the complex64-orbital form against the complex128
form on the same input.

The modified Ehrenfest dynamics conserve E_total = E_KS[phi, R] + sum_J M_J
|V_J|^2 / 2 (Sec. 4, the conserved quantity of the modified equations of
motion); with the time-reversible AETRS propagator (Sec. 5) a discrete run
shows no secular drift beyond the integrator's error.  This module runs both
precisions side by side and reports, per run:

* ``drift_rel``      |E(t_N) - E(0)| / |E(0)|
* ``max_dev_rel``    max_t |E(t) - E(0)| / |E(0)|
* ``slope_rel_1000`` least-squares slope of E(t) over the run, times 1000
                     steps, divided by |E(0)| (separates a secular drift from
                     a bounded oscillation)

and, for the complex64 form against the complex128 form:

* ``force_err_traj``  max_J |F32_J - F64_J| / max_J |F64_J| at each sample,
                      the two runs each on its own trajectory
* ``force_err_state`` the same with the complex64 forces evaluated at the
                      complex128 run's state (its R and orbitals loaded into a
                      complex64 system), i.e. the error of the force
                      evaluation alone
* ``state_errors``    at those samples, per result of the complex64 system
                      against the complex128 one at the same state: forces,
                      density (max |drho| / max rho) and each energy term
                      (|dE_term| / |E_term|), split into the part due to
                      rounding the orbitals to complex64 and the part due to
                      the complex64 kernels

Everything runs through the C ABI; this module only schedules calls and
reduces the returned host arrays.

    python -m paper_0812_2801_gb300.precision --mu 1 10 50 --steps 1000
"""

from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import emd, inputs


def _rel_force_err(F: np.ndarray, F_ref: np.ndarray) -> float:
    scale = float(np.max(np.linalg.norm(F_ref, axis=1)))
    return float(np.max(np.linalg.norm(F - F_ref, axis=1)) / scale)


def _drift(E: np.ndarray, steps: np.ndarray) -> dict:
    e0 = abs(float(E[0]))
    slope = float(np.polyfit(steps.astype(np.float64), E, 1)[0]) if len(E) > 1 else 0.0
    return {"E0": float(E[0]), "E_end": float(E[-1]),
            "drift_rel": abs(float(E[-1] - E[0])) / e0,
            "max_dev_rel": float(np.max(np.abs(E - E[0]))) / e0,
            "slope_rel_1000": abs(slope) * 1000.0 / e0}


def _errors(a, b) -> dict:
    """Relative errors of system ``a`` against system ``b`` (same state)."""
    ea, eb = a.energy(), b.energy()
    rho_a = a.state(want_psi=False, want_rho=True)[3]
    rho_b = b.state(want_psi=False, want_rho=True)[3]
    out = {"forces": _rel_force_err(a.forces(), b.forces()),
           "rho": float(np.max(np.abs(rho_a - rho_b)) / np.max(np.abs(rho_b)))}
    for k in ("kin_e", "nl", "es", "xc", "ks", "total"):
        out[k] = abs(ea[k] - eb[k]) / max(abs(eb[k]), 1e-300)
    return out


def _state_errors(step: int, s32, s64r, s64) -> dict:
    """Errors at one state of the complex128 run: ``s32`` (complex64 system
    loaded with it) and ``s64r`` (complex128 system loaded with the same
    orbitals rounded to complex64) against ``s64``.  ``all`` is the complex64
    form's error; ``rounding`` the part due to storing the orbitals in
    complex64 at all; ``eval`` the part due to the complex64 kernels."""
    return {"step": step, "all": _errors(s32, s64), "rounding": _errors(s64r, s64),
            "eval": _errors(s32, s64r)}


def compare(sysin, n_steps: int, every: int = 10, state_every: int = 100) -> dict:
    """Run ``sysin`` for ``n_steps`` MD steps in both precisions, sampling the
    energy and forces every ``every`` steps and the same-state force error
    every ``state_every`` steps (and at the end)."""
    import torch
    s64 = emd.System(sysin, emd.EMD_FP64)
    s32 = emd.System(sysin, emd.EMD_FP32_ORBITALS)
    probe = emd.System(sysin, emd.EMD_FP32_ORBITALS)
    probe64 = emd.System(sysin, emd.EMD_FP64)
    emd.emd_set_orbitals_c64(probe64.handle, sysin.psi.astype(np.complex64))
    t = [0]
    E64 = [s64.energy()["total"]]
    E32 = [s32.energy()["total"]]
    f_traj = [_rel_force_err(s32.forces(), s64.forces())]
    f_state = [(0, _rel_force_err(probe.forces(), s64.forces()))]
    state_errors = [_state_errors(0, probe, probe64, s64)]
    n_elec = [s32.energy()["n_elec"]]
    ms64 = ms32 = 0.0
    done = 0
    while done < n_steps:
        k = min(every, n_steps - done)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64.propagate(k)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s32.propagate(k)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ms64 += (t1 - t0) * 1e3
        ms32 += (t2 - t1) * 1e3
        done += k
        e64, e32 = s64.energy(), s32.energy()
        t.append(done)
        E64.append(e64["total"])
        E32.append(e32["total"])
        n_elec.append(e32["n_elec"])
        F64 = s64.forces()
        f_traj.append(_rel_force_err(s32.forces(), F64))
        if done % state_every == 0 or done == n_steps:
            R, V, psi, _ = s64.state(want_psi=True, want_rho=False)
            emd.emd_set_ions(probe.handle, R, V)
            emd.emd_set_orbitals(probe.handle, psi)
            emd.emd_set_ions(probe64.handle, R, V)
            emd.emd_set_orbitals_c64(probe64.handle, psi.astype(np.complex64))
            f_state.append((done, _rel_force_err(probe.forces(), F64)))
            state_errors.append(_state_errors(done, probe, probe64, s64))
            del psi
    for s in (s64, s32, probe, probe64):
        s.close()
    steps = np.asarray(t)
    E64, E32 = np.asarray(E64), np.asarray(E32)
    return {
        "workload": sysin.name, "mu": sysin.mu, "dt": sysin.dt, "steps": n_steps,
        "sample_every": every,
        "fp64": dict(_drift(E64, steps), ms_per_step=ms64 / n_steps),
        "fp32": dict(_drift(E32, steps), ms_per_step=ms32 / n_steps,
                     n_elec_dev=float(np.max(np.abs(np.asarray(n_elec) - n_elec[0])))),
        "energy_diff_end_rel": abs(float(E32[-1] - E64[-1])) / abs(float(E64[0])),
        "force_err_traj_max": float(max(f_traj)),
        "force_err_traj_end": float(f_traj[-1]),
        "force_err_state": [{"step": k, "err": e} for k, e in f_state],
        "state_errors": state_errors,
    }


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--mu", type=float, nargs="+", default=[1.0, 10.0, 50.0])
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--state-every", type=int, default=250)
    ap.add_argument("--out", default=None, help="also write the results here (JSON)")
    args = ap.parse_args(argv)
    emd.load()
    results = []
    for mu in args.mu:
        r = compare(inputs.precision_c96(mu=mu), args.steps, args.every, args.state_every)
        results.append(r)
        print(json.dumps({k: v for k, v in r.items()
                          if k not in ("force_err_state", "state_errors")}), flush=True)
        print(json.dumps({"mu": mu, "state_errors": r["state_errors"]}), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(results, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
