"""The Poisson entry point that allocates nothing (emd_poisson_static).

It exists for callers that cannot call cudaMalloc -- code running while a
CUDA graph is being captured, applications whose device memory belongs to
another allocator or a fixed budget, latency-critical loops where an
allocation would synchronise the device.  Its FFT work arrays live in a
fixed-size static device array, so it handles grids up to 64^3.

The tests check it, on two calls in a row each time, against the Hartree
potential the library computes with its own (allocating) solver for the same
density, and against the oracle's spectral Poisson solve (numpy FFT) on an
even grid, an odd grid and the largest grid it accepts; and that a grid above
the limit is refused with a message.
"""
import numpy as np
import pytest

from oracle import emd_oracle as O
from paper_0812_2801_gb300 import emd, inputs

pytestmark = pytest.mark.gpu


def _solve_twice(n, h, charge):
    import torch
    # the test owns these buffers; the entry point itself allocates nothing
    q_d = torch.from_numpy(np.ascontiguousarray(charge)).to("cuda")
    out_d = torch.empty_like(q_d)
    outs = []
    for _ in range(2):
        out_d.fill_(float("nan"))
        emd.emd_poisson_static(n, h, q_d.data_ptr(), out_d.data_ptr())
        torch.cuda.synchronize()
        outs.append(out_d.cpu().numpy())
    return outs


def test_poisson_static_matches_library_hartree_potential():
    s = inputs.small_system(n=24, h=0.3, fd_order=4, n_atoms=2, seed=13)
    sysg = emd.System(s)
    _, _, _, rho = sysg.state(want_psi=False)
    v_h = emd.emd_get_potentials(sysg.handle, s.n)["v_h"]
    sysg.close()
    for v in _solve_twice(s.n, s.h, rho):
        assert np.max(np.abs(v - v_h)) <= 1e-12 * np.max(np.abs(v_h))


@pytest.mark.parametrize("n", [24, 45, 64])
def test_poisson_static_matches_oracle(n):
    """Against the oracle's v(G) = 4 pi n(G)/|G|^2, v(0) = 0 (numpy FFT), on a
    seeded random charge; FP64 FFTs of either kind agree to ~1e-14."""
    h = 0.3
    rng = np.random.default_rng(100 + n)
    charge = rng.normal(size=(n, n, n))
    ref = O.poisson(charge, h)
    for v in _solve_twice(n, h, charge):
        assert np.max(np.abs(v - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_poisson_static_rejects_grids_above_the_limit():
    import torch
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(emd.EmdError) as ei:
        emd.emd_poisson_static(65, 0.3, buf.data_ptr(), buf.data_ptr())
    assert ei.value.code == emd.EMD_EINVAL
    assert "64" in str(ei.value)
