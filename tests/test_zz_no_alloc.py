"""The Poisson entry point that allocates nothing (emd_poisson_static).

It exists for callers that cannot call cudaMalloc -- code running while a
CUDA graph is being captured, applications whose device memory belongs to
another allocator or a fixed budget, latency-critical loops where an
allocation would synchronise the device.  Its FFT work arrays live in a
fixed-size static device array, so it handles grids up to 64^3.

The test checks it against the Hartree potential the library computes with
its own (allocating) solver for the same density, on two calls in a row, and
that a grid above the limit is refused with a message.
"""
import ctypes

import numpy as np
import pytest

from paper_0812_2801_gb300 import emd, inputs

pytestmark = pytest.mark.gpu


def test_poisson_static_matches_library_hartree_potential():
    import torch
    s = inputs.small_system(n=24, h=0.3, fd_order=4, n_atoms=2, seed=13)
    sysg = emd.System(s)
    _, _, _, rho = sysg.state(want_psi=False)
    v_h = emd.emd_get_potentials(sysg.handle, s.n)["v_h"]
    sysg.close()
    # the test owns these buffers; the entry point itself allocates nothing
    rho_d = torch.from_numpy(rho).to("cuda")
    out_d = torch.empty_like(rho_d)
    for _ in range(2):
        out_d.fill_(float("nan"))
        emd.emd_poisson_static(s.n, s.h, rho_d.data_ptr(), out_d.data_ptr())
        torch.cuda.synchronize()
        v = out_d.cpu().numpy()
        assert np.max(np.abs(v - v_h)) <= 1e-12 * np.max(np.abs(v_h))


def test_poisson_static_rejects_grids_above_the_limit():
    import torch
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(emd.EmdError) as ei:
        emd.emd_poisson_static(65, 0.3, buf.data_ptr(), buf.data_ptr())
    assert ei.value.code == emd.EMD_EINVAL
    assert "64" in str(ei.value)
