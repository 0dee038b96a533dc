"""The allocation-free volume reduction (nlbm_phase_mass_noalloc) against the
workspace-backed one (nlbm_phase_mass) on the same phase fields.

Some callers cannot give the library any device memory for scratch -- they
run where cudaMalloc is not allowed or not affordable -- so this entry point
keeps its partial sums in a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test."""

import numpy as np
import pytest

from paper_2306_06983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_mass_matches_workspace_mass_twice_in_a_row():
    import torch
    from paper_2306_06983_gb300.build import build
    from paper_2306_06983_gb300 import nlbm
    from paper_2306_06983_gb300.nlbm import Simulation

    assert torch.cuda.is_available(), "GPU test needs CUDA"
    build()
    torch.cuda.set_device(0)
    p, phi0 = W.disks_256("B")
    N, plane = p["n_phases"], p["nx"] * p["ny"]
    sim = Simulation(p)
    sim.set_phi(phi0.astype(np.float32))
    stream = torch.cuda.current_stream().cuda_stream
    mass = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
    flag = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for steps in (3, 11):                      # two calls in a row, different fields
        sim.step(steps)
        phi = sim.moments()[0]                 # [N, ny, nx]; the first N-1 planes are inputs
        ref = sim.phase_mass()
        st = nlbm.nlbm_phase_mass_noalloc(phi.data_ptr(), N, plane, mass.data_ptr(),
                                          flag.data_ptr(), stream)
        assert st == nlbm.NLBM_OK
        torch.cuda.synchronize()
        np.testing.assert_allclose(mass.cpu().numpy(), ref, rtol=1e-12, atol=0)
        assert int(flag.item()) == 0
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2306_06983_gb300.build import build
    from paper_2306_06983_gb300 import nlbm

    build()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = nlbm.nlbm_phase_mass_noalloc(buf.data_ptr(), 9, 4, buf.data_ptr(), flag.data_ptr(), 0)
    assert st == nlbm.NLBM_EINVAL
    st = nlbm.nlbm_phase_mass_noalloc(buf.data_ptr(), 3, (1 << 28) + 1, buf.data_ptr(),
                                      flag.data_ptr(), 0)
    assert st == nlbm.NLBM_EINVAL
