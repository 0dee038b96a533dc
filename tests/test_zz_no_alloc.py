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


@pytest.mark.parametrize("N", [2, 8])
def test_noalloc_mass_smallest_and_largest_phase_count(N):
    """N = 2 and N = 8 (the whole 512 x 9 scratch array in use): the volumes
    of synthetic phase fields against an FP64 sum on the host, two calls in
    a row with different fields; a planted out-of-range value raises the
    flag."""
    import torch
    from paper_2306_06983_gb300.build import build
    from paper_2306_06983_gb300 import nlbm

    build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(40 + N)
    n_nodes = 300 * 217   # ragged: not a multiple of the reduction's block size
    mass = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
    flag = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        phi = rng.dirichlet(np.ones(N), size=n_nodes).T[:N - 1].astype(np.float32)
        dphi = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
        st = nlbm.nlbm_phase_mass_noalloc(dphi.data_ptr(), N, n_nodes, mass.data_ptr(), flag.data_ptr(), stream)
        assert st == nlbm.NLBM_OK
        torch.cuda.synchronize()
        p64 = phi.astype(np.float64)
        ref = np.concatenate([p64.sum(axis=1), [(1.0 - p64.sum(axis=0)).sum()]])
        np.testing.assert_allclose(mass.cpu().numpy(), ref, rtol=1e-12, atol=1e-9)
        assert int(flag.item()) == 0, call
    phi[0, 1234] = 7.0
    dphi = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
    st = nlbm.nlbm_phase_mass_noalloc(dphi.data_ptr(), N, n_nodes, mass.data_ptr(), flag.data_ptr(), stream)
    assert st == nlbm.NLBM_OK
    torch.cuda.synchronize()
    assert int(flag.item()) == 1


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
    # below the range, and missing pointers: rejected before any GPU work
    assert nlbm.nlbm_phase_mass_noalloc(buf.data_ptr(), 1, 4, buf.data_ptr(), flag.data_ptr(), 0) == nlbm.NLBM_EINVAL
    assert nlbm.nlbm_phase_mass_noalloc(buf.data_ptr(), 3, 0, buf.data_ptr(), flag.data_ptr(), 0) == nlbm.NLBM_EINVAL
    assert nlbm.nlbm_phase_mass_noalloc(0, 3, 4, buf.data_ptr(), flag.data_ptr(), 0) == nlbm.NLBM_EINVAL
    assert nlbm.nlbm_phase_mass_noalloc(buf.data_ptr(), 3, 4, 0, flag.data_ptr(), 0) == nlbm.NLBM_EINVAL
    assert nlbm.nlbm_phase_mass_noalloc(buf.data_ptr(), 3, 4, buf.data_ptr(), 0, 0) == nlbm.NLBM_EINVAL
