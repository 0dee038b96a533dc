"""GPU test of the static droplets (Sec. 4.1, Table 1) through the C ABI.

Drops of radius 20 (eps = 5, sigma_pq = 0.01) of phases 1..N-1 at x = -100,
0, 100 on the centre line of the periodic 300x100 domain, phase N around
them, densities 1000:500:100:1 and viscosities 100:50:10:0.1, mobility 0.01
(the paper does not print it; with 0.01 the FP64 oracle reproduces the
table to 0.02 %).  After 10,000 FP32 steps, for the quaternary, ternary and
binary systems and for Model A (n = 1, 2) and Model B:
  - the relative L1 errors of the phase fields against the initial tanh
    profiles (the continuum equilibrium) match the paper's printed values
    (tests/golden/static_droplets_table1.txt) within 0.5 %;
  - the three models give the same errors, as the table prints them;
  - spurious velocities stay below 1e-6 (the paper's histograms peak near
    1e-7) and every phase keeps its volume;
  - with bfloat16 or binary16 population storage the errors stay within
    about twice the shift the oracle's noise model of that storage gives;
  - the quaternary system with phase 3 absent reproduces the ternary one
    (the paper's reduction check, Fig. 4) to FP32 round-off: the two lattice
    sizes run different instruction sequences."""

import os

import numpy as np
import pytest

from paper_2306_06983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "static_droplets_table1.txt")
STEPS = 10000
MODELS = [("A", 1.0), ("A", 2.0), ("B", 1.0)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2306_06983_gb300.build import build
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    torch.cuda.set_device(0)


def golden():
    t = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            n, k, e = line.split()
            t.setdefault(int(n), []).append(float(e))
    return t


def run(N, model, n, absent=(), storage=None):
    """Runs the N-phase system; phases listed in absent (1-based, < N) are
    zero everywhere.  Returns the full fields (N rows), the analytical
    fields, max |u|, and the initial and final phase masses."""
    from paper_2306_06983_gb300.nlbm import Simulation
    p, phi0 = W.static_droplets(N, model=model, model_a_n=n, absent=absent)
    sim = Simulation(dict(p, storage=storage) if storage else p)
    sim.set_phi(phi0)
    m0 = sim.phase_mass()
    sim.step(STEPS)
    phi, u, _ = (t.cpu().numpy().astype(np.float64) for t in sim.moments())
    m1 = sim.phase_mass()
    sim.close()
    full = np.concatenate([phi, (1.0 - phi.sum(0))[None]])
    ana = np.concatenate([phi0, (1.0 - phi0.sum(0))[None]])
    return full, ana, np.abs(u).max(), m0, m1


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("N", [4, 3, 2])
def test_table1_errors(N):
    want = np.array(golden()[N])
    errs = {}
    for model, n in MODELS:
        full, ana, umax, m0, m1 = run(N, model, n)
        e = np.array([rel_l1(full[k], ana[k]) for k in range(N)])
        print(f"\nN={N} {model} n={n}: E_L1 {' '.join(f'{v:.5e}' for v in e)}  max|u| {umax:.2e}")
        np.testing.assert_allclose(e, want, rtol=5e-3)
        assert umax < 1e-6
        assert np.all(np.abs(m1 - m0) <= 1e-6 * np.abs(m0))
        errs[(model, n)] = e
    for k, e in errs.items():
        np.testing.assert_allclose(e, errs[("B", 1.0)], rtol=1e-3, err_msg=str(k))


@pytest.mark.parametrize("model,n", [("A", 1.0), ("B", 1.0)])
def test_absent_phase_reduces_to_ternary(model, n):
    q, _, _, _, _ = run(4, model, n, absent=(3,))
    t, _, _, _, _ = run(3, model, n)
    assert np.abs(q[2]).max() == 0.0
    d = max(np.abs(q[0] - t[0]).max(), np.abs(q[1] - t[1]).max(), np.abs(q[3] - t[2]).max())
    print(f"\n{model} n={n}: max |phi(N=4, phase 3 absent) - phi(N=3)| = {d:.2e}")
    assert d < 4e-6


@pytest.mark.parametrize("storage,rtol", [("bf16", 1.5e-2), ("f16", 2.5e-2)])
@pytest.mark.parametrize("N", [4, 2])
def test_table1_errors_16bit_storage(N, storage, rtol):
    """The same errors with the populations stored as 16-bit deviations
    (Model B).  The storage rounding moves them.  On this 300x100 domain the
    oracle's FP32 noise model with the same rounding gives, for the binary
    drop, E_L1 = 2.604e-3 (bfloat16, +0.65 % from the printed value) and
    2.618e-3 (binary16, +1.17 %).  Binary16 quantises the small velocities
    of the far field to its subnormal spacing, 2^-24.  The bounds are about
    twice those offsets.  The spurious flow stays below 5e-6."""
    want = np.array(golden()[N])
    full, ana, umax, m0, m1 = run(N, "B", 1.0, storage=storage)
    e = np.array([rel_l1(full[k], ana[k]) for k in range(N)])
    print(f"\nN={N} {storage}: E_L1 {' '.join(f'{v:.5e}' for v in e)}  max|u| {umax:.2e}")
    np.testing.assert_allclose(e, want, rtol=rtol)
    assert umax < 5e-6
    assert np.all(np.abs(m1 - m0) <= 1e-6 * np.abs(m0))


def test_table1_as_one_ensemble():
    """The quaternary system under Model A (n = 1, 2) and Model B as the
    three members of one ensemble (one persistent launch per step advances
    all of them): each member gives the printed errors and, after 10,000
    steps, the same bits as the simulation run alone (a member takes the
    same code path), with its volumes conserved."""
    import torch
    from paper_2306_06983_gb300.nlbm import Batch
    want = np.array(golden()[4])
    members = [W.static_droplets(4, model=m, model_a_n=n) for m, n in MODELS]
    b = Batch([p for p, _ in members])
    for k, (_, phi0) in enumerate(members):
        b.set_phi(k, phi0.astype(np.float32))
    m0 = [b.phase_mass(k) for k in range(len(members))]
    b.step(STEPS)
    got = []
    for k in range(len(members)):
        phi, u, _ = (t.cpu().numpy().astype(np.float64) for t in b.moments(k))
        got.append((np.concatenate([phi, (1.0 - phi.sum(0))[None]]), np.abs(u).max(), b.phase_mass(k)))
    b.close()
    torch.cuda.empty_cache()
    for k, (model, n) in enumerate(MODELS):
        full, umax, m1 = got[k]
        alone, ana, _, _, _ = run(4, model, n)
        e = np.array([rel_l1(full[j], ana[j]) for j in range(4)])
        d = np.abs(full - alone).max()
        print(f"\nensemble member {model} n={n}: E_L1 {' '.join(f'{v:.5e}' for v in e)}, "
              f"max|u| {umax:.2e}, |member - alone| {d:.2e}")
        np.testing.assert_allclose(e, want, rtol=5e-3)
        assert umax < 1e-6 and d == 0.0
        assert np.all(np.abs(m1 - m0[k]) <= 1e-6 * np.abs(m0[k]))
