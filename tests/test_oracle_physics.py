"""Dynamic pins of the FP64 oracle: invariants and closed forms the paper
claims for the method (volume conservation, reduction consistency, Model A
and Model B coinciding in binary regions, the static droplets' errors
printed in Table 1, symmetry under relabelling the solved phases, a
stationary flat interface, Laplace's law) plus the oracle's own sensitivity
to FP32-level input rounding, which sets what element-wise parity can mean
after many steps."""

import os

import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2306_06983_gb300 import workloads as W


@pytest.mark.parametrize("model,n", [("A", 1.0), ("A", 2.0), ("B", 1.0)])
def test_mass_conserved_droplets_64(oracle_built, model, n):
    """Eq. (1) with sum phi = 1: every phase volume is conserved; the LB with
    mass-conserving collision and periodic streaming keeps it to round-off
    over 2000 steps on the 64x64 three-phase droplet case."""
    p, phi0 = W.droplets_64(model, n)
    s = OracleSim(p, phi0)
    m0 = s.phase_mass()
    s.step(2000)
    m1 = s.phase_mass()
    assert np.all(np.abs(m1 - m0) / m0 < 1e-11), (m0, m1)


def test_mass_conserved_with_walls(oracle_built):
    """Half-way bounce-back walls (Sec. 4) are no-flux: volumes conserved."""
    p, phi0 = W.random_smooth(37, 29, 4, seed=11, model="B", wall_y=True, wall_x=True)
    s = OracleSim(p, phi0)
    m0 = s.phase_mass()
    s.step(400)
    m1 = s.phase_mass()
    assert np.all(np.abs(m1 - m0) < 1e-12 * p["nx"] * p["ny"]), (m0, m1)


@pytest.mark.parametrize("model,n", [("A", 1.0), ("A", 2.0), ("B", 1.0)])
@pytest.mark.parametrize("walls", [False, True])
def test_reduction_consistency_bitwise(oracle_built, model, n, walls):
    """Reduction consistency (Sec. 1, Sec. 4.1): a three-phase run whose phase
    2 is absent everywhere is the two-phase run, exactly -- phase 2 stays 0
    and phases 1, 3 equal the N = 2 phases 1, 2 bit for bit."""
    nx, ny = 48, 40
    d = W.disk(nx, ny, 20.3, 17.6, 9, 4.0, not walls, not walls)
    rho3, mu3 = [1.0, 7.0, 3.0], [0.2, 0.9, 0.1]
    sig3 = [[0, 0.013, 0.01], [0.013, 0, 0.017], [0.01, 0.017, 0]]
    p3 = W.base_params(nx, ny, 3, model=model, model_a_n=n, rho=rho3, mu=mu3, sigma=sig3,
                       wall_x=walls, wall_y=walls)
    p2 = W.base_params(nx, ny, 2, model=model, model_a_n=n, rho=[1.0, 3.0], mu=[0.2, 0.1],
                       sigma=[[0, 0.01], [0.01, 0]], wall_x=walls, wall_y=walls)
    s3 = OracleSim(p3, np.stack([d, np.zeros_like(d)]))
    s2 = OracleSim(p2, np.stack([d]))
    s3.step(300)
    s2.step(300)
    a3, a2 = s3.moments(), s2.moments()
    assert np.all(a3[0][1] == 0.0)
    np.testing.assert_array_equal(a3[0][0], a2[0][0])
    np.testing.assert_array_equal(a3[0][2], a2[0][1])
    np.testing.assert_array_equal(a3[1], a2[1])
    np.testing.assert_array_equal(a3[2], a2[2])


def test_two_phase_models_coincide(oracle_built):
    """Sec. 2.1: for N = 2 Model A (any n) and Model B are the same equation;
    the runs agree to round-off (10 steps, before the bulk sensitivity at the
    drop centre has had time to amplify rounding)."""
    p = W.base_params(64, 64, 2, sigma=0.01)
    d = W.disk(64, 64, 31.4, 32.7, 12, 4.0)
    runs = []
    for model, n in [("B", 1.0), ("A", 1.0), ("A", 2.0), ("A", 0.5)]:
        s = OracleSim(dict(p, model=model, model_a_n=n), np.stack([d]))
        s.step(10)
        runs.append(s.moments())
    for r in runs[1:]:
        assert np.abs(r[0] - runs[0][0]).max() < 1e-12
        assert np.abs(r[1] - runs[0][1]).max() < 1e-14


def test_models_coincide_in_binary_regions(oracle_built):
    """Sec. 4.1, Table 1: three separated drops (phases 1-3) in phase 4 -- every
    region is binary, where Model A (n = 1, 2) and Model B coincide (Eq. (9)
    with exact equilibrium norms); the printed E_L1 of the drops are identical
    across models to five digits.  Here: identical to round-off after 10
    steps, E_L1 after 500 steps equal across models to 1 %, and of the
    printed order (1e-3)."""
    nx, ny = 240, 80
    ds = [W.disk(nx, ny, cx, 40, 16, 4.0) for cx in (40, 120, 200)]
    full = np.stack(ds + [1 - sum(ds)])
    a10, el1 = {}, {}
    for model, n in [("A", 1.0), ("A", 2.0), ("B", 1.0)]:
        p = W.base_params(nx, ny, 4, model=model, model_a_n=n, sigma=0.01)
        s = OracleSim(p, np.stack(ds))
        s.step(10)
        a10[(model, n)] = s.moments()[0]
        s.step(490)
        a = s.moments()[0]
        el1[(model, n)] = np.array([np.abs(a[k] - full[k]).sum() / np.abs(full[k]).sum()
                                    for k in range(4)])
    ref = a10[("B", 1.0)]
    for k, v in a10.items():
        assert np.abs(v - ref).max() < 1e-12, k
    for k, v in el1.items():
        np.testing.assert_allclose(v, el1[("B", 1.0)], rtol=1e-2)
        assert np.all(v[:3] > 5e-4) and np.all(v[:3] < 1e-2)


def test_static_drop_matches_table1(oracle_built):
    """Sec. 4.1, Table 1 (tests/golden/static_droplets_table1.txt): a drop of
    radius 20 (eps = 5, sigma = 0.01, densities 1000:1, viscosities 100:0.1,
    mobility 0.01 -- the paper does not print it) centred between nodes as
    in the paper's 300x100 domain, here on an 80x80 box (the tanh tails at
    the images are below 1e-7).  After 4000 steps its relative L1 error is
    the printed drop value within 1e-3.  The drops of the three systems are
    separated, so each has this error, and phase N = 1 - sum phi_p carries
    their absolute errors over the rest of the 300x100 domain:
    E_N = k E_1 S_1 / (30000 - k S_1) with k drops of area S_1 -- the
    printed phase-N values within 1e-3 as well."""
    n = 80
    c = np.arange(n) + 0.5 - n / 2
    phi = 0.5 + 0.5 * np.tanh((20.0 - np.sqrt(c[None, :] ** 2 + c[:, None] ** 2)) / 2.5)
    p = W.base_params(n, n, 2, model="B", eps=5.0, mobility=0.01, rho=[1000.0, 1.0],
                      mu=[100.0, 0.1], sigma=0.01)
    s = OracleSim(p, phi[None])
    s.step(4000)
    e1 = np.abs(s.moments()[0][0] - phi).sum() / phi.sum()
    S1 = phi.sum()
    golden = os.path.join(os.path.dirname(__file__), "golden", "static_droplets_table1.txt")
    rows = [l.split() for l in open(golden) if l.strip() and not l.startswith("#")]
    for system, phase, printed in ((int(a), int(b), float(v)) for a, b, v in rows):
        k = system - 1
        want = e1 if phase < system else k * e1 * S1 / (300 * 100 - k * S1)
        print(f"system {system} phase {phase}: {want:.5e} (printed {printed:.4e})")
        assert abs(want / printed - 1) < 1e-3


def test_flat_interface_stationary(oracle_built):
    """Eq. (5): the flat profile 0.5 + 0.5 tanh(2x/eps) at rest is an
    equilibrium of the continuum equations.  The lattice settles to its own
    discrete profile, E_L1 = 1.78e-3 from the tanh at eps = 4 (below 2e-3).
    That profile is stationary: from 2000 to 4000 steps it moves by
    E_L1 = 2e-7 (bound 1e-6), and it drives no flow (max |u| < 1e-7)."""
    nx, ny = 16, 64
    p = W.base_params(nx, ny, 2, model="B", sigma=0.01)
    b = W.flat_band(nx, ny, 16, 48, 4.0)
    s = OracleSim(p, np.stack([b]))
    s.step(2000)
    phi, u, _ = s.moments()
    assert np.abs(phi[0] - b).sum() / np.abs(b).sum() < 2e-3
    assert np.abs(u).max() < 1e-7
    s.step(2000)
    phi2 = s.moments()[0]
    assert np.abs(phi2[0] - phi[0]).sum() / np.abs(b).sum() < 1e-6


@pytest.mark.parametrize("N", [2, 3])
def test_laplace_law(oracle_built, N):
    """Static drop: the pressure jump equals sigma/R (2D Laplace law) within
    10 % for R = 12, eps = 4 after 3000 steps.  N = 3 places two drops of
    phases 2 and 3 with different sigma against the phase-1 matrix."""
    if N == 2:
        nx = ny = 64
        p = W.base_params(nx, ny, 2, model="B", sigma=0.01)
        d = W.disk(nx, ny, 32, 32, 12, 4.0)
        s = OracleSim(p, np.stack([1 - d]))
        s.step(3000)
        P = s.moments()[2]
        assert abs((P[32, 32] - P[0, 0]) / (0.01 / 12) - 1) < 0.1
    else:
        nx, ny = 128, 64
        sig = [[0, 0.01, 0.02], [0.01, 0, 0.015], [0.02, 0.015, 0]]
        p = W.base_params(nx, ny, 3, model="B", sigma=sig)
        d2 = W.disk(nx, ny, 32, 32, 12, 4.0)
        d3 = W.disk(nx, ny, 96, 32, 12, 4.0)
        s = OracleSim(p, np.stack([1 - d2 - d3, d2]))
        s.step(3000)
        P = s.moments()[2]
        far = P[0, 64]
        assert abs((P[32, 32] - far) / (0.01 / 12) - 1) < 0.1
        assert abs((P[32, 96] - far) / (0.02 / 12) - 1) < 0.1


def test_transpose_symmetry(oracle_built):
    """The method is isotropic: a transposed initial state yields the
    transposed state with the velocity components swapped (catches a wrong
    velocity/weight table or a transposed stencil index)."""
    p, phi0 = W.random_smooth(40, 40, 4, seed=5, model="B")
    s = OracleSim(p, phi0)
    st = OracleSim(p, np.ascontiguousarray(phi0.transpose(0, 2, 1)))
    s.step(10)
    st.step(10)
    a, b = s.moments(), st.moments()
    np.testing.assert_allclose(b[0], a[0].transpose(0, 2, 1), atol=1e-13)
    np.testing.assert_allclose(b[1][0], a[1][1].T, atol=1e-15)
    np.testing.assert_allclose(b[1][1], a[1][0].T, atol=1e-15)
    np.testing.assert_allclose(b[2], a[2].T, atol=1e-15)


@pytest.mark.parametrize("model,n", [("B", 1.0), ("A", 1.0), ("A", 2.0)])
@pytest.mark.parametrize("perm", [(2, 1, 0, 3), (1, 2, 0, 3), (0, 2, 1, 3)])
def test_phase_relabelling_symmetry(oracle_built, perm, model, n):
    """Both models treat the phases alike: Model B through pairwise normals
    (Sec. 2.1, Eqs. (3)-(4)), and Model A through one Lagrange multiplier
    shared by all phases (Eq. (2)).  Relabelling the solved phases, with the
    densities, viscosities and tensions permuted to match, relabels the
    result up to rounding order.  This catches a phase-asymmetric term, such
    as a wrong index in the pair loops.  Exchanging a solved phase with the
    unsolved phase N is not an exact symmetry of the scheme.  With all N
    sets solved, sum phi would drift where div u != 0 (the weakly
    compressible flow advects it like a passive scalar), so the closure
    phi_N = 1 - sum phi_p differs from what phase N's own set would give.
    That exchange moves phi by about 1e-3 after 10 steps here."""
    p, phi0 = W.random_smooth(40, 36, 4, seed=41, model=model, model_a_n=n)
    full0 = np.concatenate([phi0, (1.0 - phi0.sum(0))[None]])
    pi = list(perm)
    sig = np.asarray(p["sigma"])
    q = dict(p, rho=[p["rho"][k] for k in pi], mu=[p["mu"][k] for k in pi],
             sigma=sig[np.ix_(pi, pi)].tolist())
    a, b = OracleSim(p, phi0), OracleSim(q, full0[pi][:3])
    a.step(10)
    b.step(10)
    (pa, ua, Pa), (pb, ub, Pb) = a.moments(), b.moments()
    np.testing.assert_allclose(pb, pa[pi], atol=1e-13, rtol=0)
    np.testing.assert_allclose(ub, ua, atol=1e-15, rtol=0)
    np.testing.assert_allclose(Pb, Pa, atol=1e-15, rtol=0)


def test_self_sensitivity_envelope(oracle_built):
    """The oracle against itself: rounding only the initial fields to FP32
    moves phi by far more than 1e-5 after 2000 steps on the 64x64 droplets
    (the source R = a n is driven by near-zero gradients in the bulk where
    phi overshoots 1), while velocity, the mean |d phi| and the masses stay
    close.  Element-wise phi parity after many steps is therefore judged
    against this envelope, not against 1e-5."""
    p, phi0 = W.droplets_64("B")
    s0 = OracleSim(p, phi0)
    s1 = OracleSim(p, phi0.astype(np.float32).astype(np.float64))
    s0.step(2000)
    s1.step(2000)
    a, b = s0.moments(), s1.moments()
    d = np.abs(a[0] - b[0])
    assert d.max() > 1e-4            # no FP32 path can meet 1e-5 here
    assert d.mean() < 2e-4
    assert np.abs(a[1] - b[1]).max() < 1e-5


def test_store16_noise_model(oracle_built):
    """The 16-bit-storage noise model (FP32 build only): the FP64 oracle
    refuses it; at rest on a uniform field every stored deviation is zero, so
    it equals the plain FP32 build bitwise; on droplets it conserves each
    phase's volume to FP32 round-off and, over the first steps (before the
    method's own amplification of rounding takes over), binary16 (11 bits)
    moves the result less than bfloat16 (8 bits) and more than FP32 alone."""
    import pytest as _pt
    p = W.base_params(16, 12, 3, model="B")
    flat = np.full((2, 12, 16), 0.25)
    with _pt.raises(ValueError):
        OracleSim(p, flat, store16=1)
    a = OracleSim(p, flat, fp32=True)
    b = OracleSim(p, flat, fp32=True, store16=1)
    a.step(5)
    b.step(5)
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
    p, phi0 = W.droplets_64("B")
    ref = OracleSim(p, phi0)
    ref.step(3)
    d = {}
    for mode in (1, 2):
        s = OracleSim(p, phi0, fp32=True, store16=mode)
        m0 = s.phase_mass()
        s.step(3)
        # the noise model sums its volumes in FP32 (4096 terms): 1e-5 relative
        assert np.all(np.abs(s.phase_mass() - m0) / m0 < 1e-5)
        d[mode] = np.abs(s.moments()[0] - ref.moments()[0]).max()
    plain = OracleSim(p, phi0, fp32=True)
    plain.step(3)
    d0 = np.abs(plain.moments()[0] - ref.moments()[0]).max()
    assert d[1] > d[2] > d0


def test_lens_reaches_neumann_equilibrium(oracle_built):
    """A three-phase lens (phase 3) on the 1|2 interface between no-flux
    walls, equal tensions (Table 3 case (c)): after 4000 steps the cap
    heights are within 3% and the half-length within 6% of the closed form
    of Sec. 4.3 for the measured lens area (160 x 80, R = 16, eps = 4: the
    diffuse triple junction shortens the measured chord).  With a cheaper
    lower interface the lower cap is the deeper one."""
    from oracle.oracle import lens_equilibrium, measure_lens
    p, phi0 = W.lens(160, 80, 16.0, 0.01, 0.01, 0.01, model="B")
    o = OracleSim(p, phi0)
    o.step(4000)
    hd, hlo, hup, S = measure_lens(o.moments()[0])
    ad, alo, aup, _, _ = lens_equilibrium(0.01, 0.01, 0.01, S)
    assert abs(hlo / alo - 1) < 0.03 and abs(hup / aup - 1) < 0.03, (hlo, hup, alo)
    assert abs(hd / ad - 1) < 0.06, (hd, ad)
    p, phi0 = W.lens(160, 80, 16.0, 0.01, 0.006, 0.012, model="B")
    o = OracleSim(p, phi0)
    o.step(2000)
    _, hlo, hup, _ = measure_lens(o.moments()[0])
    assert hlo > 1.2 * hup


def test_lens_at_density_ratio_1000_needs_the_light_phase_unsolved(oracle_built):
    """The lens of Sec. 4.3 at the paper's densities (1 : 0.5 : 0.001 for
    lower layer, lens, upper layer; every kinematic viscosity 0.1), equal
    tensions, 160 x 64, R = 16.  With the paper's labels (the light upper
    layer is the unsolved phase N) it settles after 10,000 steps. The cap
    heights are then within 3% and the half-length within 6% of the
    closed form.  The same problem with the lens as the unsolved phase (the
    light layer solved as a phase set) diverges within 100 steps."""
    from oracle.oracle import lens_equilibrium, measure_lens
    p, phi0 = W.lens_papers_labels(160, 64, 16.0, 0.01, 0.01)
    o = OracleSim(p, phi0)
    o.step(10000)
    phi = o.moments()[0]
    assert np.isfinite(phi).all()
    hd, hlo, hup, S = measure_lens(phi[[0, 2, 1]])
    ad, alo, aup, _, _ = lens_equilibrium(0.01, 0.01, 0.01, S)
    assert abs(hlo / alo - 1) < 0.03 and abs(hup / aup - 1) < 0.03, (hlo, hup, alo)
    assert abs(hd / ad - 1) < 0.06, (hd, ad)
    q, psi0 = W.lens(160, 64, 16.0, 0.01, 0.01, 0.01)
    bad = OracleSim(dict(q, rho=[1.0, 0.001, 0.5], mu=[0.1, 1e-4, 0.05]), psi0)
    bad.step(100)
    assert not np.isfinite(bad.moments()[0]).all()
