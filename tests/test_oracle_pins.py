"""Pins of the FP64 oracle's building blocks against what the paper and the
mathematics fix independently of the oracle's own formulas.

Each test is chosen so that a plausible slip (a dropped term, a wrong sign,
weight or index, a transposed operand) in the corresponding oracle function
fails it."""

import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2306_06983_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)


def test_moment_matrix_is_the_printed_one(oracle_built):
    """Eq. (28) as printed in the paper, and M^-1 M = I."""
    M, Mi = O.mrt_matrices()
    printed = np.loadtxt(os.path.join(HERE, "golden", "moment_matrix_eq28.txt"))
    np.testing.assert_array_equal(M, printed)
    np.testing.assert_allclose(Mi @ M, np.eye(9), atol=1e-14)
    np.testing.assert_allclose(M @ Mi, np.eye(9), atol=1e-14)


@pytest.mark.parametrize("mx,my", [(1, 0), (0, 1), (2, 3), (5, 1)])
@pytest.mark.parametrize("wall", [False])
def test_isotropic_stencils_fourier_symbol(oracle_built, mx, my, wall):
    """Eq. (27) on a periodic plane wave: the discrete gradient of
    exp(i(kx x + ky y)) is i sin(kx)(2 + cos ky)/3 (x part) and the
    Laplacian symbol is (4/3)(cos kx + cos ky - 2) + (2/3)(cos kx cos ky - 1)
    (textbook symbols of the D2Q9 isotropic central differences)."""
    nx, ny = 24, 18
    kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    th = kx * x + ky * y
    for field, dfield in [(np.cos(th), -np.sin(th)), (np.sin(th), np.cos(th))]:
        g = O.field_grad(field)
        l = O.field_lap(field)
        gx_sym = np.sin(kx) * (2 + np.cos(ky)) / 3
        gy_sym = np.sin(ky) * (2 + np.cos(kx)) / 3
        lap_sym = 4 / 3 * (np.cos(kx) + np.cos(ky) - 2) + 2 / 3 * (np.cos(kx) * np.cos(ky) - 1)
        np.testing.assert_allclose(g[0], gx_sym * dfield, atol=1e-13)
        np.testing.assert_allclose(g[1], gy_sym * dfield, atol=1e-13)
        np.testing.assert_allclose(l, lap_sym * field, atol=1e-13)


def test_stencils_exact_on_quadratics_away_from_walls(oracle_built):
    """Second-order central differences are exact on quadratics:
    grad(x^2 + 3xy - y^2) = (2x + 3y, 3x - 2y), lap = 0; lap(x^2 + y^2) = 4."""
    nx = ny = 16
    x = np.arange(nx, dtype=float)[None, :] * np.ones((ny, 1))
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    f = x * x + 3 * x * y - y * y
    g = O.field_grad(f, wall_x=True, wall_y=True)
    l = O.field_lap(f, wall_x=True, wall_y=True)
    inner = (slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(g[0][inner], (2 * x + 3 * y)[inner], atol=1e-11)
    np.testing.assert_allclose(g[1][inner], (3 * x - 2 * y)[inner], atol=1e-11)
    np.testing.assert_allclose(l[inner], 0.0, atol=1e-11)
    l2 = O.field_lap(x * x + y * y, wall_x=True, wall_y=True)
    np.testing.assert_allclose(l2[inner], 4.0, atol=1e-11)


def test_wall_mirror_ghost(oracle_built):
    """Half-way wall: the ghost row equals its mirror image, so the
    y-derivative of f(y) = y at y = 0 is (1 - 0)/3 + 2(1 - 0)/12 = 1/2 and the
    normal derivative of a field symmetric about the wall vanishes."""
    nx, ny = 8, 8
    f = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    g = O.field_grad(f, wall_x=False, wall_y=True)
    np.testing.assert_allclose(g[1][0], 0.5, atol=1e-14)
    np.testing.assert_allclose(g[1][-1], 0.5, atol=1e-14)
    np.testing.assert_allclose(g[1][3], 1.0, atol=1e-14)


def test_phase_equilibrium_and_source_moments(oracle_built):
    """Eq. (19): the moments that the Taylor/Chapman-Enskog recovery of
    Eq. (1) requires -- sum f^eq = phi, sum c f^eq = phi u,
    sum c c f^eq = phi c_s^2 I; sum R_i = 0, sum c_i R_i = d_t(phi u) + c_s^2 R_p."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        phi, ux, uy = rng.uniform(-0.1, 1.1), rng.normal() * 0.05, rng.normal() * 0.05
        f = O.phase_feq(phi, ux, uy)
        assert abs(f.sum() - phi) < 1e-15
        np.testing.assert_allclose([CX @ f, CY @ f], [phi * ux, phi * uy], atol=1e-15)
        np.testing.assert_allclose([(CX * CX) @ f, (CY * CY) @ f, (CX * CY) @ f],
                                   [phi / 3, phi / 3, 0.0], atol=1e-15)
        dtx, dty, Rx, Ry = rng.normal(size=4) * 0.01
        r = O.phase_src(dtx, dty, Rx, Ry)
        assert abs(r.sum()) < 1e-16
        np.testing.assert_allclose([CX @ r, CY @ r], [dtx + Rx / 3, dty + Ry / 3], atol=1e-16)


def test_flow_equilibrium_and_forcing_moments(oracle_built):
    """Eqs. (22),(23): sum g^eq = rho_0, sum c g^eq = rho u,
    sum c_a c_b g^eq = P delta_ab + (m_a u_b + u_a m_b)/2;
    sum F_i = u.grad rho, sum c F_i = F, sum c_a c_b F_i = (M_2F)_ab."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        P, rho0, rho = rng.normal() * 0.01, rng.normal(), rng.uniform(1, 10)
        ux, uy, mx, my = rng.normal(size=4) * 0.05
        g = O.flow_geq(P, rho0, rho, ux, uy, mx, my)
        assert abs(g.sum() - rho0) < 1e-13
        np.testing.assert_allclose([CX @ g, CY @ g], [rho * ux, rho * uy], atol=1e-14)
        np.testing.assert_allclose(
            [(CX * CX) @ g, (CY * CY) @ g, (CX * CY) @ g],
            [P + mx * ux, P + my * uy, 0.5 * (mx * uy + ux * my)], atol=1e-14)
        ugr, Fx, Fy = rng.normal(size=3) * 0.01
        M2F = rng.normal(size=(2, 2)) * 0.01
        M2F = M2F + M2F.T
        Fi = O.flow_force(ugr, Fx, Fy, M2F)
        assert abs(Fi.sum() - ugr) < 1e-15
        np.testing.assert_allclose([CX @ Fi, CY @ Fi], [Fx, Fy], atol=1e-15)
        np.testing.assert_allclose([(CX * CX) @ Fi, (CY * CY) @ Fi, (CX * CY) @ Fi],
                                   [M2F[0, 0], M2F[1, 1], M2F[0, 1]], atol=1e-15)


def _params(N, model, n=1.0, eps=4.0, sigma=None, rng=None):
    from paper_2306_06983_gb300.workloads import base_params
    if sigma is None:
        sigma = 0.01
    return base_params(4, 4, N, model=model, model_a_n=n, eps=eps, sigma=sigma)


@pytest.mark.parametrize("model,n", [("A", 1.0), ("A", 2.0), ("A", 0.5), ("B", 1.0)])
def test_source_two_phase_reduces_to_conservative_ac(oracle_built, model, n):
    """Sec. 2.1: for N = 2 both models equal the two-phase conservative AC
    source 4 phi (1 - phi)/eps * grad phi/|grad phi|."""
    rng = np.random.default_rng(2)
    p = _params(2, model, n)
    for _ in range(20):
        phi = rng.uniform(0.01, 0.99)
        gvec = rng.normal(size=2)
        R = O.point_source(p, np.array([phi, 1 - phi]), np.array([gvec, -gvec]))
        expect = 4 * phi * (1 - phi) / 4.0 * gvec / np.linalg.norm(gvec)
        np.testing.assert_allclose(R[0], expect, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(R[1], -expect, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("model,n", [("A", 1.0), ("A", 3.0), ("B", 1.0)])
@pytest.mark.parametrize("N", [3, 4, 5])
def test_source_conserves_volume(oracle_built, model, n, N):
    """Sec. 2.1: both sources conserve volume, sum_p R_p = 0, whenever
    sum phi = 1 and sum grad phi = 0."""
    rng = np.random.default_rng(3 + N)
    p = _params(N, model, n)
    for _ in range(20):
        phi = rng.dirichlet(np.ones(N))
        g = rng.normal(size=(N, 2))
        g -= g.mean(axis=0)
        R = O.point_source(p, phi, g)
        np.testing.assert_allclose(R.sum(axis=0), 0.0, atol=1e-15)


@pytest.mark.parametrize("model,n", [("A", 1.0), ("A", 2.0), ("B", 1.0)])
def test_source_reduction_consistent(oracle_built, model, n):
    """Sec. 1/2.1 reduction consistency: an absent phase (phi_q = 0,
    grad phi_q = 0) receives no source, and the others see the (N-1)-phase
    source."""
    rng = np.random.default_rng(4)
    p3, p2 = _params(3, model, n), _params(2, model, n)
    for _ in range(20):
        a = rng.uniform(0.01, 0.99)
        g = rng.normal(size=2)
        R3 = O.point_source(p3, np.array([a, 0.0, 1 - a]), np.array([g, [0, 0], -g]))
        R2 = O.point_source(p2, np.array([a, 1 - a]), np.array([g, -g]))
        np.testing.assert_array_equal(R3[1], [0.0, 0.0])
        np.testing.assert_allclose(R3[[0, 2]], R2, rtol=1e-13, atol=1e-16)


def test_source_vanishing_flux_at_tanh_equilibrium(oracle_built):
    """Eq. (5): on the equilibrium profile phi = 0.5 + 0.5 tanh(2x/eps),
    |grad phi| = 4 phi(1-phi)/eps, so the source equals grad phi exactly and
    the diffusive flux M(grad phi - R) vanishes (both models, N = 2 and an
    N = 3 binary region)."""
    eps = 4.0
    for model in ("A", "B"):
        for xx in np.linspace(-6, 6, 13):
            phi = 0.5 + 0.5 * np.tanh(2 * xx / eps)
            dphi = (1.0 / eps) * (1 - np.tanh(2 * xx / eps) ** 2)
            g = np.array([dphi * 0.6, dphi * 0.8])
            R = O.point_source(_params(2, model), np.array([phi, 1 - phi]), np.array([g, -g]))
            np.testing.assert_allclose(R[0], g, rtol=1e-12, atol=1e-16)
            R3 = O.point_source(_params(3, model), np.array([phi, 1 - phi, 0.0]),
                                np.array([g, -g, [0, 0]]))
            np.testing.assert_allclose(R3[0], g, rtol=1e-12, atol=1e-16)


def test_unit_vector_zero_gradient_reading(oracle_built):
    """Reading for n_p at a vanishing gradient: n = 0, so a node with no
    gradient at all receives no source."""
    for model in ("A", "B"):
        R = O.point_source(_params(3, model), np.array([0.2, 0.3, 0.5]), np.zeros((3, 2)))
        np.testing.assert_array_equal(R, 0.0)


def test_chemical_potential_two_phase_form(oracle_built):
    """Eqs. (14)-(17) at N = 2 reduce to the two-phase potential form
    mu_1 - mu_2 = beta g'(phi) - kappa lap phi with beta = 12 sigma/eps and
    kappa = 3 sigma eps / 2 (so F_s = (mu_1 - mu_2) grad phi)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        sigma, eps = rng.uniform(0.001, 0.05), rng.uniform(2, 6)
        p = _params(2, "B", eps=eps, sigma=sigma)
        phi, lap = rng.uniform(-0.05, 1.05), rng.normal() * 0.1
        mu = O.point_chempot(p, np.array([phi, 1 - phi]), np.array([lap, -lap]))
        gprime = 2 * phi * (1 - phi) * (1 - 2 * phi)
        expect = 12 * sigma / eps * gprime - 1.5 * sigma * eps * lap
        assert abs((mu[0] - mu[1]) - expect) < 1e-13


def test_chemical_potential_is_bulk_free_energy_derivative(oracle_built):
    """Eq. (17), bulk part: mu_phi_p = dE/dphi_p of the free-energy density of
    Eq. (14) summed over ordered pairs, taken numerically (all N phi treated
    as independent, zero Laplacians)."""
    rng = np.random.default_rng(6)
    N, eps = 4, 4.0
    sig = rng.uniform(0.005, 0.02, size=(N, N))
    sig = np.triu(sig, 1)
    sig = sig + sig.T
    p = _params(N, "B", eps=eps, sigma=sig)

    def g(s):
        return s * s * (1 - s) ** 2

    def E(ph):
        e = 0.0
        for a in range(N):
            for b in range(N):
                if a != b:
                    e += 3 * sig[a, b] / eps * (g(ph[a]) + g(ph[b]) - g(ph[a] + ph[b]))
        return e

    for _ in range(5):
        ph = rng.dirichlet(np.ones(N))
        mu = O.point_chempot(p, ph, np.zeros(N))
        h = 1e-6
        for a in range(N):
            e1, e2 = ph.copy(), ph.copy()
            e1[a] += h
            e2[a] -= h
            assert abs((E(e1) - E(e2)) / (2 * h) - mu[a]) < 1e-9


def test_lens_closed_form_reproduces_table3():
    """The Neumann closed form (Sec. 4.3, Eq. (33)) gives the analytical
    columns of Table 3 (tests/golden/lens_table3_analytic.txt) for S = pi R^2,
    R = 1: layer tension sigma_13 = 0.01, caps sigma_23 (h_1) and sigma_12
    (h_2)."""
    import os
    from oracle.oracle import lens_equilibrium
    path = os.path.join(os.path.dirname(__file__), "golden", "lens_table3_analytic.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for case, s12, s23, d, h1, h2 in rows:
        hd, ha, hb, _, _ = lens_equilibrium(0.01, float(s23), float(s12), np.pi)
        assert abs(hd - float(d)) < 6e-5, case
        assert abs(ha - float(h1)) < 6e-5, case
        assert abs(hb - float(h2)) < 6e-5, case
    # symmetric tensions: 60 degree caps, equal heights
    hd, ha, hb, ta, tb = lens_equilibrium(1.0, 1.0, 1.0, 3.0)
    assert abs(ta - np.pi / 3) < 1e-12 and abs(ha - hb) < 1e-12


def test_smooth_unit_vector_reading(oracle_built):
    """The smooth reading v / sqrt(|v|^2 + delta^2) of the sources' unit
    vectors: a zero gradient still gives R = 0, at interface gradients
    (|grad phi| ~ 1/eps) the source differs from the thresholded reading by
    O(delta^2 / |v|^2), and the two-phase reduction of Model B (R = 4 phi (1 -
    phi) / eps n) holds with the smoothed n."""
    from oracle.oracle import point_source
    for model in ("A", "B"):
        p = W.base_params(1, 1, 3, model=model, model_a_n=1.0)
        ph = np.array([0.3, 0.5, 0.2])
        g = np.array([[0.05, -0.02], [-0.08, 0.01], [0.03, 0.01]])
        r0 = point_source(p, ph, g)
        r1 = point_source(dict(p, unit_delta=1e-3), ph, g)
        r2 = point_source(dict(p, unit_delta=2e-3), ph, g)
        # |v| ~ 0.02 here: the smooth reading moves R by O(delta^2 / |v|^2)
        assert np.abs(r1 - r0).max() < 1e-2 * np.abs(r0).max()
        ratio = np.abs(r2 - r0).max() / np.abs(r1 - r0).max()
        assert 3.6 < ratio < 4.1, ratio   # 4 (delta^2) less the next order
        z = point_source(dict(p, unit_delta=1e-3), ph, np.zeros((3, 2)))
        assert np.all(z == 0.0)
    p = W.base_params(1, 1, 2, model="B")
    phi, gv = 0.3, np.array([0.04, -0.03])
    d = 1e-3
    R = point_source(dict(p, unit_delta=d), np.array([phi, 1 - phi]), np.array([gv, -gv]))
    # v = phi_2 grad phi_1 - phi_1 grad phi_2 = grad phi_1 (phi_1 + phi_2 = 1)
    n = gv / np.sqrt(gv @ gv + d * d)
    np.testing.assert_allclose(R[0], 4 * phi * (1 - phi) / 4.0 * n, rtol=1e-12, atol=1e-15)
