"""Pins of the oracle's gravity and wetting walls against what the
mathematics fixes.

Gravity enters the total force as F_g = rho g (Sec. 2.2, F = F_s + F_g +
F_c).  Wetting walls impose n_w . grad phi_p = sum_{q != p} (4/eps) phi_p
phi_q cos theta_pq (Sec. 4.2), with the pairwise angles from the N-1 angles
against phase N by Young's relation.  Pinned here:
  - a uniform fluid on a periodic lattice accelerates by exactly g per step;
  - a fluid at rest between walls settles to the hydrostatic pressure,
    dP/dy = rho g_y;
  - a 2D sessile drop relaxes to the circular cap with the prescribed
    contact angle (closed form from its conserved area);
  - with unequal tensions and the angles given against a third phase, a
    drop of phase 1 in phase 2 takes the 1|2 angle of Young's relation;
  - all cosines 0 is the no-flux wall.
"""

import math

import numpy as np
import pytest

from oracle.oracle import OracleSim, build_oracle
from paper_2306_06983_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    build_oracle()


def test_uniform_fluid_accelerates_by_g_each_step():
    p = dict(W.base_params(8, 8, 2, model="B", sigma=0.01), gx=2e-6, gy=1e-5)
    o = OracleSim(p, np.ones((1, 8, 8)))
    us = []
    for _ in range(6):
        o.step(1)
        _, u, P = o.moments()
        assert np.ptp(u[0]) == 0.0 and np.ptp(u[1]) == 0.0 and np.ptp(P) == 0.0
        us.append((u[0, 0, 0], u[1, 0, 0]))
    du = np.diff(np.array(us), axis=0)
    np.testing.assert_allclose(du[:, 0], 2e-6, rtol=1e-12)
    np.testing.assert_allclose(du[:, 1], 1e-5, rtol=1e-12)


def test_hydrostatic_pressure_between_walls():
    rho = 1.7
    p = W.base_params(4, 40, 2, model="B", sigma=0.01, wall_y=True, rho=[rho, 1.0], mu=[rho / 6, 1 / 6])
    p = dict(p, gy=-1e-5)
    o = OracleSim(p, np.ones((1, 40, 4)))
    o.step(20000)
    _, u, P = o.moments()
    assert np.abs(u).max() < 1e-8
    slope = np.polyfit(np.arange(40), P.mean(axis=1), 1)[0]
    assert abs(slope / (rho * -1e-5) - 1) < 1e-4, slope


def measure_cap(phi, theta_deg):
    """Contact chord on row 0 and height on the centre line of the phase
    whose field is phi (wall at y = -1/2), with the closed-form values of
    both for the circular cap of the same area and contact angle."""
    ny, nx = phi.shape
    th = math.radians(theta_deg)
    Rc = math.sqrt(phi.sum() / (th - math.sin(th) * math.cos(th)))
    row = phi[0]
    idx = np.where(row >= 0.5)[0]
    i0, i1 = idx[0], idx[-1]
    chord = (i1 + (row[i1] - 0.5) / (row[i1] - row[i1 + 1])) - (i0 - (row[i0] - 0.5) / (row[i0] - row[i0 - 1]))
    col = 0.5 * (phi[:, nx // 2] + phi[:, nx // 2 - 1])
    j = np.where(col >= 0.5)[0][-1]
    height = j + (col[j] - 0.5) / (col[j] - col[j + 1]) + 0.5
    # the cap's circle meets z = 0 at angle theta: centre at z = -Rc cos theta
    chord_th = 2 * math.sqrt(Rc ** 2 - (0.5 + Rc * math.cos(th)) ** 2)
    return chord, height, chord_th, Rc * (1 - math.cos(th))


def half_disk(nx, ny, R0, eps):
    z = np.arange(ny)[:, None] + 0.5
    x = np.arange(nx)[None, :] - (nx - 1) / 2
    return 0.5 + 0.5 * np.tanh((R0 - np.sqrt(x ** 2 + z ** 2)) / (eps / 2))


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_sessile_drop_relaxes_to_the_contact_angle(theta):
    """Phase 1 starts as a half-disk of radius 18 on the wall at y = -1/2 of
    a 96x48 lattice (phase 2 around it, N = 2)."""
    nx, ny = 96, 48
    p = W.base_params(nx, ny, 2, model="B", sigma=0.01, wall_y=True)
    p = dict(p, wall_cos=[math.cos(math.radians(theta)), 0.0])
    o = OracleSim(p, half_disk(nx, ny, 18.0, p["eps"])[None])
    o.step(12000)
    chord, height, chord_th, height_th = measure_cap(o.moments()[0][0], theta)
    print(f"\ntheta {theta}: chord {chord:.3f} (cap {chord_th:.3f}), height {height:.3f} (cap {height_th:.3f})")
    assert abs(chord / chord_th - 1) < 0.03
    assert abs(height / height_th - 1) < 0.03


def test_young_relation_sets_the_pairwise_angle():
    """N = 3: a drop of phase 1 in phase 2 on the bottom wall, phase 3 a band
    under the top wall, away from the drop.  The wall angles are given
    against phase 3 only; with unequal tensions Young's relation makes the
    1|2 angle cos theta_12 = (sigma_13 cos theta_13 - sigma_23 cos theta_23)
    / sigma_12 = 0.5.  (Dropping the tension ratios would give 81 degrees,
    a sign error complete wetting.)"""
    nx, ny = 64, 48
    s12, s13, s23 = 0.01, 0.02, 0.015
    c13, c23 = 0.55, 0.4
    eps = 4.0
    sig = [[0, s12, s13], [s12, 0, s23], [s13, s23, 0]]
    p = W.base_params(nx, ny, 3, model="B", sigma=sig, wall_y=True)
    p = dict(p, wall_cos=[c13, c23, 0.0, 0.0])
    drop = half_disk(nx, ny, 12.0, eps)
    band = (0.5 + 0.5 * np.tanh((np.arange(ny)[:, None] + 0.5 - 38.0) / (eps / 2))) * np.ones((1, nx))
    phi1 = drop
    phi2 = np.clip(1.0 - drop - band, 0.0, 1.0)
    o = OracleSim(p, np.stack([phi1, phi2]))
    o.step(8000)
    chord, height, chord_th, height_th = measure_cap(o.moments()[0][0], 60.0)
    print(f"\nYoung: chord {chord:.3f} (cap {chord_th:.3f}), height {height:.3f} (cap {height_th:.3f})")
    assert abs(chord / chord_th - 1) < 0.04
    assert abs(height / height_th - 1) < 0.04


def test_zero_cosines_are_the_no_flux_wall():
    p, phi0 = W.random_smooth(24, 20, 3, seed=31, model="B", wall_y=True)
    a = OracleSim(p, phi0)
    b = OracleSim(dict(p, wall_cos=[0.0, 0.0, 0.0, 0.0]), phi0)
    a.step(20)
    b.step(20)
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
