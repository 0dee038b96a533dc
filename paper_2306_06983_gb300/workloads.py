"""Seeded synthetic workloads shaped like the paper's test problems.

This module holds only initial conditions and parameter draws; it contains
none of the lattice Boltzmann arithmetic, so the CUDA library and the FP64
oracle can both be fed from it without sharing any of the method.

Every workload is a pair ``(params, phi0)``:

* ``params`` -- dict with nx, ny, n_phases, model ('A'/'B'), model_a_n, eps,
  mobility, rho[N], mu[N] (dynamic viscosities), sigma[N][N] (symmetric,
  zero diagonal), wall_x, wall_y;
* ``phi0`` -- float64 array [N-1, ny, nx] with the volume fractions of
  phases 1..N-1; phase N is 1 minus their sum (the paper solves only N-1
  phase equations, Sec. 4).

Interface profiles follow the static-droplet initialisation of Sec. 4.1,
Eq. (30): phi = 0.5 + 0.5 tanh((R - r) / (eps/2)), with r the minimum-image
distance on a periodic axis.
"""

from __future__ import annotations

import numpy as np

SEED = 2306


def _axis_dist(coord: np.ndarray, c: float, n: int, periodic: bool) -> np.ndarray:
    d = coord - c
    if periodic:
        d = (d + n / 2.0) % n - n / 2.0
    return d


def disk(nx: int, ny: int, cx: float, cy: float, R: float, eps: float,
         periodic_x: bool = True, periodic_y: bool = True) -> np.ndarray:
    """tanh disk of radius R centred at node coordinates (cx, cy), Eq. (30)."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    dx = _axis_dist(x, cx, nx, periodic_x)
    dy = _axis_dist(y, cy, ny, periodic_y)
    r = np.sqrt(dx * dx + dy * dy)
    return 0.5 + 0.5 * np.tanh((R - r) / (eps / 2.0))


def _add_disk_windowed(field: np.ndarray, cx: float, cy: float, R: float, eps: float) -> None:
    """Add a periodic tanh disk (Eq. (30) profile) inside the window of
    half-width R + 10 eps around its centre; outside it the profile is below
    1e-17 and is taken as exactly 0."""
    ny, nx = field.shape
    h = R + 10.0 * eps
    xs = np.arange(int(np.floor(cx - h)), int(np.ceil(cx + h)) + 1)
    ys = np.arange(int(np.floor(cy - h)), int(np.ceil(cy + h)) + 1)
    if len(xs) >= nx:
        xs = np.arange(nx)
    if len(ys) >= ny:
        ys = np.arange(ny)
    dx = _axis_dist(xs.astype(np.float64), cx, nx, True)[None, :]
    dy = _axis_dist(ys.astype(np.float64), cy, ny, True)[:, None]
    r = np.sqrt(dx * dx + dy * dy)
    val = 0.5 + 0.5 * np.tanh((R - r) / (eps / 2.0))
    val[r > h] = 0.0
    field[np.ix_(ys % ny, xs % nx)] += val


def flat_band(nx: int, ny: int, y0: float, y1: float, eps: float) -> np.ndarray:
    """Band y0 < y < y1 (periodic in y) with the equilibrium profile
    0.5 + 0.5 tanh(2 d / eps) of Sec. 2.1, d the signed distance to the
    nearer interface (positive inside the band)."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    c, h = 0.5 * (y0 + y1), 0.5 * (y1 - y0)
    d = h - np.abs(_axis_dist(y, c, ny, True))
    return 0.5 + 0.5 * np.tanh(2.0 * d / eps)


def base_params(nx, ny, N, model="B", model_a_n=1.0, eps=4.0, mobility=0.1,
                rho=None, mu=None, sigma=0.01, wall_x=False, wall_y=False) -> dict:
    rho = np.ones(N) if rho is None else np.asarray(rho, dtype=np.float64)
    mu = rho / 6.0 if mu is None else np.asarray(mu, dtype=np.float64)
    if np.isscalar(sigma):
        sig = np.full((N, N), float(sigma))
        np.fill_diagonal(sig, 0.0)
    else:
        sig = np.asarray(sigma, dtype=np.float64).reshape(N, N)
    return dict(nx=int(nx), ny=int(ny), n_phases=int(N), model=model,
                model_a_n=float(model_a_n), eps=float(eps), mobility=float(mobility),
                rho=[float(v) for v in rho], mu=[float(v) for v in mu],
                sigma=sig.tolist(), wall_x=bool(wall_x), wall_y=bool(wall_y))


def droplets_64(model="B", model_a_n=1.0):
    """Three-phase droplets on a 64x64 periodic lattice (small CPU case):
    N = 3, eps = 4, all densities 1, relaxation time 1 for every phase
    (nu = 1/6, mu_p = rho_p / 6), mobility 0.1, all sigma = 0.01; phase 2 a
    disk R = 12 at (32, 32), phase 3 a disk R = 8 at (14, 14), phase 1 the
    rest."""
    nx = ny = 64
    p = base_params(nx, ny, 3, model=model, model_a_n=model_a_n, eps=4.0, mobility=0.1,
                    rho=[1.0, 1.0, 1.0], sigma=0.01)
    d2 = disk(nx, ny, 32, 32, 12, 4.0)
    d3 = disk(nx, ny, 14, 14, 8, 4.0)
    phi0 = np.stack([1.0 - d2 - d3, d2])
    return p, phi0


def random_disks(nx, ny, N, n_disks, rmin, rmax, seed=SEED, model="B", model_a_n=1.0,
                 eps=4.0, mobility=0.1, rho=None, nu_range=(0.01, 0.1),
                 sigma_range=(0.005, 0.02), max_tries=200000):
    """Non-overlapping tanh disks in a matrix of phase 1 on a periodic lattice.

    Radii U[rmin, rmax], labels U{2..N}, periodic gap >= R_i + R_j + 2 eps
    (rejection sampling), kinematic viscosities U[nu_range] per phase
    (mu_p = rho_p nu_p), pairwise sigma U[sigma_range] per unordered pair.
    With N = 5 the default densities are {1, 2, 5, 10, 1}."""
    rng = np.random.default_rng(seed)
    if rho is None:
        rho = [1.0, 2.0, 5.0, 10.0, 1.0][:N] if N <= 5 else list(np.linspace(1, 10, N))
    rho = np.asarray(rho, dtype=np.float64)
    nu = rng.uniform(nu_range[0], nu_range[1], size=N)
    sig = np.zeros((N, N))
    for a in range(N):
        for b in range(a + 1, N):
            sig[a, b] = sig[b, a] = rng.uniform(sigma_range[0], sigma_range[1])
    disks = []
    tries = 0
    while len(disks) < n_disks and tries < max_tries:
        tries += 1
        R = rng.uniform(rmin, rmax)
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        ok = True
        for (ox, oy, oR, _) in disks:
            dx = _axis_dist(np.array(cx), ox, nx, True)
            dy = _axis_dist(np.array(cy), oy, ny, True)
            if np.hypot(dx, dy) < R + oR + 2 * eps:
                ok = False
                break
        if ok:
            disks.append((cx, cy, R, int(rng.integers(2, N + 1))))
    if len(disks) < n_disks:
        raise RuntimeError(f"placed only {len(disks)} of {n_disks} disks")
    fields = np.zeros((N + 1, ny, nx))
    for (cx, cy, R, lab) in disks:
        _add_disk_windowed(fields[lab], cx, cy, R, eps)
    phi = np.empty((N, ny, nx))
    phi[0] = 1.0 - fields[2:N + 1].sum(axis=0)
    for lab in range(2, N + 1):
        phi[lab - 1] = fields[lab]
    p = base_params(nx, ny, N, model=model, model_a_n=model_a_n, eps=eps, mobility=mobility,
                    rho=rho, mu=rho * nu, sigma=sig)
    p["disks"] = len(disks)
    return p, phi[:N - 1].copy()


def disks_2048(model="B", model_a_n=1.0, seed=SEED):
    """Five-phase disk suspension on a 2048x2048 periodic lattice: 200 disks,
    radii U[10, 40], labels U{2..5}, phase 1 the matrix, densities
    {1, 2, 5, 10, 1}, kinematic viscosities U[0.01, 0.1], sigma U[0.005, 0.02],
    eps = 4, mobility 0.1."""
    return random_disks(2048, 2048, 5, 200, 10.0, 40.0, seed=seed, model=model,
                        model_a_n=model_a_n)


def disks_256(model="B", model_a_n=1.0, seed=SEED):
    """The 2048^2 five-phase suspension cut to 256x256: 25 disks with radii
    U[6, 12] (the full-size radii scaled by 1/8 would fall below the
    interface width), same parameter draws."""
    return random_disks(256, 256, 5, 25, 6.0, 12.0, seed=seed, model=model,
                        model_a_n=model_a_n)


def random_smooth(nx, ny, N, seed=SEED, model="B", model_a_n=1.0, eps=4.0,
                  wall_x=False, wall_y=False, n_disks=None):
    """Small ragged-size test lattice with a few disks of random phases
    (no gap constraint beyond rejection of exact overlap of centres)."""
    rng = np.random.default_rng(seed)
    n_disks = n_disks if n_disks is not None else max(2, (nx * ny) // 300)
    fields = np.zeros((N + 1, ny, nx))
    for _ in range(n_disks):
        R = rng.uniform(3.0, max(3.5, min(nx, ny) / 4.0))
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        lab = int(rng.integers(2, N + 1))
        fields[lab] = np.maximum(fields[lab], disk(nx, ny, cx, cy, R, eps,
                                                   not wall_x, not wall_y))
    tot = fields[2:].sum(axis=0)
    scale = np.where(tot > 1.0, 1.0 / np.maximum(tot, 1e-300), 1.0)
    fields[2:] *= scale
    phi = np.empty((N, ny, nx))
    phi[0] = 1.0 - fields[2:N + 1].sum(axis=0)
    for lab in range(2, N + 1):
        phi[lab - 1] = fields[lab]
    rho = rng.uniform(1.0, 5.0, size=N)
    nu = rng.uniform(0.02, 0.1, size=N)
    sig = np.zeros((N, N))
    for a in range(N):
        for b in range(a + 1, N):
            sig[a, b] = sig[b, a] = rng.uniform(0.005, 0.02)
    p = base_params(nx, ny, N, model=model, model_a_n=model_a_n, eps=eps, mobility=0.1,
                    rho=rho, mu=rho * nu, sigma=sig, wall_x=wall_x, wall_y=wall_y)
    return p, phi[:N - 1].copy()


def lens(nx, ny, R, s12, s13, s23, model="B", model_a_n=1.0, eps=4.0, mobility=0.1,
         y0=None, cx=None):
    """Ternary liquid lens (Sec. 4.3's problem, relabelled): phase 1 the lower
    layer, phase 2 the upper layer, phase 3 (the unsolved phase) a disk of
    radius R centred on their flat interface at height y0 (default ny/2 - 0.5,
    midway between the walls).  Periodic in x, no-flux walls at the bottom and
    top.  Profiles as in Sec. 4.3: the disk 0.5 + 0.5 tanh((R - r)/(eps/2)),
    the layers 0.5 + 0.5 tanh(2 (y0 - y)/eps) outside it.  Densities 1,
    relaxation time 1 (mu = rho/6), mobility 0.1 unless given.  For the
    paper's 1000:500:1 densities use lens_papers_labels(): with the lens as
    the unsolved phase and the light layer solved, that run diverges."""
    y0 = ny / 2.0 - 0.5 if y0 is None else float(y0)
    cx = nx / 2.0 - 0.5 if cx is None else float(cx)
    L = disk(nx, ny, cx, y0, R, eps, periodic_x=True, periodic_y=False)
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    B = 0.5 + 0.5 * np.tanh(2.0 * (y0 - y) / eps)
    sig = [[0.0, s12, s13], [s12, 0.0, s23], [s13, s23, 0.0]]
    p = base_params(nx, ny, 3, model=model, model_a_n=model_a_n, eps=eps, mobility=mobility,
                    sigma=sig, wall_y=True)
    phi0 = np.stack([(1.0 - L) * B, (1.0 - L) * (1.0 - B)])
    return p, phi0


def lens_papers_labels(nx, ny, R, s12, s23, s13=0.01, rho=(1.0, 0.5, 0.001), mu=(0.1, 0.05, 1e-4),
                       model="B", model_a_n=1.0, eps=4.0, mobility=0.1):
    """The liquid lens with the paper's labels and densities (Sec. 4.3):
    phase 1 the lower layer, phase 2 the lens, phase 3 (the unsolved phase)
    the upper layer; s12, s23 the lens's tensions against the lower and
    upper layers, s13 the layers' own.  The printed densities and
    viscosities are taken as lattice values (every kinematic viscosity
    0.1); eps and the mobility are not given (4 and 0.1 here).  With a
    density ratio of 1000 the light layer must be the unsolved phase: solved
    as a phase set, it makes the run diverge.  Same geometry as lens()."""
    p, phi0 = lens(nx, ny, R, s13, s12, s23, model=model, model_a_n=model_a_n, eps=eps,
                   mobility=mobility)
    full = np.concatenate([phi0, (1.0 - phi0.sum(0))[None]])
    order = [0, 2, 1]          # lens() labels: 1 lower, 2 upper, 3 lens
    sig = np.asarray(p["sigma"])[np.ix_(order, order)]
    p = dict(p, rho=[float(v) for v in rho], mu=[float(v) for v in mu], sigma=sig.tolist())
    return p, full[order][:2].copy()


LENS_SIZES = ((128, 64), (256, 128), (512, 256))
MODEL_A_SWEEP = (0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0)


def lens_ensemble(count=64, seed=SEED, sizes=LENS_SIZES):
    """Ensemble of independent three-phase lens problems: lattice sizes drawn
    from `sizes`, lens radius 0.2 * height on the 1|2 interface, sigma_12 =
    0.01, sigma_13 and sigma_23 uniform in [0.005, 0.015]; the first half run
    Model B, the second half Model A with its exponent swept over
    MODEL_A_SWEEP (equal shares).  Returns a list of (params, phi0)."""
    rng = np.random.default_rng(seed)
    out = []
    half = count // 2
    for k in range(count):
        nx, ny = sizes[int(rng.integers(len(sizes)))]
        s13, s23 = (float(v) for v in rng.uniform(0.005, 0.015, 2))
        if k < half:
            model, n = "B", 1.0
        else:
            model, n = "A", MODEL_A_SWEEP[(k - half) * len(MODEL_A_SWEEP) // max(count - half, 1)]
        out.append(lens(nx, ny, 0.2 * ny, 0.01, s13, s23, model=model, model_a_n=n))
    return out


def adjoint_problem(nx=256, ny=256, seed=SEED, sigma=(0.01, 0.01, 0.01), unit_delta=1e-3):
    """Three-phase, Model B, periodic problem of the gradient studies: disks
    of phases 2 and 3 (seeded positions, radii U[s/16, s/8], s = min(nx,
    256), but at least 1.5 eps; 8 disks per 256^2 nodes) in phase 1;
    densities 1, relaxation time 1, mobility 0.1, eps = 4; sigma = (sigma_12,
    sigma_13, sigma_23); unit vectors in the smooth reading with delta =
    unit_delta (differentiable)."""
    s = min(nx, 256)
    rmin, rmax = max(6.0, s / 16.0), max(7.0, s / 8.0)
    n_disks = max(2, int(round(8 * nx * ny / 256 ** 2)))
    p, phi0 = random_disks(nx, ny, 3, n_disks, rmin, rmax, seed=seed, model="B")
    s12, s13, s23 = sigma
    p = base_params(nx, ny, 3, model="B", sigma=[[0.0, s12, s13], [s12, 0.0, s23], [s13, s23, 0.0]])
    p["unit_delta"] = float(unit_delta)
    return p, phi0


def static_droplets(N=4, model="B", model_a_n=1.0, absent=(), nx=300, ny=100, R=20.0, eps=5.0,
                    sigma=0.01, mobility=0.01):
    """Static droplets (Sec. 4.1): drops of radius R of phases 1..N-1 centred
    at x = -100, 0, 100 (the first N-1 of them) on the centre line of the
    periodic domain [-nx/2, nx/2] x [-ny/2, ny/2], phase N around them,
    phi_p = 0.5 + 0.5 tanh((R - |x - x_p|)/(eps/2)).  Densities and
    viscosities 1000:500:100:1 and 100:50:10:0.1 for the quaternary system;
    the ternary and binary systems keep those of phases 1, 2 and of phase 1
    with the last entry for phase N.  Phases listed in absent (1-based) are
    zero everywhere (the reduction check).  The mobility is not given in the
    paper (0.01 here).  Node (i, j) sits at x = i + 1/2 - nx/2,
    y = j + 1/2 - ny/2."""
    centres = [-100.0, 0.0, 100.0][: N - 1]
    rho = [1000.0, 500.0, 100.0][: N - 1] + [1.0]
    mu = [100.0, 50.0, 10.0][: N - 1] + [0.1]
    x = np.arange(nx, dtype=np.float64)[None, :] + 0.5 - nx / 2.0
    y = np.arange(ny, dtype=np.float64)[:, None] + 0.5 - ny / 2.0
    phi = np.stack([0.5 + 0.5 * np.tanh((R - np.sqrt((x - c) ** 2 + y ** 2)) / (eps / 2.0))
                    for c in centres])
    for k in absent:
        phi[k - 1] = 0.0
    p = base_params(nx, ny, N, model=model, model_a_n=model_a_n, eps=eps, mobility=mobility,
                    rho=rho, mu=mu, sigma=sigma)
    return p, phi


def compound_droplet(theta23, theta13=75.0, nx=300, ny=150, R=60.0, eps=5.0, sigma=0.01,
                     mobility=0.1, rho=(1.0, 0.5, 0.001), mu=(0.1, 0.05, 1e-4), model="B",
                     model_a_n=1.0):
    """Compound droplet on a wetting wall (Sec. 4.2): a half-disk of
    radius R on the bottom wall of [-nx/2, nx/2] x [0, ny], its left half
    phase 1 and its right half phase 2, in phase 3; periodic in x, the bottom
    wall wetting with contact angles theta13 and theta23 (degrees, against
    phase 3), the top wall no-flux.  Profiles as in Sec. 4.2:
    phi_1 = D (0.5 - 0.5 tanh(2x/eps)), phi_2 = D (0.5 + 0.5 tanh(2x/eps)),
    D = 0.5 + 0.5 tanh((R - r)/(eps/2)).  Material properties of the ternary
    system of Sec. 4.1 (rho 1000:500:1, mu 100:50:0.1, scaled so that every
    kinematic viscosity is 0.1), sigma_pq = 0.01, eps = 5; the mobility is
    not given there (0.1 here).  Node (i, j) sits at x = i + 1/2 - nx/2,
    y = j + 1/2 above the wall."""
    x = np.arange(nx, dtype=np.float64)[None, :] + 0.5 - nx / 2.0
    y = np.arange(ny, dtype=np.float64)[:, None] + 0.5
    D = 0.5 + 0.5 * np.tanh((R - np.sqrt(x ** 2 + y ** 2)) / (eps / 2.0))
    phi1 = D * (0.5 - 0.5 * np.tanh(2.0 * x / eps))
    phi2 = D * (0.5 + 0.5 * np.tanh(2.0 * x / eps))
    p = base_params(nx, ny, 3, model=model, model_a_n=model_a_n, eps=eps, mobility=mobility,
                    rho=list(rho), mu=list(mu), sigma=sigma, wall_y=True)
    c13, c23 = np.cos(np.radians(theta13)), np.cos(np.radians(theta23))
    p["wall_cos"] = [float(c13), float(c23), 0.0, 0.0]
    return p, np.stack([phi1, phi2])


def rayleigh_taylor(d=256, ternary=True, eps=4.0, mobility=0.1, model="B", model_a_n=1.0,
                    sqrt_gd=0.04):
    """Rayleigh-Taylor instability (Sec. 4.4) on [-d/2, d/2] x [-2d, 2d]
    (d x 4d nodes), periodic in x, no-flux walls at the bottom and top, the
    heavy fluid 1 on top.  At = 0.5, Re = d rho_3 sqrt(g d) / mu_3 = 1000,
    Ca = mu_3 sqrt(g d) / sigma = 0.28, rho_1 : rho_2 : rho_3 = 3 : 2 : 1,
    equal viscosities, gravity (0, -g).  The lattice velocity scale
    sqrt(g d) (0.04 here), eps and the mobility are not given (readings).
    Ternary: phi_1 = 0.5 + 0.5 tanh((y - 2d/3 - 0.1 d sin(2 pi x/d))/(eps/2)),
    phi_2 = (1 - phi_1)(0.5 + 0.5 tanh((y + 2d/3 + 0.1 d sin(2 pi x/d))/(eps/2)));
    binary (phi_2 = 0): phi_1 = 0.5 + 0.5 tanh((y - 0.1 d cos(2 pi x/d))/(eps/2)).
    Node (i, j) sits at x = i + 1/2 - d/2, y = j + 1/2 - 2d."""
    nx, ny = int(d), int(4 * d)
    x = np.arange(nx, dtype=np.float64)[None, :] + 0.5 - d / 2.0
    y = np.arange(ny, dtype=np.float64)[:, None] + 0.5 - 2.0 * d
    if ternary:
        s = 0.1 * d * np.sin(2 * np.pi * x / d)
        phi1 = 0.5 + 0.5 * np.tanh((y - 2 * d / 3 - s) / (eps / 2.0))
        phi2 = (1.0 - phi1) * (0.5 + 0.5 * np.tanh((y + 2 * d / 3 + s) / (eps / 2.0)))
    else:
        phi1 = 0.5 + 0.5 * np.tanh((y - 0.1 * d * np.cos(2 * np.pi * x / d)) / (eps / 2.0))
        phi2 = np.zeros_like(phi1)
    g = sqrt_gd ** 2 / d
    mu3 = d * 1.0 * sqrt_gd / 1000.0
    sigma = mu3 * sqrt_gd / 0.28
    p = base_params(nx, ny, 3, model=model, model_a_n=model_a_n, eps=eps, mobility=mobility,
                    rho=[3.0, 2.0, 1.0], mu=[mu3, mu3, mu3], sigma=sigma, wall_y=True)
    p["gy"] = -g
    return p, np.stack([phi1, phi2])
