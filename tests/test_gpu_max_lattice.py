"""GPU parity at the largest lattice the library accepts (2^28 nodes,
16384 x 16384), where plane offsets pass 2^31 and the population arrays of
one phase set span more than 8 GB.

The initial fields tile a periodic 64 x 64 three-phase field 256 x 256
times, so every tile of the big lattice has the same solution as the 64 x 64
problem.  After 3 steps, the tiles sampled across the lattice (the first,
the last, and two on the far edges) must equal each other bit for bit,
because every node runs the same arithmetic on the same inputs.  They must
also agree with the FP64 oracle on the small problem within the tolerances of
the short-horizon parity tests (K times the FP32 or 16-bit noise model's
spread, with floors).  With walls across x the lattice is no longer periodic in x,
and only tiles far from them are compared (the dependence of a node reaches
a few nodes per step).  Per-phase volume over the 2^28 nodes is conserved.
The forms covered: FP32 with row windows, FP32 with per-node pulls (walls
across x), and bfloat16 storage."""

import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2306_06983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_SIDE = 16384
TILE = 64
STEPS = 3
K = 4.0
FLOORS = (2e-6, 1e-8, 1e-8)
STORE = {None: 0, "bf16": 1}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2306_06983_gb300.build import build
    from oracle.oracle import build_oracle
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    build_oracle()
    torch.cuda.set_device(0)


def reference(p, phi0, storage):
    """FP64 oracle moments on the 64 x 64 tile after STEPS steps and the
    max differences of the noise model (FP32, or FP32 with 16-bit storage)
    from them."""
    a = OracleSim(p, phi0)
    b = OracleSim(p, phi0, fp32=True, store16=STORE[storage])
    a.step(STEPS)
    b.step(STEPS)
    A, B = a.moments(), b.moments()
    return A, [np.abs(x - y).max() for x, y in zip(A, B)]


@pytest.mark.parametrize("storage,wall_x", [(None, False), (None, True), ("bf16", False)])
def test_maximum_lattice(storage, wall_x):
    import torch
    from paper_2306_06983_gb300.nlbm import Simulation
    p, tile = W.random_smooth(TILE, TILE, 3, seed=21, model="B")
    tile = np.asarray(tile, dtype=np.float32)
    (ophi, ou, oP), spread = reference(p, tile.astype(np.float64), storage)
    big = dict(p, nx=N_SIDE, ny=N_SIDE, wall_x=wall_x)
    if storage:
        big["storage"] = storage
    reps = N_SIDE // TILE
    sim = Simulation(big)
    phi0 = torch.from_numpy(tile).cuda().repeat(1, reps, reps)
    sim.set_phi(phi0)
    del phi0
    m0 = sim.phase_mass()
    sim.step(STEPS)
    m1 = sim.phase_mass()
    gphi, gu, gP = sim.moments()
    # tiles (row, column) in units of TILE; with walls across x, columns
    # away from the first and last
    cols = [1, reps // 2, reps - 2] if wall_x else [0, reps // 2, reps - 1]
    picks = [(0, cols[0]), (reps - 1, cols[2]), (reps // 2, cols[2]), (reps - 1, cols[1])]
    got = []
    for r, c in picks:
        ys, xs = slice(r * TILE, (r + 1) * TILE), slice(c * TILE, (c + 1) * TILE)
        got.append(tuple(t.cpu().numpy().astype(np.float64)
                         for t in (gphi[:, ys, xs], gu[:, ys, xs], gP[ys, xs])))
    sim.close()
    del sim, gphi, gu, gP
    torch.cuda.empty_cache()
    first = got[0]
    for (r, c), g in zip(picks, got):
        for name, gv, fv, ov, sp, fl in zip(("phi", "u", "P"), g, first, (ophi, ou, oP), spread, FLOORS):
            err = np.abs(gv - ov).max()
            tol = max(fl, K * sp)
            print(f"\n{storage or 'f32'} wall_x={wall_x} tile ({r},{c}) {name}: |gpu - oracle| {err:.2e} "
                  f"(tol {tol:.2e}), |tile - first tile| {np.abs(gv - fv).max():.2e}")
            assert err <= tol, (r, c, name, err, tol)
            assert np.array_equal(gv, fv), (r, c, name)
    assert np.all(np.abs(m1 - m0) <= 1e-6 * np.abs(m0))
