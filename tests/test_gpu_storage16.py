"""GPU parity of the 16-bit population storage forms (bfloat16 and binary16
deviations, FP32 arithmetic) against the FP64 oracle.

Tolerances come from a noise model, as for the FP32 path: the oracle's own
source built in FP32 with the storage rounding emulated (each moving
population rounded, as a deviation from w_i phi of the receiving node or
3 w_i P of the sending node, to 8 or 11 significant bits) is run beside the
FP64 oracle, and the GPU must stay within K times that spread (plus a
floor).  The noise model is never a reference value.  Per-phase volume must
still be conserved to 1e-6 relative (the FP32 rest population absorbs the
rounding), and the full-size run is reported against the FP32 GPU run."""

import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2306_06983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STORE = {"bf16": 1, "f16": 2}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2306_06983_gb300.build import build
    from oracle.oracle import build_oracle
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    build_oracle()
    torch.cuda.set_device(0)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def gpu_run(p, phi0, steps, storage, tile=None):
    from paper_2306_06983_gb300.nlbm import Simulation
    sim = Simulation(dict(p, storage=storage))
    if tile:
        sim.set_tile(*tile)
    sim.set_phi(phi0)
    m0 = sim.phase_mass()
    out, done = [], 0
    for s in steps:
        sim.step(s - done)
        done = s
        phi, u, P = (t.cpu().numpy().astype(np.float64) for t in sim.moments())
        out.append((phi, u, P, sim.phase_mass()))
    sim.close()
    return m0, out


def store16_spread(p, phi0, steps, storage):
    """Per checkpoint: FP64 moments and max |phi|, |u|, |P| differences of the
    16-bit-storage noise model from them."""
    a = OracleSim(p, phi0)
    b = OracleSim(p, phi0, fp32=True, store16=STORE[storage])
    out = []
    for s in steps:
        a.step(s - a.steps_done)
        b.step(s - b.steps_done)
        A, B = a.moments(), b.moments()
        out.append((A, [np.abs(x - y).max() for x, y in zip(A, B)], np.abs(A[0] - B[0]).mean()))
    return out


K = 4.0
FLOORS = (2e-6, 1e-8, 1e-8)

CASES = {
    "droplets64_B": lambda: W.droplets_64("B"),
    "droplets64_A2": lambda: W.droplets_64("A", 2.0),
    "disks256_B": lambda: W.disks_256("B"),
    "disks256_A2": lambda: W.disks_256("A", 2.0),
    "walls68x46_N4_A": lambda: W.random_smooth(68, 46, 4, seed=4, model="A", model_a_n=1.5,
                                               wall_x=True, wall_y=True),
    "wally46x67_N2_B": lambda: W.random_smooth(46, 67, 2, seed=5, model="B", wall_y=True),
    "wally48x67_N2_B": lambda: W.random_smooth(48, 67, 2, seed=16, model="B", wall_y=True),
    "wallx130x33_N8_B": lambda: W.random_smooth(130, 33, 8, seed=6, model="B", wall_x=True),
    "ragged200x71_N6_A3": lambda: W.random_smooth(200, 71, 6, seed=7, model="A", model_a_n=3.0),
    "tiny8x8_N7_A": lambda: W.random_smooth(8, 8, 7, seed=9, model="A", n_disks=3),
    "tiny4x4_N2_B_walls": lambda: W.random_smooth(4, 4, 2, seed=10, model="B", wall_x=True,
                                                  wall_y=True, n_disks=1),
}


@pytest.mark.parametrize("storage", list(STORE))
@pytest.mark.parametrize("case", list(CASES))
def test_short_horizon_parity16(case, storage):
    p, phi0 = CASES[case]()
    phi0 = f32(phi0)
    steps = [1, 3]
    m0, g = gpu_run(p, phi0, steps, storage)
    ref = store16_spread(p, phi0, steps, storage)
    for s, (gphi, gu, gP, _), (orc, spread, _) in zip(steps, g, ref):
        for name, gv, ov, sp, fl in zip(("phi", "u", "P"), (gphi, gu, gP), orc, spread, FLOORS):
            err = np.abs(gv - ov).max()
            tol = max(fl, K * sp)
            assert err <= tol, (case, storage, s, name, err, tol)
    assert np.abs(g[-1][3] - m0).max() / (p["nx"] * p["ny"]) < 1e-7


@pytest.mark.parametrize("storage", list(STORE))
@pytest.mark.parametrize("case", ["droplets64_B", "disks256_B", "walls68x46_N4_A"])
def test_ten_step_parity16(case, storage):
    p, phi0 = CASES[case]()
    phi0 = f32(phi0)
    _, g = gpu_run(p, phi0, [10], storage)
    (orc, spread, _), = store16_spread(p, phi0, [10], storage)
    for name, gv, ov, sp, fl in zip(("phi", "u", "P"), g[0][:3], orc, spread, FLOORS):
        err = np.abs(gv - ov).max()
        assert err <= max(fl, K * sp), (case, storage, name, err, sp)


@pytest.mark.parametrize("storage", list(STORE))
@pytest.mark.parametrize("model,n", [("B", 1.0), ("A", 2.0)])
def test_droplets64_2000_steps16(model, n, storage):
    """2000 steps: per-phase mass drift <= 1e-6 relative, and max / mean
    |d phi|, max |d u| within 3x the spread of the storage noise model."""
    p, phi0 = W.droplets_64(model, n)
    phi0 = f32(phi0)
    m0, g = gpu_run(p, phi0, [2000], storage)
    gphi, gu, _, m1 = g[0]
    ((ophi, ou, _), spread, mean_spread), = store16_spread(p, phi0, [2000], storage)
    d = np.abs(gphi - ophi)
    drift = np.abs(m1 - m0) / m0
    print(f"\n{storage} {model}{n}: max|dphi| {d.max():.3e} (spread {spread[0]:.3e}) mean "
          f"{d.mean():.3e} (spread {mean_spread:.3e}) max|du| {np.abs(gu - ou).max():.3e} "
          f"(spread {spread[1]:.3e}) drift {drift.max():.3e}")
    assert np.all(drift <= 1e-6), drift
    assert d.max() <= max(1e-5, 3 * spread[0])
    assert d.mean() <= max(1e-6, 3 * mean_spread)
    assert np.abs(gu - ou).max() <= max(1e-8, 3 * spread[1])


@pytest.mark.parametrize("storage", list(STORE))
def test_tile_invariance16(storage):
    p, phi0 = W.random_smooth(200, 71, 5, seed=12, model="B", wall_y=True)
    phi0 = f32(phi0)
    _, ref = gpu_run(p, phi0, [25], storage, tile=(128, 32))
    for tile in ((64, 7), (256, 0), (128, 0)):
        _, got = gpu_run(p, phi0, [25], storage, tile=tile)
        for a, b in zip(got[0][:3], ref[0][:3]):
            assert np.array_equal(a, b), tile


@pytest.mark.parametrize("storage", list(STORE))
def test_checkpoint_and_host_paths16(storage):
    import torch
    from paper_2306_06983_gb300.nlbm import Simulation
    p, phi0 = W.random_smooth(70, 50, 4, seed=14, model="B")
    p = dict(p, storage=storage)
    phi0 = f32(phi0)
    sim = Simulation(p)
    sim.set_phi(phi0)
    sim.step(21)
    ck = sim.save()
    sim.step(30)
    a = [t.clone() for t in sim.moments()]
    sim.restore(ck)
    assert sim.steps_done == 21
    sim.step(30)
    for x, y in zip(a, sim.moments()):
        assert torch.equal(x, y)
    h = Simulation(p)
    h.set_phi_host(torch.from_numpy(phi0.astype(np.float32)).pin_memory())
    h.step(51)
    for x, y in zip(a, h.moments_host()):
        assert torch.equal(x.cpu(), y)
    sim.close()
    h.close()


def test_storage_forms_are_distinct_and_reduce_bytes():
    from paper_2306_06983_gb300.nlbm import nlbm_workspace_bytes
    p, phi0 = W.disks_256("B")
    phi0 = f32(phi0)
    res = {st: gpu_run(p, phi0, [5], st)[1][0][0] for st in ("f32", "bf16", "f16")}
    assert not np.array_equal(res["bf16"], res["f16"])
    assert not np.array_equal(res["bf16"], res["f32"])
    assert nlbm_workspace_bytes(dict(p, storage="bf16")) < 0.7 * nlbm_workspace_bytes(p)


@pytest.mark.parametrize("storage", list(STORE))
def test_full_size_disks_2048_16(storage):
    """The 2048x2048 five-phase suspension in the benchmark's launch
    configuration: 3 steps element-wise on sampled rows against the oracle
    (tolerance from the noise model on a 256x256 corner cut of the same
    suspension), then 200 steps: mass drift <= 1e-6, bounded phase fields,
    and the distance to the FP32 GPU run reported."""
    p, phi0 = W.disks_2048("B")
    phi0 = f32(phi0)
    m0, g = gpu_run(p, phi0, [3, 200], storage)
    _, g32 = gpu_run(p, phi0, [200], "f32")
    o = OracleSim(p, phi0)
    o.step(3)
    ophi, ou, oP = o.moments()
    cut = dict(p, nx=256, ny=256)
    (_, spread, _), = store16_spread(cut, np.ascontiguousarray(phi0[:, :256, :256]), [3], storage)
    gphi, gu, gP, _ = g[0]
    rows = np.random.default_rng(0).choice(p["ny"], 64, replace=False)
    for name, gv, ov, sp, fl in zip(("phi", "u", "P"), (gphi[:, rows], gu[:, rows], gP[rows]),
                                    (ophi[:, rows], ou[:, rows], oP[rows]), spread, FLOORS):
        err = np.abs(gv - ov).max()
        assert err <= max(fl, K * sp), (storage, name, err, sp)
    phi200, u200, _, m200 = g[1]
    assert np.all(np.abs(m200 - m0) / np.abs(m0) < 1e-6)
    assert np.isfinite(phi200).all() and phi200.min() > -0.05 and phi200.max() < 1.05
    f_phi, f_u = g32[0][0], g32[0][1]
    du = np.sqrt(((u200 - f_u) ** 2).sum() / (f_u ** 2).sum())
    print(f"\n{storage} vs FP32 after 200 steps at 2048^2: max|dphi| "
          f"{np.abs(phi200 - f_phi).max():.3e}, rel L2(u) {du:.3e}")
