"""GPU tests of the adjoint (reverse) of the fused step behind
torch.autograd: gradients of L = 1/2 sum_x sum_p (phi_p(T) - phi_hat_p)^2
with respect to the pairwise surface tensions, the mobility and the initial
phase fields, with checkpoint-and-recompute over the time steps, for Model B
and (its source transposed separately) Model A.

The problem is the three-phase Model B gradient study (disks of phases 2 and
3 in phase 1, periodic, target phi_hat generated by the forward model with
sigma = (0.012, 0.008, 0.010), start sigma = (0.01, 0.01, 0.01), 500 steps,
a checkpoint every 50), with unit vectors in the smooth reading
v / sqrt(|v|^2 + delta^2), delta = 1e-3: the thresholded reading is not
differentiable where v passes through 0 and its linearisation amplifies
rounding.  The reference gradient is FP64: central differences (h = 1e-6) of
the FP64 oracle, which shares no code with the CUDA adjoint; the target is
generated by the oracle too."""

import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2306_06983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

S0 = (0.01, 0.01, 0.01)
ST = (0.012, 0.008, 0.010)
T, EVERY = 500, 50
# FP32 adjoint against FP64 differences: measured agreement 1e-5 .. 1e-4
# relative on 128^2; the bound leaves room for the FP32 accumulation over
# 500 reverse steps (about 500 x 2^-24 x the growth of the tangent dynamics).
RTOL = 2e-3
RTOL_NODE = 5e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2306_06983_gb300.build import build
    from oracle.oracle import build_oracle
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    build_oracle()
    torch.cuda.set_device(0)


def with_sigma(p, s):
    from paper_2306_06983_gb300.nlbm import pair_list
    N = p["n_phases"]
    sig = np.zeros((N, N))
    for (a, b), v in zip(pair_list(N), s):
        sig[a, b] = sig[b, a] = v
    return dict(p, sigma=sig.tolist())


def oracle_loss(p, phi0, tgt, steps=T):
    o = OracleSim(p, phi0)
    o.step(steps)
    return 0.5 * float(((o.moments()[0] - tgt) ** 2).sum())


def adjoint_vs_oracle(n, points=(), steps=T, every=EVERY, **extra):
    import torch
    from paper_2306_06983_gb300.nlbm import AdjointRun, pair_list
    p, phi0 = W.adjoint_problem(n, n)
    p = dict(p, **extra)
    phi0 = phi0.astype(np.float32).astype(np.float64)
    o = OracleSim(with_sigma(p, ST), phi0)
    o.step(steps)
    tgt = o.moments()[0]
    p0 = with_sigma(p, S0)

    def loss(q, f0, t):
        return oracle_loss(q, f0, t, steps)
    run = AdjointRun(p0, steps, every)
    phiT = run.forward(phi0).cpu().numpy().astype(np.float64)
    g0, gs, gm = run.backward(torch.from_numpy((phiT - tgt).astype(np.float32)))
    g0 = g0.cpu().numpy().astype(np.float64)
    run.close()
    got, ref = {}, {}
    h = 1e-6
    for k, (a, b) in enumerate(pair_list(3)):
        sp, sm = list(S0), list(S0)
        sp[k] += h
        sm[k] -= h
        ref[f"sigma_{a + 1}{b + 1}"] = (loss(with_sigma(p, sp), phi0, tgt) -
                                      loss(with_sigma(p, sm), phi0, tgt)) / (2 * h)
        got[f"sigma_{a + 1}{b + 1}"] = gs[a, b]
    ref["mobility"] = (loss(dict(p0, mobility=0.1 + h), phi0, tgt) -
                       loss(dict(p0, mobility=0.1 - h), phi0, tgt)) / (2 * h)
    got["mobility"] = gm
    X, Y = np.meshgrid(np.arange(n), np.arange(n))
    d = np.stack([np.sin(2 * np.pi * X / n + 0.4) * np.cos(4 * np.pi * Y / n + 1.1),
                  np.cos(2 * np.pi * (X + Y) / n + 0.2)])
    ref["phi0 direction"] = (loss(p0, phi0 + h * d, tgt) - loss(p0, phi0 - h * d, tgt)) / (2 * h)
    got["phi0 direction"] = float((g0 * d).sum())
    for q in points:
        e = np.zeros_like(phi0)
        e[q] = 1.0
        ref[f"phi0{q}"] = (loss(p0, phi0 + h * e, tgt) - loss(p0, phi0 - h * e, tgt)) / (2 * h)
        got[f"phi0{q}"] = float(g0[q])
    return got, ref, float(np.abs(g0).max())


def check(got, ref, label, gmax=0.0):
    scale = max(abs(v) for k, v in ref.items() if k.startswith("sigma"))
    for k in ref:
        err = abs(got[k] - ref[k])
        print(f"\n{label} {k:20s} oracle FD {ref[k]: .6e}  adjoint {got[k]: .6e}  rel {err / max(abs(ref[k]), 1e-30):.1e}",
              end="")
        # scalar parameters: an absolute floor of 1e-4 of the largest tension
        # gradient (their per-node terms cancel, so small ones carry FP32 sums)
        floor = 1e-4 * scale if (k.startswith("sigma") or k == "mobility") else 0.0
        rtol = RTOL
        if k.startswith("phi0("):
            # single initial-phi components (1e-6 .. 1e-5) carry the FP32 sums
            # of 500 reverse steps: 5e-3 relative plus 1e-3 of the gradient's
            # largest component
            rtol, floor = RTOL_NODE, 1e-3 * gmax
        assert err <= rtol * abs(ref[k]) + floor, (label, k, got[k], ref[k])


def test_adjoint_matches_fp64_oracle_gradient_32():
    """The 32 x 32 reduction of the gradient study: all three tension
    gradients, the mobility gradient, a smooth direction of the initial-phi
    gradient and four single initial-phi components."""
    got, ref, gmax = adjoint_vs_oracle(32, points=((0, 16, 24), (1, 1, 4), (1, 30, 7), (0, 20, 17)))
    check(got, ref, "32^2", gmax)


GRAVITY = dict(rho=[1.0, 2.0, 1.5], mu=[1.0 / 6, 2.0 / 6, 1.5 / 6], gx=2e-5, gy=-5e-5)
CASES = {"periodic": {}, "gravity": GRAVITY, "walls_y": dict(wall_y=True), "walls_x": dict(wall_x=True),
         "walls_xy": dict(wall_x=True, wall_y=True), "walls_y_gravity": dict(GRAVITY, wall_y=True, gx=0.0),
         "walls_y_weak_gravity": dict(GRAVITY, wall_y=True, gx=0.0, gy=-5e-6)}


@pytest.mark.parametrize("model,n_exp,case", [("B", 1.0, "periodic"), ("A", 1.0, "periodic"), ("A", 1.5, "periodic"),
                                              ("A", 2.0, "periodic"), ("B", 1.0, "gravity"), ("A", 2.0, "gravity"),
                                              ("B", 1.0, "walls_y"), ("B", 1.0, "walls_x"), ("A", 2.0, "walls_xy"),
                                              ("B", 1.0, "walls_y_gravity")])
def test_adjoint_few_steps_tight(model, n_exp, case):
    """Five steps on 32 x 32 (a checkpoint every 2) and the linear loss L =
    sum_x sum_p c_p(x) phi_p(T) with a fixed smooth weight c: the seed is c
    itself and no long trajectory amplifies the FP32 rounding of the
    forward, so every gradient of the adjoint, Model A's source transpose
    included, must agree closely with FP64 oracle central differences."""
    import torch
    from paper_2306_06983_gb300.nlbm import AdjointRun, pair_list
    n, steps = 32, 5
    p, phi0 = W.adjoint_problem(n, n)
    p0 = with_sigma(dict(p, model=model, model_a_n=n_exp, **CASES[case]), S0)
    phi0 = phi0.astype(np.float32).astype(np.float64)
    X, Y = np.meshgrid(np.arange(n), np.arange(n))
    c = np.stack([np.sin(2 * np.pi * X / n + 0.3 * k) * np.cos(2 * np.pi * Y / n - 0.5 * k) for k in range(3)])

    def loss(q, f0):
        o = OracleSim(q, f0)
        o.step(steps)
        return float((o.moments()[0] * c).sum())
    run = AdjointRun(p0, steps, 2)
    run.forward(phi0)
    g0, gs, gm = run.backward(torch.from_numpy(c.astype(np.float32)).cuda())
    g0 = g0.cpu().numpy().astype(np.float64)
    run.close()
    h = 1e-6
    got, ref = {}, {}
    for k, (a, b) in enumerate(pair_list(3)):
        sp, sm = list(S0), list(S0)
        sp[k] += h
        sm[k] -= h
        ref[f"sigma_{a + 1}{b + 1}"] = (loss(with_sigma(p0, sp), phi0) - loss(with_sigma(p0, sm), phi0)) / (2 * h)
        got[f"sigma_{a + 1}{b + 1}"] = gs[a, b]
    ref["mobility"] = (loss(dict(p0, mobility=0.1 + h), phi0) - loss(dict(p0, mobility=0.1 - h), phi0)) / (2 * h)
    got["mobility"] = gm
    d = np.stack([np.sin(2 * np.pi * X / n + 0.4) * np.cos(4 * np.pi * Y / n + 1.1),
                  np.cos(2 * np.pi * (X + Y) / n + 0.2)])
    ref["phi0 direction"] = (loss(p0, phi0 + h * d) - loss(p0, phi0 - h * d)) / (2 * h)
    got["phi0 direction"] = float((g0 * d).sum())
    for q in ((0, 16, 24), (1, 1, 4)):
        e = np.zeros_like(phi0)
        e[q] = 1.0
        ref[f"phi0{q}"] = (loss(p0, phi0 + h * e) - loss(p0, phi0 - h * e)) / (2 * h)
        got[f"phi0{q}"] = float(g0[q])
    scale = max(abs(v) for v in ref.values())
    for k in ref:
        err = abs(got[k] - ref[k])
        print(f"\n{model} n={n_exp} {case} 5 steps {k:20s} oracle FD {ref[k]: .6e}  adjoint {got[k]: .6e}  "
              f"rel {err / max(abs(ref[k]), 1e-30):.1e}", end="")
    for k in ref:
        assert abs(got[k] - ref[k]) <= 1e-3 * abs(ref[k]) + 1e-6 * scale, (model, n_exp, case, k, got[k], ref[k])


@pytest.mark.parametrize("n_exp", [1.0, 1.5, 2.0])
def test_adjoint_model_a_matches_fp64_oracle_gradient_128(n_exp):
    """Model A (Eq. (2): R_p = a_p n_p - phi_p^n / sum_q phi_q^n sum_q a_q
    n_q) through the 500-step study on 128 x 128, for a linear, a real and
    an integer exponent.  (On the 32 x 32 reduction the smallest tension
    gradient of Model A, five times below the others, moves by 0.2-0.7 %
    with the FP32 rounding of the 500-step forward; the five-step test
    above checks the transpose itself to 1e-5.)"""
    got, ref, gmax = adjoint_vs_oracle(128, model="A", model_a_n=n_exp)
    check(got, ref, f"Model A n={n_exp} 128^2", gmax)


def test_adjoint_gravity_matches_fp64_oracle_gradient_128():
    """Gravity F_g = rho g with densities 1 : 2 : 1.5 (Model B) on 128 x 128
    over 200 steps.  (Over 500 steps the whole periodic box accelerates, the
    gradients grow 3-10x and the FP32 rounding of the forward moves them by
    1-5 %; the same densities without gravity, or a tenth of the gravity,
    agree to 3e-5 .. 2e-4 over 500 steps, and the five-step test checks the
    transpose to 5e-6.)"""
    got, ref, gmax = adjoint_vs_oracle(128, steps=200, **GRAVITY)
    check(got, ref, "gravity 128^2", gmax)


@pytest.mark.parametrize("case", ["walls_y", "walls_xy", "walls_y_weak_gravity"])
def test_adjoint_walls_matches_fp64_oracle_gradient_128(case):
    """Half-way bounce-back walls (the pull, both stencils and F_c's gather
    transposed with their ghost nodes), Model B on 128 x 128 over 200
    steps.  (With walls and the full gravity of the five-step test the
    disks sink within the 200 steps, the tension gradients grow 130x and
    the FP32 rounding of the forward moves them by 5 %; the five-step test
    checks that case's transpose to 7.5e-6.)"""
    got, ref, gmax = adjoint_vs_oracle(128, steps=200, **CASES[case])
    check(got, ref, f"{case} 128^2", gmax)


def test_adjoint_matches_fp64_oracle_gradient_128():
    got, ref, gmax = adjoint_vs_oracle(128)
    check(got, ref, "128^2", gmax)


def test_adjoint_config_256_against_oracle_and_gpu_differences():
    """The 256 x 256 study itself: the adjoint against FP64 oracle central
    differences (h = 1e-6), and against central differences of the FP32 GPU
    forward with h = 1e-3 relative (reported; FP32 rounding of the loss makes
    those good to a few percent only)."""
    import torch
    from paper_2306_06983_gb300.nlbm import AdjointRun, Simulation, pair_list
    got, ref, gmax = adjoint_vs_oracle(256)
    check(got, ref, "256^2", gmax)
    p, phi0 = W.adjoint_problem(256, 256)
    phi0 = phi0.astype(np.float32)

    def gpu_loss(q, tgt):
        s = Simulation(q)
        s.set_phi(phi0)
        s.step(T)
        v = 0.5 * float(((s.moments()[0].cpu().numpy().astype(np.float64) - tgt) ** 2).sum())
        s.close()
        return v
    s = Simulation(with_sigma(p, ST))
    s.set_phi(phi0)
    s.step(T)
    tgt = s.moments()[0].cpu().numpy().astype(np.float64)
    s.close()
    run = AdjointRun(with_sigma(p, S0), T, EVERY)
    phiT = run.forward(phi0).cpu().numpy().astype(np.float64)
    _, gs, gm = run.backward(torch.from_numpy((phiT - tgt).astype(np.float32)))
    run.close()
    for k, (a, b) in enumerate(pair_list(3)):
        h = 1e-3 * S0[k]
        sp, sm = list(S0), list(S0)
        sp[k] += h
        sm[k] -= h
        fd = (gpu_loss(with_sigma(p, sp), tgt) - gpu_loss(with_sigma(p, sm), tgt)) / (2 * h)
        print(f"\n256^2 GPU FD (h = 1e-3 rel) sigma_{a + 1}{b + 1}: {fd: .6e} adjoint {gs[a, b]: .6e}", end="")
        if k < 2:   # the two tensions the loss depends on strongly
            assert abs(fd - gs[a, b]) <= 0.1 * abs(gs[a, b])


def test_checkpoint_interval_does_not_change_gradients():
    """Recomputed segments are bitwise the forward states, so the gradients
    do not depend on the checkpoint interval."""
    import torch
    from paper_2306_06983_gb300.nlbm import AdjointRun
    p, phi0 = W.adjoint_problem(48, 48)
    phi0 = phi0.astype(np.float32)
    res = []
    for every in (50, 7, 120):
        run = AdjointRun(with_sigma(p, S0), 120, every)
        phiT = run.forward(phi0)
        g0, gs, gm = run.backward(torch.ones_like(phiT) * 0.01 + 0.1 * phiT)
        res.append((g0.cpu(), gs, gm))
        run.close()
    for g0, gs, gm in res[1:]:
        assert torch.equal(g0, res[0][0])
        assert np.array_equal(gs, res[0][1]) and gm == res[0][2]


def test_autograd_function_and_descent():
    """torch.autograd through the library: the Function's gradients equal the
    direct reverse sweep, and one gradient step on the tensions lowers the
    loss toward the target's."""
    import torch
    from paper_2306_06983_gb300.nlbm import AdjointRun, nphase_lbm
    p, phi0 = W.adjoint_problem(64, 64)
    phi0 = torch.from_numpy(phi0.astype(np.float32)).cuda()
    with torch.no_grad():
        tgt = nphase_lbm(phi0, torch.tensor(ST, dtype=torch.float64), torch.tensor(0.1, dtype=torch.float64),
                         p, 200, 50)
    sig = torch.tensor(S0, dtype=torch.float64, requires_grad=True)
    mob = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    x0 = phi0.clone().requires_grad_(True)
    out = nphase_lbm(x0, sig, mob, p, 200, 50)
    L = 0.5 * ((out.double() - tgt.double()) ** 2).sum()
    L.backward()
    run = AdjointRun(with_sigma(p, S0), 200, 50)
    phiT = run.forward(phi0)
    g0, gs, gm = run.backward((phiT.double() - tgt.double()).float())
    run.close()
    assert torch.allclose(x0.grad, g0, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(sig.grad.numpy(), [gs[0, 1], gs[0, 2], gs[1, 2]], rtol=1e-6)
    assert abs(mob.grad.item() - gm) <= 1e-6 * abs(gm)
    step = 1e-6 / float(sig.grad.abs().max())
    with torch.no_grad():
        out2 = nphase_lbm(phi0, sig - step * sig.grad, mob, p, 200, 50)
        L2 = 0.5 * ((out2.double() - tgt.double()) ** 2).sum()
    assert float(L2) < float(L.detach())


def test_second_backward_is_refused():
    """The Function releases its run after one reverse sweep: a second
    backward through the same graph (retain_graph=True) raises a clear
    error instead of returning gradients of a released run."""
    import torch
    from paper_2306_06983_gb300.nlbm import nphase_lbm
    p, phi0 = W.adjoint_problem(32, 32)
    sig = torch.tensor(S0, dtype=torch.float64, requires_grad=True)
    mob = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    out = nphase_lbm(torch.from_numpy(phi0.astype(np.float32)).cuda(), sig, mob, p, 10, 5)
    L = (out.double() ** 2).sum()
    L.backward(retain_graph=True)
    assert sig.grad is not None
    with pytest.raises(RuntimeError, match="retain_graph"):
        L.backward()


def test_taped_sweep_matches_tape_passes():
    """The reverse sweep takes each step's intermediate fields from the taping
    forward kernel that rebuilds the segment; the single-step entry point
    rebuilds them with three separate tape passes over the step's input
    state.  Over four steps (two segments of two) both give the same tension
    and mobility gradients, up to the FP32 rounding of the intermediate
    fields (summation orders differ between the two)."""
    import torch
    from paper_2306_06983_gb300.nlbm import AdjointRun, Simulation, pair_list
    p, phi0 = W.adjoint_problem(32, 32)
    p0 = with_sigma(p, S0)
    phi0 = phi0.astype(np.float32)
    n, every = 4, 2
    ns = p0["n_phases"] - 1
    pl = p0["nx"] * p0["ny"]
    run = AdjointRun(p0, n, every)
    phiT = run.forward(phi0)
    seed = (phiT - 1.0 / 3.0).contiguous()
    _, gs, gm = run.backward(seed)
    # the input state of every step, from a plain simulation of the same run
    sim = Simulation(p0)
    sim.set_phi(phi0)
    states = []
    for _ in range(n):
        states.append(sim.save().view(torch.float32)[:(10 * ns + 12) * pl].clone())
        sim.step(1)
    sim.close()
    # seed of the last step's outputs [f 9(N-1), g 8, phi N-1, u 2, m_phi 2]:
    # only phi(T), with phase N folded onto the solved phases
    sd = torch.zeros((10 * ns + 12) * pl, dtype=torch.float32, device=seed.device)
    sd[(9 * ns + 8) * pl:(10 * ns + 8) * pl] = (seed[:ns] - seed[ns]).reshape(-1)
    gs_sum, gm_sum = np.zeros_like(gs), 0.0
    for s in reversed(range(n)):
        sd, g_s, g_m = run.reverse_step(states[s], sd)
        gs_sum += g_s
        gm_sum += g_m
    run.close()
    scale = max(abs(gs[a, b]) for a, b in pair_list(ns + 1))
    for a, b in pair_list(ns + 1):
        print(f"\nsigma_{a + 1}{b + 1}: sweep {gs[a, b]: .9e}  step by step {gs_sum[a, b]: .9e}", end="")
        assert abs(gs[a, b] - gs_sum[a, b]) <= 1e-4 * scale, (a, b, gs[a, b], gs_sum[a, b])
    print(f"\nmobility: sweep {gm: .9e}  step by step {gm_sum: .9e}")
    assert abs(gm - gm_sum) <= 1e-4 * abs(gm_sum) + 1e-6 * scale, (gm, gm_sum)
