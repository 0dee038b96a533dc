"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/nlbm.h declares, and validates the
problem statement (no compute call is made here)."""

import ctypes

import numpy as np
import pytest

from paper_2306_06983_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_2306_06983_gb300.build import build
    from paper_2306_06983_gb300 import nlbm
    build()
    return nlbm.load_library()


def test_every_declared_symbol_is_exported(lib):
    from paper_2306_06983_gb300 import nlbm
    names = nlbm.declared_symbols()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_every_exported_symbol_is_declared(lib):
    """The converse: no extern "C" entry point of the library is missing
    from include/nlbm.h (read with nm when the host has it)."""
    import shutil
    import subprocess
    from paper_2306_06983_gb300 import nlbm
    if shutil.which("nm") is None:
        pytest.skip("nm not available")
    out = subprocess.run(["nm", "-D", "--defined-only", nlbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines()
                if line.split() and line.split()[-1].startswith("nlbm_")}
    assert exported, "no nlbm_ symbols found"
    missing = sorted(exported - set(nlbm.declared_symbols()))
    assert not missing, missing


def test_status_strings(lib):
    from paper_2306_06983_gb300 import nlbm
    assert nlbm.nlbm_status_string(0) == "ok"
    assert nlbm.nlbm_status_string(5) == "diverged"


def test_workspace_bytes_scales_with_lattice(lib):
    from paper_2306_06983_gb300 import nlbm
    p, _ = W.droplets_64("B")
    b64 = nlbm.nlbm_workspace_bytes(p)
    b128 = nlbm.nlbm_workspace_bytes(dict(p, nx=128, ny=128))
    # 2x(9(N-1)+8) + (N-1) + 2x2 + 2 + 1 planes of float32
    planes = 2 * (9 * 2 + 8) + 2 + 4 + 2 + 1
    assert b64 >= planes * 64 * 64 * 4
    assert abs(b128 / b64 - 4.0) < 0.05


def test_workspace_bytes_of_16bit_storage(lib):
    from paper_2306_06983_gb300 import nlbm
    p, _ = W.droplets_64("B")
    b32 = nlbm.nlbm_workspace_bytes(p)
    ns, pl = p["n_phases"] - 1, 64 * 64
    for st in ("bf16", "f16", 1, 2):
        b16 = nlbm.nlbm_workspace_bytes(dict(p, storage=st))
        # 2x(8(N-1)+8) 2-byte deviations, 2x(N-1) rest populations, 2x(N-1) phi,
        # 2x2 u, 2 m_phi, 2 P of 4 bytes
        need = 2 * (8 * ns + 8) * pl * 2 + (2 * ns + 2 * ns + 4 + 2 + 2) * pl * 4
        assert need <= b16 < need + 64 * 1024
        assert b16 < b32


@pytest.mark.parametrize("mutate,status", [
    (dict(n_phases=1), 1), (dict(n_phases=9), 1), (dict(nx=0), 1), (dict(eps=0.0), 1),
    (dict(eps=float("nan")), 1), (dict(mobility=-0.1), 1), (dict(model="A", model_a_n=0.0), 1),
    (dict(gx=float("nan")), 1), (dict(storage=1, nx=63), 1), (dict(storage="f16", nx=65), 1),
    (dict(storage=7), 1),
    (dict(nx=16384, ny=16385), 1), (dict(nx=(1 << 28) + 1, ny=1), 1),   # above 2^28 nodes
    (dict(wall_y=True, ny=3), 1),
    (dict(wall_cos=[0.5, 0.0, 0.0, 0.0]), 1),                 # wetting needs walls on y
    (dict(wall_y=True, wall_cos=[1.5, 0.0, 0.0, 0.0]), 1),   # |cos| <= 1
    (dict(wall_y=True, wall_cos=[0.0, 0.0, float("nan"), 0.0]), 1),
])
def test_parameter_validation(lib, mutate, status):
    from paper_2306_06983_gb300 import nlbm
    p, _ = W.droplets_64("B")
    q = dict(p)
    N = int(mutate.get("n_phases", q["n_phases"]))
    if N != q["n_phases"]:
        q["rho"] = [1.0] * max(N, 1)
        q["mu"] = [0.1] * max(N, 1)
        q["sigma"] = (np.full((max(N, 1), max(N, 1)), 0.01) * (1 - np.eye(max(N, 1)))).tolist()
    q.update(mutate)
    with pytest.raises(nlbm.NlbmError) as ei:
        nlbm.nlbm_workspace_bytes(q)
    assert ei.value.status == status


def test_largest_lattice_is_accepted(lib):
    """2^28 nodes is the cap (plane offsets up to 8 planes stay in 32 bits);
    its workspace is sized like any other lattice's."""
    from paper_2306_06983_gb300 import nlbm
    p, _ = W.droplets_64("B")
    small = nlbm.nlbm_workspace_bytes(p)
    per_node = (nlbm.nlbm_workspace_bytes(dict(p, nx=128, ny=128)) - small) // (128 * 128 - 64 * 64)
    fixed = small - per_node * 64 * 64
    for nx, ny in [(16384, 16384), (1 << 28, 1), (1, 1 << 28)]:
        big = nlbm.nlbm_workspace_bytes(dict(p, nx=nx, ny=ny))
        assert abs(big - per_node * nx * ny - fixed) <= 4096


def test_gravity_and_wetting_walls_are_accepted(lib):
    from paper_2306_06983_gb300 import nlbm
    p, _ = W.droplets_64("B")
    base = nlbm.nlbm_workspace_bytes(dict(p, wall_y=True))
    q = dict(p, wall_y=True, gx=1e-6, gy=-2e-5, wall_cos=[0.5, -0.25, 0.0, 1.0])
    assert nlbm.nlbm_workspace_bytes(q) == base


def test_adjoint_scope_models_and_boundaries(lib):
    """Both models, gravity and walls without wetting are accepted; wetting
    walls and 16-bit storage are refused."""
    from paper_2306_06983_gb300 import nlbm
    p, _ = W.adjoint_problem(32, 32)
    a = nlbm.nlbm_adjoint_workspace_bytes(dict(p, model="A", model_a_n=1.5), 10, 5)
    assert a == nlbm.nlbm_adjoint_workspace_bytes(p, 10, 5)
    assert a == nlbm.nlbm_adjoint_workspace_bytes(dict(p, gx=1e-5, gy=-2e-5), 10, 5)
    assert a == nlbm.nlbm_adjoint_workspace_bytes(dict(p, wall_x=True, wall_y=True), 10, 5)
    for bad in (dict(p, wall_y=True, wall_cos=[0.3, -0.2, 0.0, 0.0]), dict(p, storage="bf16")):
        with pytest.raises(nlbm.NlbmError) as ei:
            nlbm.nlbm_adjoint_workspace_bytes(bad, 10, 5)
        assert ei.value.status == 4


def test_sigma_must_be_symmetric_positive(lib):
    from paper_2306_06983_gb300 import nlbm
    p, _ = W.droplets_64("B")
    s = np.array(p["sigma"])
    s[0, 1] = 0.02
    with pytest.raises(nlbm.NlbmError):
        nlbm.nlbm_workspace_bytes(dict(p, sigma=s.tolist()))
    s = np.array(p["sigma"])
    s[1, 1] = 0.01
    with pytest.raises(nlbm.NlbmError):
        nlbm.nlbm_workspace_bytes(dict(p, sigma=s.tolist()))
    with pytest.raises(nlbm.NlbmError):
        nlbm.nlbm_workspace_bytes(dict(p, rho=[1.0, -1.0, 1.0]))


def test_create_rejects_bad_workspace(lib):
    from paper_2306_06983_gb300 import nlbm
    p, _ = W.droplets_64("B")
    n = nlbm.nlbm_workspace_bytes(p)
    with pytest.raises(nlbm.NlbmError) as ei:
        nlbm.nlbm_create(p, 0, n, 0)
    assert ei.value.status == nlbm.NLBM_EINVAL
    with pytest.raises(nlbm.NlbmError) as ei:
        nlbm.nlbm_create(p, 4096 + 16, n, 0)      # unaligned (never dereferenced)
    assert ei.value.status == nlbm.NLBM_EINVAL
    with pytest.raises(nlbm.NlbmError) as ei:
        nlbm.nlbm_create(p, 4096, n - 256, 0)     # too small (never dereferenced)
    assert ei.value.status == nlbm.NLBM_ENOMEM


def test_tile_validation(lib):
    from paper_2306_06983_gb300 import nlbm
    p, _ = W.droplets_64("B")
    n = nlbm.nlbm_workspace_bytes(p)
    # a handle over a fake (never dereferenced) aligned address: only host
    # bookkeeping calls are made on it
    h = ctypes.c_void_p(nlbm.nlbm_create(p, 1 << 20, n, 0))
    try:
        assert nlbm.nlbm_get_tile(h) == (64, 0)
        nlbm.nlbm_set_tile(h, 128, 16)
        assert nlbm.nlbm_get_tile(h) == (128, 16)
        for tx, ty in [(16, 8), (32, 8), (96, 8), (512, 8), (64, -1)]:
            with pytest.raises(nlbm.NlbmError):
                nlbm.nlbm_set_tile(h, tx, ty)
        assert nlbm.nlbm_steps_done(h) == 0
        assert nlbm.nlbm_kernel_launches(h) == 0
        nlbm.nlbm_step(h, 0)                      # zero steps launch nothing
        assert nlbm.nlbm_kernel_launches(h) == 0
    finally:
        nlbm.nlbm_destroy(h)
