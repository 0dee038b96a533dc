"""Python binding of the C ABI in ``include/nlbm.h`` (argument marshalling
only: every step of the method runs in the CUDA library ``libnlbm.so``).

PyTorch supplies device memory and streams.  The functions ``nlbm_*`` mirror
the C entry points one to one; :class:`Simulation` wraps a handle together
with the workspace tensor that backs it.

The library must have been built (``paper_2306_06983_gb300.build.build()``);
importing this module does not build it, and loading fails loudly when the
shared object is missing -- there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libnlbm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "nlbm.h")

NLBM_OK, NLBM_EINVAL, NLBM_ENOMEM, NLBM_ECUDA, NLBM_ENOTSUP, NLBM_EDIVERGED = range(6)
NLBM_BC_PERIODIC, NLBM_BC_WALL = 0, 1
NLBM_MODEL_A, NLBM_MODEL_B = 0, 1
NLBM_STORE_F32, NLBM_STORE_BF16, NLBM_STORE_F16 = 0, 1, 2
STORAGE_CODES = {"f32": NLBM_STORE_F32, "bf16": NLBM_STORE_BF16, "f16": NLBM_STORE_F16}
STATUS_NAMES = {0: "NLBM_OK", 1: "NLBM_EINVAL", 2: "NLBM_ENOMEM", 3: "NLBM_ECUDA",
                4: "NLBM_ENOTSUP", 5: "NLBM_EDIVERGED"}


class NlbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class nlbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("n_phases", ctypes.c_int32), ("model", ctypes.c_int32),
        ("model_a_n", ctypes.c_double), ("eps", ctypes.c_double), ("mobility", ctypes.c_double),
        ("rho", ctypes.POINTER(ctypes.c_double)), ("mu", ctypes.POINTER(ctypes.c_double)),
        ("sigma", ctypes.POINTER(ctypes.c_double)),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("storage", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("unit_delta", ctypes.c_double),
        ("wall_cos", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libnlbm.so and declare every exported signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library {path} is not built; run __graft_entry__.build() or "
            "python -m paper_2306_06983_gb300.build")
    lib = ctypes.CDLL(path)
    P, vp, st = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int
    sig = {
        "nlbm_workspace_bytes": (st, [P(nlbm_params), P(ctypes.c_size_t)]),
        "nlbm_create": (st, [P(nlbm_params), vp, ctypes.c_size_t, vp, P(vp)]),
        "nlbm_set_phi": (st, [vp, vp]),
        "nlbm_set_phi_host": (st, [vp, vp]),
        "nlbm_set_velocity": (st, [vp, vp]),
        "nlbm_step": (st, [vp, ctypes.c_int64]),
        "nlbm_get_moments": (st, [vp, vp, vp, vp]),
        "nlbm_get_moments_host": (st, [vp, vp, vp, vp]),
        "nlbm_phase_mass": (st, [vp, P(ctypes.c_double)]),
        "nlbm_state_bytes": (st, [vp, P(ctypes.c_size_t)]),
        "nlbm_save": (st, [vp, vp]),
        "nlbm_restore": (st, [vp, vp]),
        "nlbm_synchronize": (st, [vp]),
        "nlbm_steps_done": (ctypes.c_int64, [vp]),
        "nlbm_batch_workspace_bytes": (st, [P(nlbm_params), ctypes.c_int32, P(ctypes.c_size_t)]),
        "nlbm_batch_create": (st, [P(nlbm_params), ctypes.c_int32, vp, ctypes.c_size_t, vp, P(vp)]),
        "nlbm_batch_set_phi": (st, [vp, ctypes.c_int32, vp]),
        "nlbm_batch_step": (st, [vp, ctypes.c_int64]),
        "nlbm_batch_get_moments": (st, [vp, ctypes.c_int32, vp, vp, vp]),
        "nlbm_batch_phase_mass": (st, [vp, ctypes.c_int32, P(ctypes.c_double)]),
        "nlbm_batch_set_tile": (st, [vp, ctypes.c_int32, ctypes.c_int32]),
        "nlbm_batch_get_tile": (st, [vp, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)]),
        "nlbm_batch_state_bytes": (st, [vp, P(ctypes.c_size_t)]),
        "nlbm_batch_autotune": (st, [vp, vp, ctypes.c_size_t, ctypes.c_int32, P(ctypes.c_int32),
                                     P(ctypes.c_int32), P(ctypes.c_float)]),
        "nlbm_batch_synchronize": (st, [vp]),
        "nlbm_batch_steps_done": (ctypes.c_int64, [vp]),
        "nlbm_batch_kernel_launches": (ctypes.c_int64, [vp]),
        "nlbm_batch_destroy": (None, [vp]),
        "nlbm_batch_last_error": (ctypes.c_char_p, [vp]),
        "nlbm_adjoint_workspace_bytes": (st, [P(nlbm_params), ctypes.c_int32, ctypes.c_int32,
                                              P(ctypes.c_size_t)]),
        "nlbm_adjoint_create": (st, [P(nlbm_params), ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_size_t, vp,
                                     P(vp)]),
        "nlbm_adjoint_forward": (st, [vp, vp, vp]),
        "nlbm_adjoint_backward": (st, [vp, vp, vp, P(ctypes.c_double), P(ctypes.c_double)]),
        "nlbm_adjoint_kernel_launches": (ctypes.c_int64, [vp]),
        "nlbm_adjoint_uses_graph": (ctypes.c_int32, [vp]),
        "nlbm_adjoint_reverse_step": (st, [vp, vp, vp, vp, P(ctypes.c_double), P(ctypes.c_double)]),
        "nlbm_adjoint_destroy": (None, [vp]),
        "nlbm_adjoint_last_error": (ctypes.c_char_p, [vp]),
        "nlbm_kernel_launches": (ctypes.c_int64, [vp]),
        "nlbm_set_tile": (st, [vp, ctypes.c_int32, ctypes.c_int32]),
        "nlbm_get_tile": (st, [vp, P(ctypes.c_int32), P(ctypes.c_int32)]),
        "nlbm_autotune": (st, [vp, vp, ctypes.c_size_t, ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32),
                               P(ctypes.c_float)]),
        "nlbm_destroy": (None, [vp]),
        "nlbm_last_error": (ctypes.c_char_p, [vp]),
        "nlbm_status_string": (ctypes.c_char_p, [st]),
        "nlbm_phase_mass_noalloc": (st, [vp, ctypes.c_int32, ctypes.c_int64, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols(header: str = HEADER):
    """Names of the functions declared in include/nlbm.h."""
    text = open(header).read()
    return sorted(set(re.findall(r"\b(nlbm_[a-z_]+)\s*\(", text)))


def _check(st: int, handle=None):
    if st != NLBM_OK:
        msg = load_library().nlbm_last_error(handle).decode()
        raise NlbmError(st, msg)


def make_params(p: dict):
    """ctypes parameter block from a workload dict; returns (struct, keepalive).

    Keys: nx, ny, n_phases, model ('A' or 'B'), eps, mobility, rho[N], mu[N],
    sigma[N][N]; optional model_a_n, wall_x, wall_y, storage ('f32', 'bf16',
    'f16'), unit_delta, gx, gy (gravity, F_g = rho g) and wall_cos (2 (N-1)
    cosines of the contact angles against phase N at the walls y = 0 and
    y = ny - 1; see nlbm_params in include/nlbm.h)."""
    N = int(p["n_phases"])
    rho = (ctypes.c_double * N)(*[float(v) for v in p["rho"]])
    mu = (ctypes.c_double * N)(*[float(v) for v in p["mu"]])
    sig = np.asarray(p["sigma"], dtype=np.float64).reshape(N, N)
    sigma = (ctypes.c_double * (N * N))(*[float(v) for v in sig.ravel()])
    s = nlbm_params()
    s.nx, s.ny = int(p["nx"]), int(p["ny"])
    s.bc_x = NLBM_BC_WALL if p.get("wall_x") else NLBM_BC_PERIODIC
    s.bc_y = NLBM_BC_WALL if p.get("wall_y") else NLBM_BC_PERIODIC
    s.n_phases = N
    s.model = {"A": NLBM_MODEL_A, "B": NLBM_MODEL_B}[p["model"]]
    s.model_a_n = float(p.get("model_a_n", 1.0))
    s.eps, s.mobility = float(p["eps"]), float(p["mobility"])
    s.rho = ctypes.cast(rho, ctypes.POINTER(ctypes.c_double))
    s.mu = ctypes.cast(mu, ctypes.POINTER(ctypes.c_double))
    s.sigma = ctypes.cast(sigma, ctypes.POINTER(ctypes.c_double))
    s.gx = float(p.get("gx", 0.0))
    s.gy = float(p.get("gy", 0.0))
    st = p.get("storage", NLBM_STORE_F32)
    s.storage = STORAGE_CODES[st] if isinstance(st, str) else int(st)
    s.reserved = 0
    s.unit_delta = float(p.get("unit_delta", 0.0))
    wc = p.get("wall_cos")
    wall_cos = None
    if wc is not None:
        wall_cos = (ctypes.c_double * len(wc))(*[float(v) for v in wc])
        if len(wc) != 2 * (N - 1):
            raise ValueError("wall_cos holds 2 (N - 1) cosines")
        s.wall_cos = ctypes.cast(wall_cos, ctypes.POINTER(ctypes.c_double))
    return s, (rho, mu, sigma, wall_cos)


# ------------------------------------------------- one-to-one C entry points

def nlbm_workspace_bytes(params: dict) -> int:
    s, keep = make_params(params)
    out = ctypes.c_size_t(0)
    _check(load_library().nlbm_workspace_bytes(ctypes.byref(s), ctypes.byref(out)))
    return int(out.value)


def nlbm_create(params: dict, workspace_ptr: int, workspace_bytes: int, stream_ptr: int) -> int:
    s, keep = make_params(params)
    h = ctypes.c_void_p()
    _check(load_library().nlbm_create(ctypes.byref(s), ctypes.c_void_p(workspace_ptr),
                                      workspace_bytes, ctypes.c_void_p(stream_ptr), ctypes.byref(h)))
    return h.value


def nlbm_set_phi(h, dev_ptr: int):
    _check(load_library().nlbm_set_phi(h, ctypes.c_void_p(dev_ptr)), h)


def nlbm_set_phi_host(h, host_ptr: int):
    _check(load_library().nlbm_set_phi_host(h, ctypes.c_void_p(host_ptr)), h)


def nlbm_set_velocity(h, dev_ptr: int):
    _check(load_library().nlbm_set_velocity(h, ctypes.c_void_p(dev_ptr)), h)


def nlbm_step(h, nsteps: int):
    _check(load_library().nlbm_step(h, int(nsteps)), h)


def nlbm_get_moments(h, phi_ptr=None, u_ptr=None, p_ptr=None):
    _check(load_library().nlbm_get_moments(h, phi_ptr, u_ptr, p_ptr), h)


def nlbm_get_moments_host(h, phi_ptr=None, u_ptr=None, p_ptr=None):
    _check(load_library().nlbm_get_moments_host(h, phi_ptr, u_ptr, p_ptr), h)


def nlbm_phase_mass(h, N: int, allow_diverged: bool = False) -> np.ndarray:
    out = (ctypes.c_double * N)()
    st = load_library().nlbm_phase_mass(h, out)
    if not (allow_diverged and st == NLBM_EDIVERGED):
        _check(st, h)
    return np.array(out[:], dtype=np.float64)


def nlbm_state_bytes(h) -> int:
    out = ctypes.c_size_t(0)
    _check(load_library().nlbm_state_bytes(h, ctypes.byref(out)), h)
    return int(out.value)


def nlbm_save(h, dev_ptr: int):
    _check(load_library().nlbm_save(h, ctypes.c_void_p(dev_ptr)), h)


def nlbm_restore(h, dev_ptr: int):
    _check(load_library().nlbm_restore(h, ctypes.c_void_p(dev_ptr)), h)


def nlbm_synchronize(h):
    _check(load_library().nlbm_synchronize(h), h)


def nlbm_steps_done(h) -> int:
    return int(load_library().nlbm_steps_done(h))


def nlbm_kernel_launches(h) -> int:
    return int(load_library().nlbm_kernel_launches(h))


def nlbm_set_tile(h, tx: int, ty: int):
    _check(load_library().nlbm_set_tile(h, int(tx), int(ty)), h)


def nlbm_get_tile(h):
    tx, ty = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().nlbm_get_tile(h, ctypes.byref(tx), ctypes.byref(ty)), h)
    return tx.value, ty.value


def nlbm_autotune(h, scratch_ptr: int, scratch_bytes: int, steps_per_trial: int):
    tx, ty, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load_library().nlbm_autotune(h, ctypes.c_void_p(scratch_ptr), scratch_bytes, steps_per_trial,
                                        ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(ms)), h)
    return tx.value, ty.value, ms.value


def nlbm_destroy(h):
    load_library().nlbm_destroy(h)


def nlbm_last_error(h=None) -> str:
    return load_library().nlbm_last_error(h).decode()


def nlbm_status_string(st: int) -> str:
    return load_library().nlbm_status_string(st).decode()


def nlbm_phase_mass_noalloc(dev_phi: int, n_phases: int, n_nodes: int, dev_mass: int,
                            dev_flag: int, stream_ptr: int = 0) -> int:
    """Volume reduction that allocates nothing (scratch is a fixed array
    inside the library); returns the status code (0 = OK)."""
    return int(load_library().nlbm_phase_mass_noalloc(
        ctypes.c_void_p(dev_phi), int(n_phases), int(n_nodes), ctypes.c_void_p(dev_mass),
        ctypes.c_void_p(dev_flag), ctypes.c_void_p(stream_ptr)))


# ------------------------------------------------------------ convenience

class Simulation:
    """One simulation on the current CUDA device; the workspace is a torch
    uint8 tensor owned by this object."""

    def __init__(self, params: dict, stream=None, device=None):
        import torch
        self.torch = torch
        self.params = dict(params)
        self.N = int(params["n_phases"])
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = nlbm_workspace_bytes(params)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.h = ctypes.c_void_p(nlbm_create(params, aligned, nbytes, self.stream.cuda_stream))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            nlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state
    def set_phi(self, phi0):
        """phi0: [N-1, ny, nx] numpy array or CUDA tensor (phases 1..N-1)."""
        torch = self.torch
        t = torch.as_tensor(phi0)
        if t.shape != (self.N - 1, self.ny, self.nx):
            raise ValueError(f"phi0 has shape {tuple(t.shape)}, expected {(self.N - 1, self.ny, self.nx)}")
        t = t.to(device=self.device, dtype=torch.float32).contiguous()
        self._phi0 = t
        nlbm_set_phi(self.h, t.data_ptr())

    def set_phi_host(self, phi0_host):
        """phi0_host: float32 CPU tensor (pinned or pageable) [N-1, ny, nx]."""
        t = self.torch.as_tensor(phi0_host)
        assert t.device.type == "cpu" and t.dtype == self.torch.float32 and t.is_contiguous()
        assert t.shape == (self.N - 1, self.ny, self.nx)
        nlbm_set_phi_host(self.h, t.data_ptr())

    def set_velocity(self, u0):
        """Start in motion (after set_phi, before the first step): u0 [2, ny,
        nx] (u_x, u_y) as a tensor or array, or a pair (u_x, u_y) for a
        uniform flow."""
        torch = self.torch
        t = torch.as_tensor(np.asarray(u0) if not isinstance(u0, torch.Tensor) else u0, dtype=torch.float32)
        if t.shape == (2,):
            t = t[:, None, None].expand(2, self.ny, self.nx)
        t = t.to(self.device).contiguous()
        assert t.shape == (2, self.ny, self.nx), t.shape
        self._u0 = t   # kept alive until the stream has read it
        nlbm_set_velocity(self.h, t.data_ptr())

    def step(self, n: int):
        nlbm_step(self.h, n)

    def moments(self):
        """(phi [N,ny,nx], u [2,ny,nx], P [ny,nx]) as new CUDA tensors."""
        torch = self.torch
        phi = torch.empty((self.N, self.ny, self.nx), dtype=torch.float32, device=self.device)
        u = torch.empty((2, self.ny, self.nx), dtype=torch.float32, device=self.device)
        P = torch.empty((self.ny, self.nx), dtype=torch.float32, device=self.device)
        nlbm_get_moments(self.h, phi.data_ptr(), u.data_ptr(), P.data_ptr())
        return phi, u, P

    def moments_host(self, phi=None, u=None, P=None):
        """Fill CPU float32 tensors (allocated if None) through the host entry point."""
        torch = self.torch
        if phi is None:
            phi = torch.empty((self.N, self.ny, self.nx), dtype=torch.float32)
        if u is None:
            u = torch.empty((2, self.ny, self.nx), dtype=torch.float32)
        if P is None:
            P = torch.empty((self.ny, self.nx), dtype=torch.float32)
        nlbm_get_moments_host(self.h, phi.data_ptr(), u.data_ptr(), P.data_ptr())
        return phi, u, P

    def phase_mass(self, allow_diverged: bool = False) -> np.ndarray:
        return nlbm_phase_mass(self.h, self.N, allow_diverged)

    def save(self):
        n = nlbm_state_bytes(self.h)
        buf = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        nlbm_save(self.h, buf.data_ptr())
        return buf

    def restore(self, buf):
        nlbm_restore(self.h, buf.data_ptr())

    def synchronize(self):
        nlbm_synchronize(self.h)

    @property
    def steps_done(self) -> int:
        return nlbm_steps_done(self.h)

    @property
    def kernel_launches(self) -> int:
        return nlbm_kernel_launches(self.h)

    def set_tile(self, tx: int, ty: int):
        nlbm_set_tile(self.h, tx, ty)

    def get_tile(self):
        return nlbm_get_tile(self.h)

    def autotune(self, steps_per_trial: int = 20):
        """Time every tile shape from the current state and keep the
        fastest; returns (tx, ty, ms per step).  State and step count are
        unchanged."""
        n = nlbm_state_bytes(self.h)
        scratch = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        return nlbm_autotune(self.h, scratch.data_ptr(), n, steps_per_trial)


# ------------------------------------------------------------ ensembles

def _check_batch(st: int, handle=None):
    if st != NLBM_OK:
        msg = load_library().nlbm_batch_last_error(handle).decode()
        raise NlbmError(st, msg)


def _params_array(sims):
    arr = (nlbm_params * len(sims))()
    keep = []
    for k, p in enumerate(sims):
        s, kp = make_params(p)
        arr[k] = s
        keep.append(kp)
    return arr, keep


def nlbm_batch_workspace_bytes(sims) -> int:
    arr, keep = _params_array(sims)
    out = ctypes.c_size_t(0)
    _check_batch(load_library().nlbm_batch_workspace_bytes(arr, len(sims), ctypes.byref(out)))
    return int(out.value)


def nlbm_batch_create(sims, workspace_ptr: int, workspace_bytes: int, stream_ptr: int) -> int:
    arr, keep = _params_array(sims)
    h = ctypes.c_void_p()
    _check_batch(load_library().nlbm_batch_create(arr, len(sims), ctypes.c_void_p(workspace_ptr),
                                                  workspace_bytes, ctypes.c_void_p(stream_ptr),
                                                  ctypes.byref(h)))
    return h.value


def nlbm_batch_set_phi(h, sim: int, dev_ptr: int):
    _check_batch(load_library().nlbm_batch_set_phi(h, sim, ctypes.c_void_p(dev_ptr)), h)


def nlbm_batch_step(h, nsteps: int):
    _check_batch(load_library().nlbm_batch_step(h, nsteps), h)


def nlbm_batch_get_moments(h, sim: int, phi_ptr=None, u_ptr=None, p_ptr=None):
    _check_batch(load_library().nlbm_batch_get_moments(h, sim, phi_ptr, u_ptr, p_ptr), h)


def nlbm_batch_phase_mass(h, sim: int, N: int) -> np.ndarray:
    out = (ctypes.c_double * N)()
    _check_batch(load_library().nlbm_batch_phase_mass(h, sim, out), h)
    return np.array(out[:], dtype=np.float64)


def nlbm_batch_set_tile(h, tx: int, ty: int):
    _check_batch(load_library().nlbm_batch_set_tile(h, tx, ty), h)


def nlbm_batch_get_tile(h):
    tx, ty, nt = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check_batch(load_library().nlbm_batch_get_tile(h, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(nt)), h)
    return tx.value, ty.value, nt.value


def nlbm_batch_state_bytes(h) -> int:
    out = ctypes.c_size_t(0)
    _check_batch(load_library().nlbm_batch_state_bytes(h, ctypes.byref(out)), h)
    return int(out.value)


def nlbm_batch_autotune(h, scratch_ptr: int, scratch_bytes: int, steps_per_trial: int):
    tx, ty, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check_batch(load_library().nlbm_batch_autotune(h, ctypes.c_void_p(scratch_ptr), scratch_bytes,
                                                    steps_per_trial, ctypes.byref(tx), ctypes.byref(ty),
                                                    ctypes.byref(ms)), h)
    return tx.value, ty.value, ms.value


def nlbm_batch_synchronize(h):
    _check_batch(load_library().nlbm_batch_synchronize(h), h)


def nlbm_batch_steps_done(h) -> int:
    return int(load_library().nlbm_batch_steps_done(h))


def nlbm_batch_kernel_launches(h) -> int:
    return int(load_library().nlbm_batch_kernel_launches(h))


def nlbm_batch_destroy(h):
    load_library().nlbm_batch_destroy(h)


def nlbm_batch_last_error(h=None) -> str:
    return load_library().nlbm_batch_last_error(h).decode()


class Batch:
    """An ensemble of independent simulations on the current CUDA device; the
    workspace is a torch uint8 tensor owned by this object."""

    def __init__(self, sims, stream=None, device=None):
        import torch
        self.torch = torch
        self.sims = [dict(p) for p in sims]
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = nlbm_batch_workspace_bytes(self.sims)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        self.h = ctypes.c_void_p(nlbm_batch_create(self.sims, aligned, nbytes, self.stream.cuda_stream))
        self._phi0 = {}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            nlbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.sims)

    def set_phi(self, k: int, phi0):
        p = self.sims[k]
        N, ny, nx = int(p["n_phases"]), int(p["ny"]), int(p["nx"])
        t = self.torch.as_tensor(phi0).to(device=self.device, dtype=self.torch.float32).contiguous()
        if t.shape != (N - 1, ny, nx):
            raise ValueError(f"phi0 of member {k} has shape {tuple(t.shape)}, expected {(N - 1, ny, nx)}")
        self._phi0[k] = t
        nlbm_batch_set_phi(self.h, k, t.data_ptr())

    def step(self, n: int):
        nlbm_batch_step(self.h, n)

    def moments(self, k: int):
        torch = self.torch
        p = self.sims[k]
        N, ny, nx = int(p["n_phases"]), int(p["ny"]), int(p["nx"])
        phi = torch.empty((N, ny, nx), dtype=torch.float32, device=self.device)
        u = torch.empty((2, ny, nx), dtype=torch.float32, device=self.device)
        P = torch.empty((ny, nx), dtype=torch.float32, device=self.device)
        nlbm_batch_get_moments(self.h, k, phi.data_ptr(), u.data_ptr(), P.data_ptr())
        return phi, u, P

    def phase_mass(self, k: int) -> np.ndarray:
        return nlbm_batch_phase_mass(self.h, k, int(self.sims[k]["n_phases"]))

    def set_tile(self, tx: int, ty: int):
        nlbm_batch_set_tile(self.h, tx, ty)

    def get_tile(self):
        return nlbm_batch_get_tile(self.h)

    def autotune(self, steps_per_trial: int = 5):
        n = nlbm_batch_state_bytes(self.h)
        scratch = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        return nlbm_batch_autotune(self.h, scratch.data_ptr(), n, steps_per_trial)

    def synchronize(self):
        nlbm_batch_synchronize(self.h)

    @property
    def steps_done(self) -> int:
        return nlbm_batch_steps_done(self.h)

    @property
    def kernel_launches(self) -> int:
        return nlbm_batch_kernel_launches(self.h)


# ------------------------------------------------------------ adjoint

def _check_adj(st: int, handle=None):
    if st != NLBM_OK:
        msg = load_library().nlbm_adjoint_last_error(handle).decode()
        raise NlbmError(st, msg)


def nlbm_adjoint_workspace_bytes(params: dict, nsteps: int, every: int) -> int:
    s, keep = make_params(params)
    out = ctypes.c_size_t(0)
    _check_adj(load_library().nlbm_adjoint_workspace_bytes(ctypes.byref(s), nsteps, every, ctypes.byref(out)))
    return int(out.value)


def nlbm_adjoint_create(params: dict, nsteps: int, every: int, workspace_ptr: int, workspace_bytes: int,
                        stream_ptr: int) -> int:
    s, keep = make_params(params)
    h = ctypes.c_void_p()
    _check_adj(load_library().nlbm_adjoint_create(ctypes.byref(s), nsteps, every, ctypes.c_void_p(workspace_ptr),
                                                  workspace_bytes, ctypes.c_void_p(stream_ptr), ctypes.byref(h)))
    return h.value


def nlbm_adjoint_forward(h, phi0_ptr: int, phi_final_ptr):
    _check_adj(load_library().nlbm_adjoint_forward(h, ctypes.c_void_p(phi0_ptr), phi_final_ptr), h)


def nlbm_adjoint_backward(h, seed_ptr: int, grad_phi0_ptr, N: int):
    gs = (ctypes.c_double * (N * N))()
    gm = ctypes.c_double(0.0)
    _check_adj(load_library().nlbm_adjoint_backward(h, ctypes.c_void_p(seed_ptr), grad_phi0_ptr, gs,
                                                    ctypes.byref(gm)), h)
    return np.array(gs[:], dtype=np.float64).reshape(N, N), float(gm.value)


def nlbm_adjoint_kernel_launches(h) -> int:
    return int(load_library().nlbm_adjoint_kernel_launches(h))


def nlbm_adjoint_destroy(h):
    load_library().nlbm_adjoint_destroy(h)


def nlbm_adjoint_last_error(h=None) -> str:
    return load_library().nlbm_adjoint_last_error(h).decode()


class AdjointRun:
    """One differentiable run: nsteps forward steps with a checkpoint every
    `every` steps, then the reverse sweep for a seed dL/dphi(T)."""

    def __init__(self, params: dict, nsteps: int, every: int = 50, stream=None, device=None):
        import torch
        self.torch = torch
        self.params = dict(params)
        self.N, self.nx, self.ny = int(params["n_phases"]), int(params["nx"]), int(params["ny"])
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        n = nlbm_adjoint_workspace_bytes(params, nsteps, every)
        self.workspace = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        self.h = ctypes.c_void_p(nlbm_adjoint_create(params, nsteps, every, aligned, n, self.stream.cuda_stream))

    def forward(self, phi0):
        """phi0 [N-1, ny, nx] -> phi(T) [N, ny, nx] (CUDA tensor)."""
        torch = self.torch
        t = torch.as_tensor(phi0).to(device=self.device, dtype=torch.float32).contiguous()
        self._phi0 = t
        out = torch.empty((self.N, self.ny, self.nx), dtype=torch.float32, device=self.device)
        nlbm_adjoint_forward(self.h, t.data_ptr(), ctypes.c_void_p(out.data_ptr()))
        return out

    def backward(self, seed):
        """seed = dL/dphi(T) [N, ny, nx] -> (dL/dphi0 [N-1, ny, nx],
        dL/dsigma [N, N] (symmetric; entry (p, q) is the derivative with
        respect to the pair's single value), dL/dmobility)."""
        torch = self.torch
        sd = torch.as_tensor(seed).to(device=self.device, dtype=torch.float32).contiguous()
        g0 = torch.empty((self.N - 1, self.ny, self.nx), dtype=torch.float32, device=self.device)
        gs, gm = nlbm_adjoint_backward(self.h, sd.data_ptr(), ctypes.c_void_p(g0.data_ptr()), self.N)
        return g0, gs, gm

    def reverse_step(self, state, seed_out):
        """One reverse step from a packed state record [f 9(N-1), g 8, u 2,
        phi N-1, m_phi 2 planes] and the adjoint seed of its outputs [f
        9(N-1), g 8, phi N-1, u 2, m_phi 2 planes]; returns the adjoint of
        its inputs in the seed layout and the parameter gradients."""
        torch = self.torch
        st = torch.as_tensor(state).to(device=self.device, dtype=torch.float32).contiguous()
        sd = torch.as_tensor(seed_out).to(device=self.device, dtype=torch.float32).contiguous()
        out = torch.empty_like(sd)
        gs = (ctypes.c_double * (self.N * self.N))()
        gm = ctypes.c_double(0.0)
        _check_adj(load_library().nlbm_adjoint_reverse_step(self.h, ctypes.c_void_p(st.data_ptr()),
                                                            ctypes.c_void_p(sd.data_ptr()),
                                                            ctypes.c_void_p(out.data_ptr()), gs,
                                                            ctypes.byref(gm)), self.h)
        return out, np.array(gs[:]).reshape(self.N, self.N), float(gm.value)

    @property
    def kernel_launches(self) -> int:
        return nlbm_adjoint_kernel_launches(self.h)

    @property
    def uses_graph(self) -> bool:
        return bool(load_library().nlbm_adjoint_uses_graph(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            nlbm_adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pair_list(N: int):
    return [(p, q) for p in range(N) for q in range(p + 1, N)]


def _make_function():
    import torch

    class NPhaseLBM(torch.autograd.Function):
        """phi(T) = step^T(phi0; sigma, mobility) through the CUDA library;
        backward is the library's adjoint (checkpoint every `every` steps).
        sigma_pairs: tensor of the N(N-1)/2 pairwise tensions in the order
        (1,2), (1,3), ..., (N-1,N); mobility: 0-d tensor."""

        @staticmethod
        def forward(ctx, phi0, sigma_pairs, mobility, params, nsteps, every):
            N = int(params["n_phases"])
            sig = np.zeros((N, N))
            for (p, q), v in zip(pair_list(N), sigma_pairs.detach().cpu().double().tolist()):
                sig[p, q] = sig[q, p] = v
            q = dict(params, sigma=sig.tolist(), mobility=float(mobility.detach().cpu()))
            run = AdjointRun(q, nsteps, every, device=phi0.device)
            out = run.forward(phi0.detach())
            ctx.run = run
            ctx.N = N
            ctx.sdtype = sigma_pairs.dtype
            return out

        @staticmethod
        @torch.autograd.function.once_differentiable
        def backward(ctx, grad_out):
            # the run (checkpoints, tapes) is released after one reverse
            # sweep: a second backward through the same graph is refused
            if ctx.run is None:
                raise RuntimeError(
                    "nphase_lbm: the adjoint run was released by the first backward; "
                    "retain_graph=True is not supported -- run the forward again")
            g0, gs, gm = ctx.run.backward(grad_out.contiguous())
            N = ctx.N
            gpairs = torch.tensor([gs[p, q] for p, q in pair_list(N)], dtype=ctx.sdtype)
            ctx.run.close()
            ctx.run = None
            return g0, gpairs, torch.tensor(gm, dtype=ctx.sdtype), None, None, None

    return NPhaseLBM


_FN = None


def nphase_lbm(phi0, sigma_pairs, mobility, params: dict, nsteps: int, every: int = 50):
    """Differentiable N-phase LBM run (autograd through the CUDA adjoint)."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(phi0, sigma_pairs, mobility, params, nsteps, every)
