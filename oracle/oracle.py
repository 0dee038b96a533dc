"""ctypes binding of the FP64 C oracle (``nlbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA library never does.  The C source is
compiled here with the host compiler (gcc, OpenMP) into ``oracle/_build``.

Parameters are passed as a plain dict with the keys the workload generator
produces: nx, ny, n_phases, model ('A' or 'B'), model_a_n, eps, mobility,
rho[N], mu[N] (dynamic viscosities), sigma[N][N], wall_x, wall_y, and
optionally unit_delta, gx, gy (gravity, F_g = rho g) and wall_cos (2 (N-1)
cosines of the contact angles against phase N at the walls y = 0 and
y = ny - 1, Sec. 4.2).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nlbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB32 = os.path.join(_BUILD, "liboracle_fp32.so")
MAXN = 8

_lock = threading.Lock()
_lib = None
_lib32 = None


class params_struct(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("n_phases", ctypes.c_int32), ("model", ctypes.c_int32),
        ("wall_x", ctypes.c_int32), ("wall_y", ctypes.c_int32),
        ("solve_all", ctypes.c_int32), ("store16", ctypes.c_int32),
        ("model_a_n", ctypes.c_double), ("eps", ctypes.c_double),
        ("mobility", ctypes.c_double),
        ("rho", ctypes.c_double * MAXN), ("mu", ctypes.c_double * MAXN),
        ("sigma", ctypes.c_double * (MAXN * MAXN)),
        ("unit_delta", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("wall_cos", ctypes.c_double * (2 * MAXN)),
    ]


def _compile(out: str, extra) -> None:
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           *extra, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build_oracle(force: bool = False) -> str:
    """Compile the FP64 oracle and its FP32 noise-model build (idempotent,
    mtime-checked); returns the FP64 library path."""
    os.makedirs(_BUILD, exist_ok=True)
    for out, extra in ((_LIB, []), (_LIB32, ["-DORACLE_FP32", "-fsingle-precision-constant"])):
        if (force or not os.path.exists(out)
                or os.path.getmtime(out) < os.path.getmtime(_SRC)):
            _compile(out, extra)
    return _LIB


def _declare_sim(lib, real):
    P = ctypes.POINTER
    lib.or_create.restype = ctypes.c_void_p
    lib.or_create.argtypes = [P(params_struct)]
    lib.or_destroy.argtypes = [ctypes.c_void_p]
    lib.or_set_phi.argtypes = [ctypes.c_void_p, P(real)]
    lib.or_step.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int]
    lib.or_get_moments.argtypes = [ctypes.c_void_p, P(real), P(real), P(real)]
    lib.or_phase_mass.argtypes = [ctypes.c_void_p, P(real)]
    lib.or_get_field.argtypes = [ctypes.c_void_p, ctypes.c_int, P(real)]
    lib.or_set_velocity.argtypes = [ctypes.c_void_p, P(real)]
    lib.or_steps_done.restype = ctypes.c_longlong
    lib.or_steps_done.argtypes = [ctypes.c_void_p]
    lib.or_max_threads.restype = ctypes.c_int


def oracle_lib_fp32():
    """The FP32 build of the same source: a noise model, never a reference."""
    global _lib32
    with _lock:
        if _lib32 is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB32)
            _declare_sim(lib, ctypes.c_float)
            _lib32 = lib
    return _lib32


def oracle_lib():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            P = ctypes.POINTER
            d = ctypes.c_double
            _declare_sim(lib, d)
            lib.or_field_grad.argtypes = [P(d), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, P(d)]
            lib.or_field_lap.argtypes = lib.or_field_grad.argtypes
            lib.or_point_source.argtypes = [P(params_struct), P(d), P(d), P(d)]
            lib.or_point_chempot.argtypes = [P(params_struct), P(d), P(d), P(d)]
            lib.or_mrt_matrices.argtypes = [P(d), P(d)]
            lib.or_phase_feq.argtypes = [d, d, d, P(d)]
            lib.or_phase_src.argtypes = [d, d, d, d, P(d)]
            lib.or_flow_geq.argtypes = [d, d, d, d, d, d, d, P(d)]
            lib.or_flow_force.argtypes = [d, d, d, P(d), P(d)]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(p: dict, solve_all: bool = False, store16: int = 0) -> params_struct:
    s = params_struct()
    s.store16 = int(store16)
    N = int(p["n_phases"])
    s.nx, s.ny, s.n_phases = int(p["nx"]), int(p["ny"]), N
    s.model = {"A": 0, "B": 1}[p["model"]]
    s.wall_x, s.wall_y = int(bool(p.get("wall_x", 0))), int(bool(p.get("wall_y", 0)))
    s.solve_all = int(bool(solve_all))
    s.model_a_n = float(p.get("model_a_n", 1.0))
    s.eps, s.mobility = float(p["eps"]), float(p["mobility"])
    s.unit_delta = float(p.get("unit_delta", 0.0))
    s.gx, s.gy = float(p.get("gx", 0.0)), float(p.get("gy", 0.0))
    # wetting: cos theta_pN of the wall at y = 0 (first N-1) and at y = ny - 1
    wc = p.get("wall_cos")
    if wc is not None:
        wc = [float(v) for v in wc]
        if len(wc) != 2 * (N - 1):
            raise ValueError("wall_cos holds 2 (N - 1) cosines")
        for a in range(N - 1):
            s.wall_cos[a] = wc[a]
            s.wall_cos[MAXN + a] = wc[N - 1 + a]
    sig = np.asarray(p["sigma"], dtype=np.float64).reshape(N, N)
    for a in range(N):
        s.rho[a] = float(p["rho"][a])
        s.mu[a] = float(p["mu"][a])
        for b in range(N):
            s.sigma[a * MAXN + b] = float(sig[a, b])
    return s


class OracleSim:
    """One FP64 oracle simulation.  ``phi0`` holds phases 1..N-1 as
    [N-1, ny, nx]; phase N is 1 - sum."""

    def __init__(self, p: dict, phi0: np.ndarray, solve_all: bool = False, threads: int = 0,
                 fp32: bool = False, store16: int = 0):
        """fp32=True runs the FP32 noise-model build instead of the oracle;
        store16 (1 bfloat16, 2 binary16; noise-model build only) adds the
        rounding of 16-bit population storage to that noise model."""
        if store16 and not fp32:
            raise ValueError("16-bit storage rounding exists only in the FP32 noise model")
        self.fp32 = fp32
        self.lib = oracle_lib_fp32() if fp32 else oracle_lib()
        self._dt = np.float32 if fp32 else np.float64
        self._ct = ctypes.c_float if fp32 else ctypes.c_double
        self.p = dict(p)
        self.N, self.nx, self.ny = int(p["n_phases"]), int(p["nx"]), int(p["ny"])
        self.threads = threads
        self._ps = make_params(p, solve_all, store16)
        self.h = self.lib.or_create(ctypes.byref(self._ps))
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        phi0 = np.ascontiguousarray(phi0, dtype=self._dt)
        assert phi0.shape == (self.N - 1, self.ny, self.nx), phi0.shape
        self.lib.or_set_phi(self.h, self._p(phi0))

    def set_velocity(self, u0: np.ndarray):
        """Start in motion: u0 [2, ny, nx] (or a pair (ux, uy) for a uniform
        flow); populations at their equilibria, previous values equal to the
        initial ones (see or_set_velocity)."""
        u0 = np.asarray(u0, dtype=np.float64)
        if u0.shape == (2,):
            u0 = np.broadcast_to(u0[:, None, None], (2, self.ny, self.nx))
        u0 = np.ascontiguousarray(u0, dtype=self._dt)
        assert u0.shape == (2, self.ny, self.nx), u0.shape
        self.lib.or_set_velocity(self.h, self._p(u0))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_destroy(h)
            self.h = None

    def step(self, n: int):
        self.lib.or_step(self.h, int(n), int(self.threads))

    @property
    def steps_done(self) -> int:
        return int(self.lib.or_steps_done(self.h))

    def _p(self, a):
        return a.ctypes.data_as(ctypes.POINTER(self._ct))

    def moments(self):
        """(phi [N,ny,nx], u [2,ny,nx], P [ny,nx]) as float64 arrays."""
        phi = np.empty((self.N, self.ny, self.nx), dtype=self._dt)
        u = np.empty((2, self.ny, self.nx), dtype=self._dt)
        P = np.empty((self.ny, self.nx), dtype=self._dt)
        self.lib.or_get_moments(self.h, self._p(phi), self._p(u), self._p(P))
        return phi.astype(np.float64), u.astype(np.float64), P.astype(np.float64)

    def phase_mass(self) -> np.ndarray:
        m = np.empty(self.N, dtype=self._dt)
        self.lib.or_phase_mass(self.h, self._p(m))
        return m.astype(np.float64)

    def field(self, name: str) -> np.ndarray:
        N, ny, nx = self.N, self.ny, self.nx
        which, shape = {
            "R": (0, (N, 2, ny, nx)), "mphi": (1, (2, ny, nx)), "muphi": (2, (N, ny, nx)),
            "F": (3, (2, ny, nx)), "grad": (4, (N, 2, ny, nx)), "lap": (5, (N, ny, nx)),
            "Fc": (6, (2, ny, nx)),
        }[name]
        out = np.empty(shape, dtype=self._dt)
        self.lib.or_get_field(self.h, which, self._p(out))
        return out.astype(np.float64)


# ---------------------------------------------------------------- field pins

def field_grad(chi: np.ndarray, wall_x=False, wall_y=False) -> np.ndarray:
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    ny, nx = chi.shape
    out = np.empty((2, ny, nx))
    oracle_lib().or_field_grad(_dp(chi), nx, ny, int(wall_x), int(wall_y), _dp(out))
    return out


def field_lap(chi: np.ndarray, wall_x=False, wall_y=False) -> np.ndarray:
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    ny, nx = chi.shape
    out = np.empty((ny, nx))
    oracle_lib().or_field_lap(_dp(chi), nx, ny, int(wall_x), int(wall_y), _dp(out))
    return out


def point_source(p: dict, phi: np.ndarray, grad: np.ndarray) -> np.ndarray:
    N = int(p["n_phases"])
    ps = make_params({**p, "nx": 1, "ny": 1})
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    grad = np.ascontiguousarray(grad, dtype=np.float64).reshape(N, 2)
    R = np.empty((N, 2))
    oracle_lib().or_point_source(ctypes.byref(ps), _dp(phi), _dp(grad), _dp(R))
    return R


def point_chempot(p: dict, phi: np.ndarray, lap: np.ndarray) -> np.ndarray:
    N = int(p["n_phases"])
    ps = make_params({**p, "nx": 1, "ny": 1})
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    lap = np.ascontiguousarray(lap, dtype=np.float64)
    mu = np.empty(N)
    oracle_lib().or_point_chempot(ctypes.byref(ps), _dp(phi), _dp(lap), _dp(mu))
    return mu


def mrt_matrices():
    M = np.empty((9, 9))
    Mi = np.empty((9, 9))
    oracle_lib().or_mrt_matrices(_dp(M), _dp(Mi))
    return M, Mi


def phase_feq(phi, ux, uy):
    out = np.empty(9)
    oracle_lib().or_phase_feq(phi, ux, uy, _dp(out))
    return out


def phase_src(dtx, dty, Rx, Ry):
    out = np.empty(9)
    oracle_lib().or_phase_src(dtx, dty, Rx, Ry, _dp(out))
    return out


def flow_geq(P, rho0, rho, ux, uy, mx, my):
    out = np.empty(9)
    oracle_lib().or_flow_geq(P, rho0, rho, ux, uy, mx, my, _dp(out))
    return out


def flow_force(ugr, Fx, Fy, M2F):
    M2F = np.ascontiguousarray(np.asarray(M2F, dtype=np.float64).reshape(4))
    out = np.empty(9)
    oracle_lib().or_flow_force(ugr, Fx, Fy, _dp(M2F), _dp(out))
    return out


def max_threads() -> int:
    return int(oracle_lib().or_max_threads())


# ------------------------------------------------------- closed-form lens pin

def lens_equilibrium(sigma_layer: float, sigma_cap_a: float, sigma_cap_b: float, S: float):
    """Equilibrium of a lens of area S floating on a flat interface without
    gravity (Sec. 4.3): Neumann's law fixes the angle each cap makes with the
    layer interface (law of cosines on the triangle of the three tensions:
    cos theta_a = (s_layer^2 + s_a^2 - s_b^2) / (2 s_layer s_a)), each cap is
    a circular arc, and the area fixes the size:
        d / 2 = sqrt(S / sum_i (theta_i / sin theta_i - cos theta_i) / sin theta_i),
        h_i = (d / 2) (1 - cos theta_i) / sin theta_i.
    Cap a is bounded by the interface of tension sigma_cap_a.  Returns
    (d / 2, h_a, h_b, theta_a, theta_b)."""
    sl, sa, sb = float(sigma_layer), float(sigma_cap_a), float(sigma_cap_b)
    ca = (sl * sl + sa * sa - sb * sb) / (2.0 * sl * sa)
    cb = (sl * sl + sb * sb - sa * sa) / (2.0 * sl * sb)
    ta, tb = np.arccos(np.clip(ca, -1.0, 1.0)), np.arccos(np.clip(cb, -1.0, 1.0))
    shape = sum((t / np.sin(t) - np.cos(t)) / np.sin(t) for t in (ta, tb))
    half_d = np.sqrt(S / shape)
    ha = half_d * (1.0 - np.cos(ta)) / np.sin(ta)
    hb = half_d * (1.0 - np.cos(tb)) / np.sin(tb)
    return half_d, ha, hb, ta, tb


def layer_height(phi: np.ndarray, x: int) -> float:
    """Height of the flat 1|2 interface in column x: where phi_1 - phi_2
    changes sign (linear interpolation)."""
    d = phi[0][:, x] - phi[1][:, x]
    j = int(np.nonzero((d[:-1] > 0) & (d[1:] <= 0))[0][0])
    return j + d[j] / (d[j] - d[j + 1])


def measure_lens(phi: np.ndarray, y_layer: float = None):
    """Half-length d/2 and the cap heights (below, above) of the lens phase
    phi[2] = phase 3 from its 0.5 level set, with linear interpolation: the
    widest chord along the layer height (rows interpolated) and the extent
    below and above it along the lens's centre column.  The layer height is
    measured in the column farthest from the lens unless given: the flat
    interface moves as the lens changes shape, since each layer keeps its
    volume.  Also returns the lens area sum(phi_3)."""
    L = phi[2]
    ny, nx = L.shape
    if y_layer is None:
        xc0 = int(np.argmax(L.sum(axis=0)))
        y_layer = layer_height(phi, (xc0 + nx // 2) % nx)
    j0 = int(np.floor(y_layer))
    t = y_layer - j0
    row = (1.0 - t) * L[j0] + t * L[min(j0 + 1, ny - 1)]

    def extent(v, c):
        # distance from index c (inside, v >= 0.5) to the 0.5 crossing on each side
        n = len(v)
        lo = c
        while lo - 1 >= 0 and v[lo - 1] >= 0.5:
            lo -= 1
        hi = c
        while hi + 1 < n and v[hi + 1] >= 0.5:
            hi += 1
        fl = (lo - 1) + (0.5 - v[lo - 1]) / (v[lo] - v[lo - 1]) if lo > 0 else float(lo)
        fh = hi + (v[hi] - 0.5) / (v[hi] - v[hi + 1]) if hi + 1 < n else float(hi)
        return fl, fh

    c = int(np.argmax(row))
    xl, xh = extent(row, c)
    xc = 0.5 * (xl + xh)
    i0 = int(np.floor(xc))
    s = xc - i0
    col = (1.0 - s) * L[:, i0] + s * L[:, min(i0 + 1, nx - 1)]
    jc = int(round(y_layer))
    if col[jc] < 0.5:
        jc = int(np.argmax(col))
    yl, yh = extent(col, jc)
    return 0.5 * (xh - xl), y_layer - yl, yh - y_layer, float(L.sum())
