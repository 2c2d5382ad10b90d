"""Thin ctypes binding of the C ABI in include/lbm3.h (argument marshalling only: every step of
the method runs in the sm_103a kernels of liblbm3.so).

The functions keep the C names (``lbm3_create``, ``lbm3_step`` ...); ``Lbm3`` wraps a handle.
There is no CPU fallback: loading fails loudly when the library or a GPU is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm3.so")

LBM3_OK = 0
LBM3_WARN_YOUNG = 1
LBM3_ERR_INVALID = -1
LBM3_ERR_CUDA = -2
LBM3_ERR_OOM = -3
LBM3_ERR_DIVERGED = -4
LBM3_ERR_STATE = -5
LBM3_ERR_TOO_LARGE = -6
LBM3_FP32, LBM3_FP16, LBM3_BF16 = 0, 1, 2

# every entry point declared in include/lbm3.h
EXPORTS = ("lbm3_create", "lbm3_set_fields", "lbm3_step", "lbm3_step_timed",
           "lbm3_step_timed_detail", "lbm3_fields",
           "lbm3_diag", "lbm3_n_wall", "lbm3_wall_nodes", "lbm3_wall_values", "lbm3_get_state",
           "lbm3_set_state", "lbm3_set_wall_angles", "lbm3_set_inflow", "lbm3_adjoint_centroid",
           "lbm3_adjoint_release", "lbm3_info", "lbm3_set_stream", "lbm3_set_copy_wait_limit", "lbm3_sync",
           "lbm3_destroy", "lbm3_last_error", "lbm3_diag_fields")


class lbm3_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("bc_x", ctypes.c_int32), ("u_in", ctypes.c_double), ("rho_out", ctypes.c_double),
                ("precision", ctypes.c_int32)]


class Lbm3Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbm3 error {code}: {msg}")
        self.code = code


_D = ctypes.POINTER(ctypes.c_double)
_lib = None


def load(path: str | None = None):
    """Load liblbm3.so (built by ``paper_2102_04709_gb300.build``, or the file named by the
    LBM3_LIB environment variable); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("LBM3_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2102_04709_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.lbm3_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(lbm3_grid),
                              ctypes.POINTER(ctypes.c_uint8), _D, _D, _D, ctypes.c_double, vp]
    L.lbm3_create.restype = ctypes.c_int
    L.lbm3_set_fields.argtypes = [vp, _D]
    L.lbm3_step.argtypes = [vp, ctypes.c_int32]
    L.lbm3_step_timed.argtypes = [vp, ctypes.c_int32, _D]
    L.lbm3_step_timed_detail.argtypes = [vp, ctypes.c_int32, _D]
    L.lbm3_fields.argtypes = [vp, _D, _D]
    L.lbm3_diag.argtypes = [vp, _D]
    L.lbm3_n_wall.argtypes = [vp]
    L.lbm3_wall_nodes.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]
    L.lbm3_wall_values.argtypes = [vp, _D, ctypes.c_int32]
    L.lbm3_get_state.argtypes = [vp, _D, _D]
    L.lbm3_set_state.argtypes = [vp, _D, _D]
    L.lbm3_set_wall_angles.argtypes = [vp, _D]
    L.lbm3_set_inflow.argtypes = [vp, ctypes.c_double]
    L.lbm3_adjoint_centroid.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, _D, _D, _D]
    L.lbm3_adjoint_release.argtypes = [vp]
    L.lbm3_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.lbm3_set_stream.argtypes = [vp, vp]
    L.lbm3_set_copy_wait_limit.argtypes = [vp, ctypes.c_int32]
    L.lbm3_sync.argtypes = [vp]
    L.lbm3_destroy.argtypes = [vp]
    L.lbm3_destroy.restype = None
    L.lbm3_last_error.argtypes = [vp]
    L.lbm3_diag_fields.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int32, vp, vp]
    L.lbm3_last_error.restype = ctypes.c_char_p
    for name in ("lbm3_set_fields", "lbm3_step", "lbm3_step_timed", "lbm3_step_timed_detail", "lbm3_fields", "lbm3_diag", "lbm3_n_wall",
                 "lbm3_wall_nodes", "lbm3_wall_values", "lbm3_get_state", "lbm3_set_state", "lbm3_info", "lbm3_set_stream",
                 "lbm3_set_copy_wait_limit", "lbm3_sync"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(_D)


def _check(h, code):
    if code < 0:
        msg = load().lbm3_last_error(h)
        raise Lbm3Error(code, msg.decode() if msg else "")
    return code


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(None)


def diag_fields(rho, u, solid, nx, ny, out, stream=None):
    """``lbm3_diag_fields`` on caller-owned device buffers given as integer addresses (float
    rho [3][ny][nx], float u [2][ny][nx], uint8 solid [ny][nx], double out [8]); enqueues on
    ``stream`` (default: torch's current stream) and returns without synchronising."""
    s = _torch_stream() if stream is None else ctypes.c_void_p(stream)
    code = load().lbm3_diag_fields(rho, u, solid, int(nx), int(ny), out, s)
    if code < 0:
        raise Lbm3Error(code, {LBM3_ERR_INVALID: "NULL buffer or nx, ny <= 0",
                               LBM3_ERR_TOO_LARGE: "grid larger than the fixed scratch accepts",
                               LBM3_ERR_CUDA: "scratch lookup or launch failed"}.get(code, ""))
    return code


class Lbm3:
    """One GPU simulation owned by a C-ABI handle."""

    def __init__(self, nx, ny, periodic_y, bc_x, solid, angles, sigma, nu, beta0=0.7, u_in=0.0,
                 rho_out=1.0, precision=LBM3_FP32, stream=None):
        L = load()
        self.nx, self.ny = int(nx), int(ny)
        self.n = self.nx * self.ny
        solid = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        angles = np.ascontiguousarray(angles, dtype=np.float64).reshape(-1)
        if solid.size != self.n or angles.size != 3 * self.n:
            raise ValueError("solid must be [ny, nx] and angles [ny, nx, 3]")
        sig = np.ascontiguousarray(sigma, dtype=np.float64)
        nus = np.ascontiguousarray(nu, dtype=np.float64)
        g = lbm3_grid(self.nx, self.ny, int(periodic_y), int(bc_x), float(u_in), float(rho_out),
                      int(precision))
        h = ctypes.c_void_p()
        st = stream if stream is not None else _torch_stream()
        code = L.lbm3_create(ctypes.byref(h), ctypes.byref(g),
                             solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dp(angles),
                             _dp(sig), _dp(nus), float(beta0), st)
        if code < 0:
            raise Lbm3Error(code, L.lbm3_last_error(None).decode())
        self._h = h
        self.bc_x = int(bc_x)
        self.warning = L.lbm3_last_error(h).decode() if code > 0 else ""

    @classmethod
    def from_workload(cls, w, precision=LBM3_FP32, stream=None, init=True):
        s = cls(w.nx, w.ny, w.periodic_y, w.bc_x, w.solid, w.angles, w.sigma, w.nu, w.beta0,
                w.u_in, w.rho_out, precision=precision, stream=stream)
        if init:
            s.set_fields(w.rho)
        return s

    def close(self):
        if getattr(self, "_h", None):
            load().lbm3_destroy(self._h)
            self._h = None

    __del__ = close

    def set_fields(self, rho):
        r = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        if r.size != 3 * self.n:
            raise ValueError("rho must be [3, ny, nx]")
        _check(self._h, load().lbm3_set_fields(self._h, _dp(r)))

    def step(self, n=1):
        _check(self._h, load().lbm3_step(self._h, int(n)))

    def step_timed(self, n):
        """Advance n steps; return CUDA-event times in ms summed over the steps:
        (wetting pass, fused kernel on pure tiles, fused kernel on the other tiles)."""
        out = np.zeros(3)
        _check(self._h, load().lbm3_step_timed(self._h, int(n), _dp(out)))
        return float(out[0]), float(out[1]), float(out[2])

    def step_timed_detail(self, n):
        """Advance n steps; return CUDA-event times in ms summed over the steps: (wetting pass,
        pure tiles, wall tiles, edge tiles, the whole run on the device)."""
        out = np.zeros(5)
        _check(self._h, load().lbm3_step_timed_detail(self._h, int(n), _dp(out)))
        return tuple(float(v) for v in out)

    def fields(self):
        rho = np.empty(3 * self.n)
        u = np.empty(2 * self.n)
        _check(self._h, load().lbm3_fields(self._h, _dp(rho), _dp(u)))
        return rho.reshape(3, self.ny, self.nx), u.reshape(2, self.ny, self.nx)

    def diag(self, check=True):
        out = np.empty(8)
        code = load().lbm3_diag(self._h, _dp(out))
        if check:
            _check(self._h, code)
        return out

    def wall_nodes(self):
        n = load().lbm3_n_wall(self._h)
        idx = np.empty(max(n, 1), np.int32)
        _check(self._h, load().lbm3_wall_nodes(self._h, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n))
        return idx[:n]

    def wall_values(self):
        n = load().lbm3_n_wall(self._h)
        c = np.empty((max(n, 1), 3))
        _check(self._h, load().lbm3_wall_values(self._h, _dp(c), n))
        return c[:n]

    def get_state(self):
        f = np.empty(27 * self.n)
        c = np.empty(3 * self.n)
        _check(self._h, load().lbm3_get_state(self._h, _dp(f), _dp(c)))
        return f.reshape(3, 9, self.ny, self.nx), c.reshape(3, self.ny, self.nx)

    def set_state(self, f_post, wall_c):
        f = np.ascontiguousarray(f_post, dtype=np.float64).reshape(-1)
        c = np.ascontiguousarray(wall_c, dtype=np.float64).reshape(-1)
        if f.size != 27 * self.n or c.size != 3 * self.n:
            raise ValueError("f_post must be [3, 9, ny, nx] and wall_c [3, ny, nx]")
        _check(self._h, load().lbm3_set_state(self._h, _dp(f), _dp(c)))

    def set_wall_angles(self, angles):
        """angles: [n_wall, 3] (theta_01, theta_20, theta_12) in degrees, lbm3_wall_nodes order."""
        a = np.ascontiguousarray(angles, dtype=np.float64).reshape(-1)
        if a.size != 3 * load().lbm3_n_wall(self._h):
            raise ValueError("angles must be [n_wall, 3]")
        _check(self._h, load().lbm3_set_wall_angles(self._h, _dp(a)))

    def set_inflow(self, u_in):
        _check(self._h, load().lbm3_set_inflow(self._h, float(u_in)))

    def adjoint_centroid(self, nsteps, checkpoint_every=100):
        """(J, dJ/d angles [n_wall, 3], dJ/du_in) for J = x-centroid of fluid 0 after nsteps."""
        n = load().lbm3_n_wall(self._h)
        J = np.zeros(1)
        dang = np.zeros(3 * max(n, 1))
        du = np.zeros(1)
        _check(self._h, load().lbm3_adjoint_centroid(self._h, int(nsteps), int(checkpoint_every),
                                                     _dp(J), _dp(dang), _dp(du)))
        return float(J[0]), dang[:3 * n].reshape(n, 3), float(du[0])

    def adjoint_release(self):
        """Release the device memory adjoint_centroid keeps for its next call."""
        _check(self._h, load().lbm3_adjoint_release(self._h))

    def info(self):
        out = np.zeros(9, np.int64)
        _check(self._h, load().lbm3_info(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return {"n_fluid": int(out[0]), "n_wall": int(out[1]), "step_bytes": int(out[2]),
                "step_kernels": int(out[3]), "wet_kernels": int(out[4]), "device_bytes": int(out[5]),
                "pure_bytes": int(out[6]), "pure_nodes": int(out[7]), "tma": bool(out[8]),
                "pure_kernel": {0: "plain", 1: "bulk copies", 2: "ring"}[int(out[8])]}

    def set_stream(self, stream):
        _check(self._h, load().lbm3_set_stream(self._h, stream))

    def set_copy_wait_limit(self, polls):
        """Polls of a tile's bulk-copy mbarrier before a block gives up (< 0: the default)."""
        _check(self._h, load().lbm3_set_copy_wait_limit(self._h, int(polls)))

    def sync(self):
        _check(self._h, load().lbm3_sync(self._h))
