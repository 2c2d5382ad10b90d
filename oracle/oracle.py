"""ctypes wrapper of the FP64 CPU oracle (``lbm3_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline
and reference legs are the only users.  The product package never imports this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm3_oracle.c")
_LIB = os.path.join(_HERE, "liblbm3_oracle.so")
_TAPE_SRC = os.path.join(_HERE, "lbm3_oracle_tape.cpp")
_TAPE_LIB = os.path.join(_HERE, "liblbm3_oracle_tape.so")
_lib = None
_tape = None

_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: it must build on x86 and Arm), with
    OpenMP where the compiler has it (the per-node loops then run on ``threads`` threads; the
    results do not depend on the thread count) and without it otherwise."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
                "-o", tmp, _SRC, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def build_tape(force: bool = False) -> str:
    """Compile the reference tape: the oracle's source again, with a recording scalar type, and
    its reverse sweep (g++, portable flags)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_TAPE_SRC))
    if force or not os.path.exists(_TAPE_LIB) or os.path.getmtime(_TAPE_LIB) < newest:
        tmp = _TAPE_LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-Wno-unknown-pragmas", "-o", tmp, _TAPE_SRC])
        os.replace(tmp, _TAPE_LIB)
    return _TAPE_LIB


def tape_lib():
    global _tape
    if _tape is None:
        build_tape()
        T = ctypes.CDLL(_TAPE_LIB)
        T.tape_centroid_gradient.restype = ctypes.c_int
        T.tape_centroid_gradient.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, _U8, _D, _D, _D,
                                             ctypes.c_double, _D, ctypes.c_int, _D, _D, _D]
        _tape = T
    return _tape


def tape_centroid_gradient(w, steps, angles=None, u_in=None):
    """Reference tape of the oracle: (J, dJ/dangles [ny, nx, 3], dJ/du_in) for J = x-centroid of
    fluid 0 after `steps` oracle steps of workload w from its initial densities (angles and u_in
    default to the workload's)."""
    ang = _c(w.angles if angles is None else angles).reshape(-1)
    u = float(w.u_in if u_in is None else u_in)
    solid = _c(w.solid, np.uint8).reshape(-1)
    rho = _c(w.rho).reshape(-1)
    J = np.zeros(1)
    g = np.zeros(3 * w.nx * w.ny)
    du = np.zeros(1)
    rc = tape_lib().tape_centroid_gradient(
        int(w.nx), int(w.ny), int(w.periodic_y), int(w.bc_x), u, float(w.rho_out),
        solid.ctypes.data_as(_U8), _dp(ang), _dp(_c(w.sigma)), _dp(_c(w.nu)), float(w.beta0),
        _dp(rho), int(steps), _dp(J), _dp(g), _dp(du))
    if rc != 0:
        raise ValueError("oracle tape: invalid configuration")
    return float(J[0]), g.reshape(w.ny, w.nx, 3), float(du[0])


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.ora_create.restype = ctypes.c_void_p
        L.ora_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_double, _U8, _D, _D, _D,
                                 ctypes.c_double]
        for name in ("ora_destroy",):
            getattr(L, name).argtypes = [ctypes.c_void_p]
        L.ora_check.argtypes = [ctypes.c_void_p]
        L.ora_check.restype = ctypes.c_int
        L.ora_set_fields.argtypes = [ctypes.c_void_p, _D]
        L.ora_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.ora_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.ora_fields.argtypes = [ctypes.c_void_p, _D, _D]
        L.ora_diag.argtypes = [ctypes.c_void_p, _D]
        for name in ("ora_get_f", "ora_set_f", "ora_get_normals", "ora_get_wallC",
                     "ora_get_force"):
            getattr(L, name).argtypes = [ctypes.c_void_p, _D]
        L.ora_get_classes.argtypes = [ctypes.c_void_p, _U8]
        L.ora_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  _D, _D, _D]
        L.ora_collide.argtypes = [_D, _D, ctypes.c_double, _D, _D]
        L.ora_gfun.argtypes = [ctypes.c_double]
        L.ora_gfun.restype = ctypes.c_double
        L.ora_gradient_periodic.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        L.ora_beta.argtypes = [ctypes.c_void_p, _D, _D]
        L.ora_wet_probe.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, _D, _D]
        L.ora_local_angles.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, _D]
        L.ora_gradient_at.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, ctypes.c_int, _D]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


class Oracle:
    """One oracle simulation: geometry, parameters and FP64 state."""

    def __init__(self, nx, ny, periodic_y, bc_x, solid, angles, sigma, nu, beta0=0.7,
                 u_in=0.0, rho_out=1.0, threads=1):
        L = lib()
        self.nx, self.ny = int(nx), int(ny)
        self.n = self.nx * self.ny
        self._solid = _c(solid, np.uint8).reshape(-1)
        self._angles = _c(angles).reshape(-1)
        assert self._solid.size == self.n and self._angles.size == 3 * self.n
        sig = _c(sigma)
        nus = _c(nu)
        self._h = L.ora_create(self.nx, self.ny, int(periodic_y), int(bc_x), float(u_in),
                               float(rho_out), self._solid.ctypes.data_as(_U8),
                               _dp(self._angles), _dp(sig), _dp(nus), float(beta0))
        code = L.ora_check(self._h)
        if code != 0:
            L.ora_destroy(self._h)
            self._h = None
            raise ValueError(f"oracle: invalid configuration (code {code})")
        self.set_threads(threads)

    @classmethod
    def from_workload(cls, w, threads=1):
        o = cls(w.nx, w.ny, w.periodic_y, w.bc_x, w.solid, w.angles, w.sigma, w.nu, w.beta0,
                w.u_in, w.rho_out, threads=threads)
        o.set_fields(w.rho)
        return o

    def set_threads(self, n):
        """OpenMP threads of the per-node loops (0 or None: every host core)."""
        n = host_threads() if not n else int(n)
        lib().ora_set_threads(self._h, n)
        self.threads = n

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ora_destroy(self._h)
            self._h = None

    def set_fields(self, rho):
        r = _c(rho).reshape(-1)
        assert r.size == 3 * self.n
        lib().ora_set_fields(self._h, _dp(r))

    def step(self, n=1):
        lib().ora_step(self._h, int(n))

    def fields(self):
        rho = np.empty(3 * self.n)
        u = np.empty(2 * self.n)
        lib().ora_fields(self._h, _dp(rho), _dp(u))
        return rho.reshape(3, self.ny, self.nx), u.reshape(2, self.ny, self.nx)

    def diag(self):
        out = np.empty(8)
        lib().ora_diag(self._h, _dp(out))
        return out

    def get_f(self):
        f = np.empty(27 * self.n)
        lib().ora_get_f(self._h, _dp(f))
        return f.reshape(3, 9, self.ny, self.nx)

    def set_f(self, f):
        f = _c(f).reshape(-1)
        assert f.size == 27 * self.n
        lib().ora_set_f(self._h, _dp(f))

    def classes(self):
        c = np.empty(self.n, np.uint8)
        lib().ora_get_classes(self._h, c.ctypes.data_as(_U8))
        return c.reshape(self.ny, self.nx)

    def normals(self):
        a = np.empty(2 * self.n)
        lib().ora_get_normals(self._h, _dp(a))
        return a.reshape(self.ny, self.nx, 2)

    def wall_C(self):
        a = np.empty(3 * self.n)
        lib().ora_get_wallC(self._h, _dp(a))
        return a.reshape(3, self.ny, self.nx)

    def force(self):
        a = np.empty(2 * self.n)
        lib().ora_get_force(self._h, _dp(a))
        return a.reshape(2, self.ny, self.nx)

    def beta(self, rho_k):
        out = np.empty(9)
        lib().ora_beta(self._h, _dp(_c(rho_k)), _dp(out))
        return out.reshape(3, 3)

    def wet_probe(self, node, k, theta_k, C):
        C = _c(C).reshape(-1)
        assert C.size == 3 * self.n
        out = np.empty(3)
        lib().ora_wet_probe(self._h, int(node), int(k), float(theta_k), _dp(C), _dp(out))
        return out

    def gradient_at(self, C, x, y):
        """Eq.(12) gradients (3, 2) of the three phase fields at node (x, y) as the step takes
        them, against the phase-field array C (3, ny, nx) holding fluid and C_SB values."""
        C = _c(C).reshape(-1)
        assert C.size == 3 * self.n
        out = np.empty(6)
        lib().ora_gradient_at(self._h, _dp(C), int(x), int(y), _dp(out))
        return out.reshape(3, 2)

    def local_angles(self, node, Cp):
        out = np.empty(2)
        lib().ora_local_angles(self._h, int(node), _dp(_c(Cp)), _dp(out))
        return out


def lattice():
    ex = (ctypes.c_int * 9)()
    ey = (ctypes.c_int * 9)()
    w = np.empty(9)
    M = np.empty(81)
    Mi = np.empty(81)
    lib().ora_lattice(ex, ey, _dp(w), _dp(M), _dp(Mi))
    return np.array(ex[:]), np.array(ey[:]), w, M.reshape(9, 9), Mi.reshape(9, 9)


def collide(f, Fs, tau):
    f = _c(f)
    Fs = _c(Fs)
    out = np.empty(9)
    u = np.empty(2)
    lib().ora_collide(_dp(f), _dp(Fs), float(tau), _dp(out), _dp(u))
    return out, u


def gfun(X):
    return lib().ora_gfun(float(X))


def gradient_periodic(psi):
    psi = _c(psi)
    ny, nx = psi.shape
    out = np.empty(2 * nx * ny)
    lib().ora_gradient_periodic(nx, ny, _dp(psi), _dp(out))
    return out.reshape(2, ny, nx)
