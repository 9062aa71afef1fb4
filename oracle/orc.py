"""Python handle on the FP64 CPU oracle (``orc.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this module; the product package never
imports it.  The oracle is the plain restatement of the MRT lattice Boltzmann
model of Liu, He, Li and Tao (arXiv:1308.2071), Sections 2-4; see ``orc.h`` for
the step order and the readings it takes where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles ``orc.c`` with gcc (-O2 -ffp-contract=off) into ``_build/liborc.so``."""
    src = os.path.join(_HERE, "orc.c")
    hdr = os.path.join(_HERE, "orc.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-D_POSIX_C_SOURCE=200809L",
           "-fPIC", "-shared", "-pthread", "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Physical(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("Ra", C.c_double), ("Da", C.c_double), ("Pr", C.c_double), ("J", C.c_double),
                ("phi", C.c_double), ("Ma", C.c_double), ("sigma", C.c_double),
                ("varpi", C.c_double), ("Th", C.c_double), ("Tc", C.c_double),
                ("RaI", C.c_double), ("thermal_bc", C.c_int)]


class Lattice(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("rho0", C.c_double), ("T0", C.c_double),
                ("s", C.c_double * 9), ("zeta", C.c_double * 5),
                ("nu", C.c_double), ("phi_bar", C.c_double), ("K_bar", C.c_double),
                ("forchheimer", C.c_int),
                ("gbeta", C.c_double), ("Gx", C.c_double), ("Gy", C.c_double),
                ("sigma", C.c_double), ("varpi", C.c_double), ("Q", C.c_double),
                ("Th", C.c_double), ("Tc", C.c_double), ("L", C.c_double), ("dT", C.c_double),
                ("periodic_x", C.c_int), ("periodic_y", C.c_int),
                ("thermal_bc", C.c_int), ("adiabatic_order", C.c_int)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            D = C.POINTER(C.c_double)
            L.orc_derive.argtypes = [C.POINTER(Physical), C.POINTER(Lattice)]
            L.orc_create.argtypes = [C.POINTER(Lattice), C.c_void_p]
            L.orc_create.restype = C.c_void_p
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_step.argtypes = [C.c_void_p, C.c_long, C.c_int]
            L.orc_time.argtypes = [C.c_void_p]
            L.orc_time.restype = C.c_long
            L.orc_get_state.argtypes = [C.c_void_p, _dp, _dp]
            L.orc_set_state.argtypes = [C.c_void_p, _dp, _dp]
            L.orc_macros.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
            L.orc_nusselt.argtypes = [C.c_void_p, D, D]
            I = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
            L.orc_velocities.argtypes = [I, I, I, I]
            for name in ("orc_matrix_M", "orc_matrix_Minv", "orc_matrix_N", "orc_matrix_Ninv"):
                getattr(L, name).argtypes = [_dp]
            L.orc_feq.argtypes = [C.c_double, C.c_double, _dp, C.c_double, _dp]
            L.orc_meq.argtypes = [C.c_double, C.c_double, _dp, C.c_double, _dp]
            L.orc_force_moments.argtypes = [C.c_double, _dp, _dp, C.c_double, _dp]
            L.orc_geq.argtypes = [C.c_double, _dp, C.c_double, C.c_double, _dp]
            L.orc_neq.argtypes = [C.c_double, _dp, C.c_double, C.c_double, _dp]
            L.orc_velocity.argtypes = [C.c_double, _dp, C.c_double, C.c_double, C.c_double,
                                       C.c_double, _dp, _dp]
            L.orc_pressure.argtypes = [C.c_double, _dp, _dp, C.c_double]
            L.orc_pressure.restype = C.c_double
            L.orc_ergun.argtypes = [C.c_double, C.c_double, D, D]
            L.orc_collide.argtypes = [C.POINTER(Lattice), C.c_double, _dp, _dp, _dp, C.c_double,
                                      C.c_double, _dp, _dp, _dp]
            _lib = L
    return _lib


def derive(nx, ny, Ra, Da, phi, Pr=1.0, J=1.0, Ma=0.1, sigma=1.0, varpi=-2.0,
           Th=1.0, Tc=0.0, RaI=0.0, thermal_bc=0) -> Lattice:
    """Lattice parameters of a cavity (Eq. 37 second occurrence, Section 4)."""
    ph = Physical(nx, ny, Ra, Da, Pr, J, phi, Ma, sigma, varpi, Th, Tc, RaI, thermal_bc)
    lat = Lattice()
    lib().orc_derive(C.byref(ph), C.byref(lat))
    return lat


class Oracle:
    """One oracle run.  State = post-stream, post-wall-rule populations."""

    def __init__(self, lat: Lattice, phi_field: np.ndarray | None = None):
        self.lat = lat
        self.nx, self.ny = lat.nx, lat.ny
        self._phi = None
        ptr = None
        if phi_field is not None:
            self._phi = np.ascontiguousarray(phi_field, dtype=np.float64).reshape(self.ny, self.nx)
            ptr = self._phi.ctypes.data
        self._h = lib().orc_create(C.byref(lat), ptr)
        if not self._h:
            raise ValueError("oracle rejected the lattice parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def t(self) -> int:
        return lib().orc_time(self._h)

    def step(self, n: int, threads: int = 1) -> "Oracle":
        lib().orc_step(self._h, int(n), int(threads))
        return self

    def state(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((5, self.ny, self.nx))
        lib().orc_get_state(self._h, f, g)
        return f, g

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx) and g.shape == (5, self.ny, self.nx)
        lib().orc_set_state(self._h, f, g)

    def macros(self):
        """Returns (ux, uy, p, T), each (ny, nx)."""
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        lib().orc_macros(self._h, *out)
        return tuple(out)

    def nusselt(self):
        a, b = C.c_double(), C.c_double()
        lib().orc_nusselt(self._h, C.byref(a), C.byref(b))
        return a.value, b.value
