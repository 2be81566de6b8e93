"""ctypes front end of the C oracle (chem_oracle.c) -- test infrastructure only.

Builds `_build/liboracle.so` with gcc (-O2 -fopenmp, no architecture-specific flags, so the same
source builds on x86-64 and aarch64) and exposes per-cell and batched calls on numpy arrays.

State layout used throughout: z = (Y_1..Y_K, T); batches are species-major SoA, Y[k, i].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (gcc, OpenMP); returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build_oracle())
        lib.or_mech_load.restype = C.c_void_p
        lib.or_mech_load.argtypes = [C.c_char_p, C.c_char_p, C.c_int]
        lib.or_mech_free.argtypes = [C.c_void_p]
        lib.or_mech_dims.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_int)]
        lib.or_mech_W.argtypes = [C.c_void_p, _dp]
        lib.or_mech_comp.argtypes = [C.c_void_p, _ip]
        lib.or_species_thermo.argtypes = [C.c_void_p, C.c_double, _dp, _dp, _dp]
        lib.or_rates.argtypes = [C.c_void_p, C.c_double, C.c_double, _dp, _dp, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p]
        lib.or_rhs.argtypes = [C.c_void_p, C.c_double, _dp, _dp]
        lib.or_jacobian.argtypes = [C.c_void_p, C.c_double, _dp, _dp]
        lib.or_integrate.argtypes = [C.c_void_p, C.c_double, _dp, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_int, _ip]
        lib.or_integrate_batch.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_double, _dp,
                                           _dp, _dp, C.c_double, C.c_double, C.c_double, C.c_int,
                                           _ip, _ip, C.c_int]
        lib.or_rk4.argtypes = [C.c_void_p, C.c_double, _dp, C.c_double, C.c_int64]
        lib.or_thermo_props.argtypes = [C.c_void_p, C.c_double, _dp, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
        lib.or_T_from_h.argtypes = [C.c_void_p, C.c_double, _dp, C.c_double,
                                    C.POINTER(C.c_double)]
        lib.or_radau_tableau.argtypes = [_dp, _dp]
        lib.or_radau_fixed.argtypes = [C.c_void_p, C.c_double, _dp, C.c_double, C.c_int]
        lib.or_max_threads.restype = C.c_int
        lib.or_dense_solve.argtypes = [C.c_int, _dp, _dp]
        _lib = lib
        return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


R_GAS = 8.314462618
P0 = 101325.0

# Oracle tolerances for the reference solution of Eq. 2 (far below the 1e-6 parity bar).
ORACLE_RTOL = 1e-10
ORACLE_ATOL_Y = 1e-20
ORACLE_ATOL_T = 1e-10


class Oracle:
    """One parsed mechanism plus the oracle's per-cell functions."""

    def __init__(self, path: str):
        self.lib = _load()
        err = C.create_string_buffer(512)
        h = self.lib.or_mech_load(path.encode(), err, 512)
        if not h:
            raise ValueError(f"oracle: cannot load mechanism: {err.value.decode()}")
        self.h = C.c_void_p(h)
        K, I, E = C.c_int(), C.c_int(), C.c_int()
        self.lib.or_mech_dims(self.h, C.byref(K), C.byref(I), C.byref(E))
        self.K, self.I, self.E = K.value, I.value, E.value
        self.n = self.K + 1
        self.W = np.zeros(self.K)
        self.lib.or_mech_W(self.h, self.W)
        comp = np.zeros(self.K * self.E, dtype=np.int32)
        self.lib.or_mech_comp(self.h, comp)
        self.comp = comp.reshape(self.K, self.E)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.or_mech_free(self.h)
                self.h = None
        except Exception:
            pass

    # -- species thermo
    def species_thermo(self, T: float) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(cp/R, h/RT, s/R) of every species at T (NASA-7)."""
        cp, h, s = np.zeros(self.K), np.zeros(self.K), np.zeros(self.K)
        self.lib.or_species_thermo(self.h, float(T), cp, h, s)
        return cp, h, s

    # -- kinetics
    def rates(self, T: float, p: float, Y: np.ndarray, with_rxn: bool = False):
        """wdot [K] mol/m^3/s and HRR W/m^3 (and per-reaction q, kf, kr if asked)."""
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        wdot = np.zeros(self.K)
        hrr = np.zeros(1)
        q = np.zeros(max(self.I, 1)) if with_rxn else None
        kf = np.zeros(max(self.I, 1)) if with_rxn else None
        kr = np.zeros(max(self.I, 1)) if with_rxn else None
        self.lib.or_rates(self.h, float(T), float(p), Y, wdot, _ptr(hrr), _ptr(q), _ptr(kf),
                          _ptr(kr))
        if with_rxn:
            return wdot, hrr[0], q[:self.I], kf[:self.I], kr[:self.I]
        return wdot, hrr[0]

    def rhs(self, p: float, z: np.ndarray) -> np.ndarray:
        z = np.ascontiguousarray(z, dtype=np.float64)
        f = np.zeros(self.n)
        self.lib.or_rhs(self.h, float(p), z, f)
        return f

    def jacobian(self, p: float, z: np.ndarray) -> np.ndarray:
        z = np.ascontiguousarray(z, dtype=np.float64)
        J = np.zeros(self.n * self.n)
        self.lib.or_jacobian(self.h, float(p), z, J)
        return J.reshape(self.n, self.n)

    # -- integration
    def integrate(self, p: float, z: np.ndarray, dt: float, rtol=ORACLE_RTOL, atol_Y=ORACLE_ATOL_Y,
                  atol_T=ORACLE_ATOL_T, max_steps=200000):
        """z(t+dt) of Eq. 2 by the Radau IIA integrator; returns (z_new, status, stats[6]):
        accepted steps, RHS evaluations, Jacobian evaluations, LU factorisations, error-test
        rejections, Newton failures."""
        z = np.array(z, dtype=np.float64)
        st = np.zeros(6, dtype=np.int32)
        s = self.lib.or_integrate(self.h, float(p), z, float(dt), rtol, atol_Y, atol_T,
                                  int(max_steps), st)
        return z, s, st

    def integrate_batch(self, T: np.ndarray, p: np.ndarray, Y: np.ndarray, dt: float,
                        rtol=ORACLE_RTOL, atol_Y=ORACLE_ATOL_Y, atol_T=ORACLE_ATOL_T,
                        max_steps=200000, nthreads: int = 0):
        """Batched Eq. 2 over cells (OpenMP); Y is [K, N] species-major.  Returns copies."""
        T = np.array(T, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
        Y = np.array(Y, dtype=np.float64, order="C")
        n = T.size
        status = np.zeros(n, dtype=np.int32)
        steps = np.zeros(n, dtype=np.int32)
        self.lib.or_integrate_batch(self.h, n, n, float(dt), T, p, Y, rtol, atol_Y, atol_T,
                                    int(max_steps), status, steps, int(nthreads))
        return T, Y, status, steps

    def radau_fixed(self, p: float, z: np.ndarray, h: float, nsteps: int) -> np.ndarray:
        """nsteps Radau IIA steps of fixed length h (no error control; for order checks)."""
        z = np.array(z, dtype=np.float64)
        if self.lib.or_radau_fixed(self.h, float(p), z, float(h), int(nsteps)) != 0:
            raise FloatingPointError("Radau IIA Newton iteration failed")
        return z

    @staticmethod
    def radau_tableau():
        """(A [3, 3], c [3]) of the three-stage Radau IIA method the integrator uses."""
        A, c = np.zeros(9), np.zeros(3)
        _load().or_radau_tableau(A, c)
        return A.reshape(3, 3), c

    def rk4(self, p: float, z: np.ndarray, dt: float, nsub: int) -> np.ndarray:
        z = np.array(z, dtype=np.float64)
        s = self.lib.or_rk4(self.h, float(p), z, float(dt), int(nsub))
        if s != 0:
            raise FloatingPointError("rk4 produced non-finite values")
        return z

    # -- properties
    def thermo_props(self, T: float, Y: np.ndarray):
        """(cp J/kg/K, h J/kg, mu Pa s, kappa W/m/K) of the mixture."""
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        out = np.zeros(4)
        self.lib.or_thermo_props(self.h, float(T), Y, _ptr(out[0:1]), _ptr(out[1:2]),
                                 _ptr(out[2:3]), _ptr(out[3:4]))
        return tuple(out)

    def T_from_h(self, h: float, Y: np.ndarray, T0: float = 1000.0) -> float:
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        T = C.c_double()
        self.lib.or_T_from_h(self.h, float(h), Y, float(T0), C.byref(T))
        return T.value

    @staticmethod
    def dense_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
        """x with A x = b by the oracle's own LU with partial pivoting."""
        A = np.array(A, dtype=np.float64, order="C")
        x = np.array(b, dtype=np.float64)
        if _load().or_dense_solve(A.shape[0], A, x) != 0:
            raise np.linalg.LinAlgError("singular matrix")
        return x

    @staticmethod
    def max_threads() -> int:
        return int(_load().or_max_threads())
