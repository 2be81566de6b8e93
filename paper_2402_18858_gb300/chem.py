"""Thin Python binding of libchem (ctypes): argument marshalling only.

Every function has the name of the C entry point it wraps (include/chem.h) and takes torch
CUDA tensors; all arithmetic runs in the library's kernels.  There is no fallback: if the
shared library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import torch

from . import build as _build

_lib = None
_lock = threading.Lock()


class ChemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libchem error {code}: {msg}")
        self.code = code


class HfrdOpts(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("theta", C.c_double), ("hc", C.c_double * 2),
                ("on", C.c_double * 2), ("phi", C.c_double * 2)]


class DiOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol_Y", C.c_double), ("atol_T", C.c_double),
                ("newton_tol", C.c_double), ("max_steps", C.c_int), ("jac_max_age", C.c_int)]


def lib(auto_build: bool = False):
    """The loaded libchem.so (built in-tree by `build.build()`)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not auto_build:
                raise RuntimeError(f"libchem is not built ({path} missing): run build() first")
            _build.build()
        L = C.CDLL(path)
        vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
        L.chem_load_mech.argtypes = [C.c_char_p, C.POINTER(vp)]
        L.chem_free_mech.argtypes = [vp]
        L.chem_free_mech.restype = None
        L.chem_mech_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.chem_rates.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp]
        L.chem_jacobian.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp]
        L.chem_step_di.argtypes = [vp, i64, i64, dbl, vp, vp, vp, vp, C.POINTER(DiOpts), vp, vp,
                                   vp, C.c_size_t, vp]
        L.chem_step_di_noalloc.argtypes = [vp, i64, i64, dbl, vp, vp, vp, vp, C.POINTER(DiOpts),
                                           vp, vp, vp]
        L.chem_workspace_bytes.argtypes = [vp, i64]
        L.chem_workspace_bytes.restype = C.c_size_t
        L.thermo_props.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp]
        L.chem_pasr_source.argtypes = [vp, i64, i64, dbl, vp, vp, vp, vp, vp, vp, dbl, dbl, vp, vp, vp]
        L.chem_hfrd_augment.argtypes = [vp, i64, i64, vp, vp, vp, vp, C.POINTER(HfrdOpts), vp, vp, vp, vp, vp,
                                        C.c_size_t, vp]
        L.chem_hfrd_workspace_bytes.restype = C.c_size_t
        L.chem_hfrd_workspace_bytes.argtypes = []
        L.chem_last_error.restype = C.c_char_p
        L.chem_fp64_peak_gflops.argtypes = [C.POINTER(dbl), vp]
        L.chem_selftest_exp.argtypes = [vp, i64, vp, vp, vp]
        L.chem_selftest_log.argtypes = [vp, i64, vp, vp, vp]
        L.chem_selftest_exp256.argtypes = [vp, i64, vp, vp, vp]
        L.chem_selftest_rcp.argtypes = [i64, vp, vp, vp]
        L.chem_selftest_gemm.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]
        L.chem_selftest_gemm_grouped.argtypes = [i32, i32, i32, i32, i32, vp, i64, i32, i32, vp, i64, i32, i32,
                                                 vp, i32, vp, i64, i64, vp, i64, i64, vp, vp]
        _lib = L
        return L


def _check(rc: int) -> None:
    if rc != 0:
        raise ChemError(rc, lib().chem_last_error().decode(errors="replace"))


def _ptr(t: Optional[torch.Tensor], dtype=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libchem takes CUDA tensors")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("libchem takes contiguous tensors")
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Mech:
    """A mechanism loaded on the current device (owns a chem_mech handle)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)
        K, I, E = C.c_int(), C.c_int(), C.c_int()
        _check(lib().chem_mech_info(self.handle, C.byref(K), C.byref(I), C.byref(E)))
        self.K, self.I, self.E = K.value, I.value, E.value
        self.n = self.K + 1

    def __del__(self):
        try:
            if self.handle:
                lib().chem_free_mech(self.handle)
                self.handle = None
        except Exception:
            pass


def chem_load_mech(path: str) -> Mech:
    h = C.c_void_p()
    _check(lib().chem_load_mech(path.encode(), C.byref(h)))
    return Mech(h.value)


def _ld(Y: torch.Tensor, m: Mech) -> int:
    if Y.dim() != 2 or Y.shape[0] != m.K:
        raise ValueError(f"Y must be [K={m.K}, ld]")
    return Y.shape[1]


def chem_rates(m: Mech, T, p, Y, wdot, hrr=None, n: Optional[int] = None, stream=None) -> None:
    ld = _ld(Y, m)
    n = ld if n is None else n
    _check(lib().chem_rates(m.handle, n, ld, _ptr(T, torch.float64), _ptr(p, torch.float64),
                            _ptr(Y, torch.float64), _ptr(wdot, torch.float64),
                            _ptr(hrr, torch.float64), _stream(stream)))


def chem_jacobian(m: Mech, T, p, Y, jac, n: Optional[int] = None, stream=None) -> None:
    ld = _ld(Y, m)
    n = ld if n is None else n
    _check(lib().chem_jacobian(m.handle, n, ld, _ptr(T, torch.float64), _ptr(p, torch.float64),
                               _ptr(Y, torch.float64), _ptr(jac, torch.float64), _stream(stream)))


def chem_workspace_bytes(m: Mech, n: int) -> int:
    return int(lib().chem_workspace_bytes(m.handle, n))


def chem_step_di(m: Mech, dt: float, T, p, Y, status, idx=None, rtol=0.0, atol_Y=0.0, atol_T=0.0,
                 max_steps=0, stats=None, workspace=None, n: Optional[int] = None,
                 stream=None, newton_tol=0.0, jac_max_age=0) -> None:
    ld = _ld(Y, m)
    if n is None:
        n = idx.numel() if idx is not None else ld
    if workspace is None:
        raise ValueError("chem_step_di needs a workspace tensor (chem_workspace_bytes)")
    o = DiOpts(rtol, atol_Y, atol_T, newton_tol, max_steps, jac_max_age)
    _check(lib().chem_step_di(m.handle, n, ld, float(dt), _ptr(T, torch.float64),
                              _ptr(p, torch.float64), _ptr(Y, torch.float64),
                              _ptr(idx, torch.int32), C.byref(o), _ptr(status, torch.int32),
                              _ptr(stats, torch.int32), _ptr(workspace),
                              workspace.numel() * workspace.element_size(), _stream(stream)))


def chem_step_di_noalloc(m: Mech, dt: float, T, p, Y, status, idx=None, rtol=0.0, atol_Y=0.0,
                         atol_T=0.0, max_steps=0, stats=None, n: Optional[int] = None,
                         stream=None, newton_tol=0.0, jac_max_age=0) -> None:
    """chem_step_di without a workspace, for callers that cannot allocate device memory.

    Its scratch is a fixed device array inside the library shared by every call: calls that
    overlap on the GPU race on it.
    """
    ld = _ld(Y, m)
    if n is None:
        n = idx.numel() if idx is not None else ld
    o = DiOpts(rtol, atol_Y, atol_T, newton_tol, max_steps, jac_max_age)
    _check(lib().chem_step_di_noalloc(m.handle, n, ld, float(dt), _ptr(T, torch.float64),
                                      _ptr(p, torch.float64), _ptr(Y, torch.float64),
                                      _ptr(idx, torch.int32), C.byref(o),
                                      _ptr(status, torch.int32), _ptr(stats, torch.int32),
                                      _stream(stream)))


def thermo_props(m: Mech, T, Y, cp=None, h=None, mu=None, kappa=None, h_in=None, T_out=None,
                 mixed_precision: bool = False, n: Optional[int] = None, stream=None) -> None:
    ld = _ld(Y, m)
    n = ld if n is None else n
    f64 = torch.float64
    _check(lib().thermo_props(m.handle, n, ld, _ptr(T, f64), _ptr(Y, f64), _ptr(cp, f64),
                              _ptr(h, f64), _ptr(mu, f64), _ptr(kappa, f64), _ptr(h_in, f64),
                              _ptr(T_out, f64), int(bool(mixed_precision)), _stream(stream)))


def chem_pasr_source(m: Mech, dt: float, rho, Y0, Y1, k_sgs, eps, nu, omega, kappa=None,
                     y_min: float = -1.0, r_min: float = -1.0, n: Optional[int] = None, stream=None) -> None:
    ld = _ld(Y0, m)
    if _ld(Y1, m) != ld or _ld(omega, m) != ld:
        raise ValueError("Y0, Y1 and omega must share the species-major layout")
    n = ld if n is None else n
    f64 = torch.float64
    _check(lib().chem_pasr_source(m.handle, n, ld, float(dt), _ptr(rho, f64), _ptr(Y0, f64), _ptr(Y1, f64),
                                  _ptr(k_sgs, f64), _ptr(eps, f64), _ptr(nu, f64), float(y_min), float(r_min),
                                  _ptr(omega, f64), _ptr(kappa, f64), _stream(stream)))


def chem_hfrd_workspace_bytes() -> int:
    return int(lib().chem_hfrd_workspace_bytes())


def chem_hfrd_augment(m: Mech, T, p, Y, gamma, T_out, p_out, Y_out, keep, workspace, opts: Optional[dict] = None,
                      n: Optional[int] = None, stream=None) -> None:
    """HFRD augmentation (Eqs. 3-6); opts: dict with alpha, beta, theta, hc, on, phi, or None."""
    ld = _ld(Y, m)
    if gamma.dim() != 2 or gamma.shape[0] != 3 + m.K or gamma.shape[1] != ld:
        raise ValueError(f"gamma must be [3 + K = {3 + m.K}, ld = {ld}]")
    n = ld if n is None else n
    o = None
    if opts is not None:
        o = HfrdOpts(opts["alpha"], opts["beta"], opts["theta"], (C.c_double * 2)(*opts["hc"]),
                     (C.c_double * 2)(*opts["on"]), (C.c_double * 2)(*opts["phi"]))
    f64 = torch.float64
    _check(lib().chem_hfrd_augment(m.handle, n, ld, _ptr(T, f64), _ptr(p, f64), _ptr(Y, f64), _ptr(gamma, f64),
                                   C.byref(o) if o is not None else None, _ptr(T_out, f64), _ptr(p_out, f64),
                                   _ptr(Y_out, f64), _ptr(keep, torch.int32), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream)))


def chem_fp64_peak_gflops(stream=None) -> float:
    v = C.c_double()
    _check(lib().chem_fp64_peak_gflops(C.byref(v), _stream(stream)))
    return v.value


def chem_selftest_exp(m: Mech, x, y, stream=None) -> None:
    _check(lib().chem_selftest_exp(m.handle, x.numel(), _ptr(x, torch.float64),
                                   _ptr(y, torch.float64), _stream(stream)))


def chem_selftest_exp256(m: Mech, x, y, stream=None) -> None:
    _check(lib().chem_selftest_exp256(m.handle, x.numel(), _ptr(x, torch.float64),
                                      _ptr(y, torch.float64), _stream(stream)))


def chem_selftest_log(m: Mech, x, y, stream=None) -> None:
    _check(lib().chem_selftest_log(m.handle, x.numel(), _ptr(x, torch.float64),
                                   _ptr(y, torch.float64), _stream(stream)))


def chem_selftest_rcp(x, y, stream=None) -> None:
    _check(lib().chem_selftest_rcp(x.numel(), _ptr(x, torch.float64), _ptr(y, torch.float64), _stream(stream)))


def chem_selftest_gemm(epi: int, A, B, out, bias=None, z=None, err=None, stream=None) -> None:
    """out = epilogue(A @ B^T) on the tensor cores (A [M,K], B [N,K] BF16; see include/chem.h)."""
    M, K = A.shape
    N = B.shape[0]
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().chem_selftest_gemm(int(epi), M, N, K, _ptr(A, torch.bfloat16), _ptr(B, torch.bfloat16),
                                    _ptr(bias, torch.float32), _ptr(z, torch.bfloat16), _ptr(out),
                                    _ptr(err, torch.int32), _stream(stream)))
    return err


def chem_selftest_gemm_grouped(epi: int, G: int, M: int, N: int, K: int, A, a_off, B, b_off, out, ldo: int,
                               out_goff: int, bias=None, bias_goff: int = 0, z=None, ldz: int = 0,
                               z_goff: int = 0, err=None, stream=None) -> None:
    """G GEMMs in one launch (see include/chem.h); a_off = (a_row, a_col), b_off = (b_row, b_col)."""
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().chem_selftest_gemm_grouped(int(epi), int(G), int(M), int(N), int(K), _ptr(A, torch.bfloat16),
                                            A.stride(0), int(a_off[0]), int(a_off[1]), _ptr(B, torch.bfloat16),
                                            B.stride(0), int(b_off[0]), int(b_off[1]), _ptr(bias, torch.float32),
                                            int(bias_goff), _ptr(z, torch.bfloat16), int(ldz), int(z_goff),
                                            _ptr(out), int(ldo), int(out_goff), _ptr(err, torch.int32),
                                            _stream(stream)))
    return err


# ------------------------------------------------------------------------------------------
# learned reaction step
# ------------------------------------------------------------------------------------------
class TrainOpts(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("w_data", C.c_float), ("w_mass", C.c_float), ("apply", C.c_int), ("w_hrr", C.c_float)]


class AnnOpts(C.Structure):
    _fields_ = [("range_margin", C.c_double), ("elem_tol", C.c_double), ("T_min", C.c_double),
                ("T_max", C.c_double), ("dT_max", C.c_double), ("no_fallback", C.c_int),
                ("reserved", C.c_int), ("di", DiOpts)]


class TrainEpochOpts(C.Structure):
    _fields_ = [("step", TrainOpts), ("batch", C.c_int64), ("lr_min", C.c_float), ("total_steps", C.c_int64),
                ("step0", C.c_int64), ("seed", C.c_uint64), ("epoch", C.c_int), ("reserved", C.c_int)]


_ann_sigs_done = False


def _ann_sigs():
    global _ann_sigs_done
    if _ann_sigs_done:
        return
    L = lib()
    vp, i64, i32, fp = C.c_void_p, C.c_int64, C.c_int, C.POINTER(C.c_float)
    L.chem_ann_create.argtypes = [vp, C.POINTER(i32), i32, C.c_uint64, C.POINTER(vp)]
    L.chem_ann_create_per_species.argtypes = [vp, C.POINTER(i32), i32, C.c_uint64, C.POINTER(vp)]
    L.chem_ann_layout.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    L.chem_ann_free.argtypes = [vp]
    L.chem_ann_free.restype = None
    L.chem_ann_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                C.POINTER(i64)]
    L.chem_ann_set_norm.argtypes = [vp, fp]
    L.chem_ann_get_norm.argtypes = [vp, fp]
    L.chem_ann_fit_norm.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp]
    L.chem_ann_features.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, C.c_double, vp, vp]
    L.chem_ann_update.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, C.POINTER(AnnOpts), vp, vp, vp]
    L.chem_ann_targets.argtypes = [vp, i64, i64, vp, vp, vp, vp]
    L.chem_ann_forward.argtypes = [vp, vp, i64, vp, vp, C.c_size_t, vp]
    L.chem_ann_train_step.argtypes = [vp, vp, vp, vp, vp, vp, i64, C.POINTER(TrainOpts), vp, vp]
    L.chem_ann_train_epoch.argtypes = [vp, vp, vp, vp, vp, vp, i64, C.POINTER(TrainEpochOpts), vp, vp]
    L.chem_selftest_epoch_order.argtypes = [i64, C.c_uint64, i32, vp, vp]
    L.chem_ann_hrr_coeffs.argtypes = [vp, i64, i64, vp, vp, vp, vp, C.c_double, C.c_double, vp, vp, vp]
    L.chem_ann_get_params.argtypes = [vp, i32, fp, i64]
    L.chem_ann_set_params.argtypes = [vp, fp, i64]
    L.chem_ann_save.argtypes = [vp, C.c_char_p, i32]
    L.chem_ann_load.argtypes = [vp, C.c_char_p, C.POINTER(vp)]
    L.chem_ann_error.argtypes = [vp, C.POINTER(i32)]
    L.chem_step_ann.argtypes = [vp, vp, i64, i64, C.c_double, vp, vp, vp, vp, C.POINTER(AnnOpts), vp,
                                vp, C.c_size_t, vp]
    L.chem_ann_workspace_bytes.argtypes = [vp, i64]
    L.chem_ann_workspace_bytes.restype = C.c_size_t
    _ann_sigs_done = True


class Ann:
    """An MLP of the learned reaction step (owns a chem_ann handle)."""

    def __init__(self, handle: int, mech: Mech):
        _ann_sigs()
        self.handle = C.c_void_p(handle)
        self.mech = mech
        n_in, n_out, nl = C.c_int(), C.c_int(), C.c_int()
        dims = (C.c_int * 9)()
        npar = C.c_int64()
        _check(lib().chem_ann_info(self.handle, C.byref(n_in), C.byref(n_out), C.byref(nl), dims,
                                   C.byref(npar)))
        self.n_in, self.n_out, self.L = n_in.value, n_out.value, nl.value
        self.dims = [dims[i] for i in range(self.L + 1)]
        groups, n_out_pad = C.c_int(), C.c_int()
        _check(lib().chem_ann_layout(self.handle, C.byref(groups), C.byref(n_out_pad)))
        self.groups = groups.value          # 1: one network; K: one network per species
        self.n_out_pad = n_out_pad.value
        self.n_params = npar.value
        self.norm_size = 4 * self.n_in + 2 * self.n_out

    def __del__(self):
        try:
            if self.handle:
                lib().chem_ann_free(self.handle)
                self.handle = None
        except Exception:
            pass


def chem_ann_create(m: Mech, hidden, seed: int = 0) -> Ann:
    _ann_sigs()
    h = C.c_void_p()
    arr = (C.c_int * len(hidden))(*hidden)
    _check(lib().chem_ann_create(m.handle, arr, len(hidden), int(seed), C.byref(h)))
    return Ann(h.value, m)


def chem_ann_create_per_species(m: Mech, hidden, seed: int = 0) -> Ann:
    """One network of the given hidden widths per species (output width 1 each)."""
    _ann_sigs()
    h = C.c_void_p()
    arr = (C.c_int * len(hidden))(*hidden)
    _check(lib().chem_ann_create_per_species(m.handle, arr, len(hidden), int(seed), C.byref(h)))
    return Ann(h.value, m)


def chem_ann_load(m: Mech, path: str) -> Ann:
    _ann_sigs()
    h = C.c_void_p()
    _check(lib().chem_ann_load(m.handle, path.encode(), C.byref(h)))
    return Ann(h.value, m)


def chem_ann_save(a: Ann, path: str, with_moments: bool = True) -> None:
    _check(lib().chem_ann_save(a.handle, path.encode(), int(bool(with_moments))))


def _fptr(arr):
    return arr.ctypes.data_as(C.POINTER(C.c_float))


def chem_ann_get_norm(a: Ann):
    import numpy as np
    out = np.zeros(a.norm_size, dtype=np.float32)
    _check(lib().chem_ann_get_norm(a.handle, _fptr(out)))
    return out


def chem_ann_set_norm(a: Ann, norm) -> None:
    import numpy as np
    arr = np.ascontiguousarray(norm, dtype=np.float32)
    _check(lib().chem_ann_set_norm(a.handle, _fptr(arr)))


def chem_ann_fit_norm(a: Ann, T, p, Y0, Y1, n: Optional[int] = None, stream=None) -> None:
    ld = Y0.shape[1]
    n = ld if n is None else n
    f64 = torch.float64
    _check(lib().chem_ann_fit_norm(a.handle, n, ld, _ptr(T, f64), _ptr(p, f64), _ptr(Y0, f64),
                                   _ptr(Y1, f64), _stream(stream)))


def chem_ann_features(a: Ann, T, p, Y, X, bcty=None, n: Optional[int] = None, stream=None,
                      flags=None, range_margin=0.05) -> None:
    """Features X [n, 64] BF16; optionally raw F(Y) (bcty) and the range flags (int32 [n])."""
    ld = Y.shape[1]
    n = ld if n is None else n
    f64 = torch.float64
    _check(lib().chem_ann_features(a.handle, n, ld, _ptr(T, f64), _ptr(p, f64), _ptr(Y, f64),
                                   _ptr(X, torch.bfloat16), _ptr(bcty, torch.float32), float(range_margin),
                                   _ptr(flags, torch.int32), _stream(stream)))


def chem_ann_update(a: Ann, T, p, Y, U, flags, status, idx=None, elem_tol=1e-2, T_min=250.0, T_max=3500.0,
                    dT_max=0.0, n: Optional[int] = None, stream=None) -> None:
    """The learned step's update on given network outputs U; flags in (range bit) / out."""
    ld = _ld(Y, a.mech)
    if n is None:
        n = idx.numel() if idx is not None else ld
    o = AnnOpts(0.0, elem_tol, T_min, T_max, dT_max, 1, 0, DiOpts(0.0, 0.0, 0.0, 0.0, 0, 0))
    _check(lib().chem_ann_update(a.handle, n, ld, _ptr(T, torch.float64), _ptr(p, torch.float64),
                                 _ptr(Y, torch.float64), _ptr(U, torch.float32), _ptr(idx, torch.int32),
                                 C.byref(o), _ptr(flags, torch.int32), _ptr(status, torch.int32),
                                 _stream(stream)))


def chem_ann_targets(a: Ann, Y0, Y1, U, n: Optional[int] = None, stream=None) -> None:
    ld = Y0.shape[1]
    n = ld if n is None else n
    _check(lib().chem_ann_targets(a.handle, n, ld, _ptr(Y0, torch.float64), _ptr(Y1, torch.float64),
                                  _ptr(U, torch.float32), _stream(stream)))


def chem_ann_workspace_bytes(a: Ann, n: int) -> int:
    _ann_sigs()
    return int(lib().chem_ann_workspace_bytes(a.handle, n))


def chem_ann_forward(a: Ann, X, U, workspace, stream=None) -> None:
    _check(lib().chem_ann_forward(a.handle, _ptr(X, torch.bfloat16), X.shape[0], _ptr(U, torch.float32),
                                  _ptr(workspace), workspace.numel() * workspace.element_size(),
                                  _stream(stream)))


def chem_ann_train_step(a: Ann, X, Ut, bcty=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                        w_data=1.0, w_mass=0.1, apply=True, loss_out=None, hrr_c=None, hrr_r=None,
                        w_hrr=0.0, stream=None) -> None:
    """One Adam step; loss_out (4 floats, device) receives L_tot, L_data, L_mass, L_HRR."""
    if loss_out is not None and loss_out.numel() < 4:
        raise ValueError("loss_out needs 4 floats")
    if w_hrr != 0.0 and (hrr_c is None or hrr_r is None or bcty is None):
        raise ValueError("w_hrr != 0 needs bcty, hrr_c and hrr_r")
    o = TrainOpts(lr, beta1, beta2, eps, w_data, w_mass if bcty is not None else 0.0, int(apply), float(w_hrr))
    _check(lib().chem_ann_train_step(a.handle, _ptr(X, torch.bfloat16), _ptr(Ut, torch.float32),
                                     _ptr(bcty, torch.float32), _ptr(hrr_c, torch.float32),
                                     _ptr(hrr_r, torch.float32), X.shape[0], C.byref(o),
                                     _ptr(loss_out, torch.float32), _stream(stream)))


def chem_ann_train_epoch(a: Ann, X, Ut, bcty=None, batch=8192, lr=1e-3, lr_min=2e-5, total_steps=0, step0=0,
                         seed=0, epoch=0, beta1=0.9, beta2=0.999, eps=1e-8, w_data=1.0, w_mass=0.1,
                         hrr_c=None, hrr_r=None, w_hrr=0.0, loss_out=None, n: Optional[int] = None,
                         stream=None) -> None:
    """One epoch in a seeded minibatch order with the cosine schedule; loss_out gets the epoch means."""
    if loss_out is not None and loss_out.numel() < 4:
        raise ValueError("loss_out needs 4 floats")
    n = X.shape[0] if n is None else n
    step = TrainOpts(lr, beta1, beta2, eps, w_data, w_mass if bcty is not None else 0.0, 1, float(w_hrr))
    o = TrainEpochOpts(step, int(batch), float(lr_min), int(total_steps), int(step0), int(seed), int(epoch), 0)
    _check(lib().chem_ann_train_epoch(a.handle, _ptr(X, torch.bfloat16), _ptr(Ut, torch.float32),
                                      _ptr(bcty, torch.float32), _ptr(hrr_c, torch.float32),
                                      _ptr(hrr_r, torch.float32), int(n), C.byref(o),
                                      _ptr(loss_out, torch.float32), _stream(stream)))


def chem_selftest_epoch_order(n: int, seed: int, epoch: int, order, stream=None) -> None:
    _ann_sigs()
    _check(lib().chem_selftest_epoch_order(int(n), int(seed), int(epoch), _ptr(order, torch.int32),
                                           _stream(stream)))


def chem_ann_hrr_coeffs(a: Ann, dt: float, scale: float, T0, p, Y0, Y1, hrr_c, hrr_r, n: Optional[int] = None,
                        stream=None) -> None:
    """Per-sample heat-release coefficients [n, K] and DI targets [n] of the L_HRR term."""
    ld = Y0.shape[1]
    n = ld if n is None else n
    f64 = torch.float64
    _check(lib().chem_ann_hrr_coeffs(a.handle, n, ld, _ptr(T0, f64), _ptr(p, f64), _ptr(Y0, f64), _ptr(Y1, f64),
                                     float(dt), float(scale), _ptr(hrr_c, torch.float32), _ptr(hrr_r, torch.float32),
                                     _stream(stream)))


def chem_ann_get_params(a: Ann, which: int = 0):
    import numpy as np
    out = np.zeros(a.n_params, dtype=np.float32)
    _check(lib().chem_ann_get_params(a.handle, int(which), _fptr(out), a.n_params))
    return out


def chem_ann_set_params(a: Ann, flat) -> None:
    import numpy as np
    arr = np.ascontiguousarray(flat, dtype=np.float32)
    _check(lib().chem_ann_set_params(a.handle, _fptr(arr), arr.size))


def chem_ann_error(a: Ann) -> int:
    v = C.c_int()
    _check(lib().chem_ann_error(a.handle, C.byref(v)))
    return v.value


def chem_step_ann(m: Mech, a: Ann, dt: float, T, p, Y, status, workspace, idx=None, range_margin=0.05,
                  elem_tol=1e-2, T_min=250.0, T_max=3500.0, dT_max=0.0, no_fallback=False,
                  di_rtol=0.0, di_atol_Y=0.0, n: Optional[int] = None, stream=None,
                  di_newton_tol=0.0, di_jac_max_age=0) -> None:
    ld = _ld(Y, m)
    if n is None:
        n = idx.numel() if idx is not None else ld
    o = AnnOpts(range_margin, elem_tol, T_min, T_max, dT_max, int(no_fallback), 0,
                DiOpts(di_rtol, di_atol_Y, 0.0, di_newton_tol, 0, di_jac_max_age))
    _check(lib().chem_step_ann(m.handle, a.handle, n, ld, float(dt), _ptr(T, torch.float64),
                               _ptr(p, torch.float64), _ptr(Y, torch.float64), _ptr(idx, torch.int32),
                               C.byref(o),
                               _ptr(status, torch.int32), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _stream(stream)))


# ------------------------------------------------------------------------------------------
# serving loop
# ------------------------------------------------------------------------------------------
class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("n_streams", C.c_int), ("max_batch_cells", C.c_int),
                ("starvation_s", C.c_double), ("di_chunk_cells", C.c_int), ("reserved", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("cells", C.c_int64), ("batches", C.c_int64), ("mean_batch_requests", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("max_ms", C.c_double), ("wall_s", C.c_double), ("cells_per_s", C.c_double),
                ("hbm_bytes", C.c_double)]


_srv_sigs_done = False


def _srv_sigs():
    global _srv_sigs_done
    if _srv_sigs_done:
        return
    L = lib()
    vp = C.c_void_p
    L.chem_server_create.argtypes = [C.POINTER(ServerOpts), C.POINTER(vp)]
    L.chem_server_add_class.argtypes = [vp, vp, vp, C.c_int64, C.POINTER(C.c_int)]
    L.chem_server_submit.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_int64, vp, vp, vp, vp, vp, vp,
                                     C.POINTER(C.c_int64)]
    L.chem_server_wait.argtypes = [vp, C.c_int64, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.chem_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
    L.chem_server_request_latency.argtypes = [vp, C.c_int64, C.POINTER(C.c_double)]
    L.chem_server_free.argtypes = [vp]
    L.chem_server_free.restype = None
    _srv_sigs_done = True


class Server:
    """A chemistry-step server (owns a chem_server handle and keeps its host buffers alive)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)
        self.keep = {}
        self.classes = []

    def __del__(self):
        try:
            if self.handle:
                lib().chem_server_free(self.handle)
                self.handle = None
        except Exception:
            pass


def chem_server_create(hbm_budget_bytes: int, n_streams: int = 2, max_batch_cells: int = 1 << 21,
                       starvation_s: float = 0.0, di_chunk_cells: int = 0) -> Server:
    _srv_sigs()
    o = ServerOpts(int(hbm_budget_bytes), int(n_streams), int(max_batch_cells), float(starvation_s),
                   int(di_chunk_cells), 0)
    h = C.c_void_p()
    _check(lib().chem_server_create(C.byref(o), C.byref(h)))
    return Server(h.value)


def chem_server_add_class(sv: Server, m: Mech, ann=None, capacity_cells: int = 1 << 20) -> int:
    cid = C.c_int()
    _check(lib().chem_server_add_class(sv.handle, m.handle, ann.handle if ann is not None else None,
                                       int(capacity_cells), C.byref(cid)))
    sv.classes.append((m, ann))
    return cid.value


def chem_server_submit(sv: Server, class_id: int, mode: int, dt: float, T, p, Y, T_out, Y_out, status_out) -> int:
    """Host numpy/torch-CPU arrays (contiguous, float64 / int32); kept alive by the server."""
    import numpy as np
    arrs = [np.ascontiguousarray(a) for a in (T, p, Y)]
    for a in (T_out, Y_out, status_out):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("output arrays must be contiguous")
    rid = C.c_int64()
    n = arrs[0].shape[0]
    _check(lib().chem_server_submit(sv.handle, int(class_id), int(mode), float(dt), n,
                                    *[a.ctypes.data_as(C.c_void_p) for a in arrs],
                                    T_out.ctypes.data_as(C.c_void_p), Y_out.ctypes.data_as(C.c_void_p),
                                    status_out.ctypes.data_as(C.c_void_p), C.byref(rid)))
    sv.keep[rid.value] = (arrs, T_out, Y_out, status_out)
    return rid.value


def chem_server_wait(sv: Server, request_id: int, timeout_s: float = 60.0):
    done, res = C.c_int(), C.c_int()
    _check(lib().chem_server_wait(sv.handle, int(request_id), float(timeout_s), C.byref(done), C.byref(res)))
    return bool(done.value), res.value


def chem_server_request_latency(sv: Server, request_id: int) -> float:
    """Submit-to-results latency of a completed request in ms (-1 while it runs)."""
    v = C.c_double()
    _check(lib().chem_server_request_latency(sv.handle, int(request_id), C.byref(v)))
    return v.value


def chem_server_stats(sv: Server) -> dict:
    st = ServerStats()
    _check(lib().chem_server_get_stats(sv.handle, C.byref(st)))
    return {f: getattr(st, f) for f, _ in ServerStats._fields_}
