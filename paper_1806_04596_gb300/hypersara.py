"""Thin ctypes binding of libhypersara.so (include/hypersara.h).

Argument marshalling only: every operation runs in the library's CUDA
kernels. Tensors are torch tensors on the CUDA device, contiguous, of the
plan's precision (FP32 plan: float32 / complex64, FP64 plan: float64 /
complex128). Calls are asynchronous on torch's current CUDA stream unless the
C function documents a synchronisation. There is no CPU fallback: if the
library is missing or fails to load, every call raises.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhypersara.so")

HS_OK, HS_ERR_ARG, HS_ERR_CUDA, HS_ERR_NOMEM, HS_ERR_TIMEOUT, HS_ERR_STATE = 0, -1, -2, -3, -4, -5
HS_F32, HS_F64 = 0, 1
HS_PLAN_COMPENSATED = 1
HS_PLAN_GRAM_FMA = 2
HS_PLAN_NO_TUNE = 4
HS_PLAN_FFT_CHUNKED = 8
STAGES = {"fft_fwd": 0, "degrid": 1, "grid": 2, "fft_adj": 3, "psi_fwd": 4, "psi_adj": 5}

_lib = None


class HSError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed with status {status}: {msg}")
        self.status = status


class PlanInfo(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("L", C.c_int), ("Kx", C.c_int), ("Ky", C.c_int),
                ("levels", C.c_int), ("prec", C.c_int), ("flags", C.c_int),
                ("total_vis", C.c_int64), ("grid_tile_entries", C.c_int64),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("kb_terms", C.c_int),
                ("kb_beta", C.c_double), ("kb_fit_max_err", C.c_double),
                ("device_bytes", C.c_int64), ("nblocks", C.c_int),
                ("gram_tc", C.c_int), ("sweep_hmax", C.c_int), ("sweep_cap", C.c_int), ("tuned", C.c_int),
                ("tune_ms", C.c_double), ("tune_grid_ms", C.c_double * 3), ("tune_gram_ms", C.c_double * 2),
                ("fft_adj_chunk", C.c_int), ("tune_fft_ms", C.c_double * 2)]


class AdaptParams(C.Structure):
    _fields_ = [("enable", C.c_int), ("lambda1", C.c_double), ("lambda2", C.c_double),
                ("lambda3", C.c_double), ("min_gap", C.c_int64)]


class PDParams(C.Structure):
    _fields_ = [("tau", C.c_double), ("kappa1", C.c_double), ("kappa2", C.c_double),
                ("kappa3", C.c_double), ("mu", C.c_double), ("psi_norm2", C.c_double),
                ("use_nuclear", C.c_int), ("use_l21", C.c_int),
                ("w_nuc", C.c_void_p), ("w_l21", C.c_void_p), ("sparsity", C.c_int)]


_P = C.c_void_p
_SIGS = {
    "hs_version": ([], C.c_char_p),
    "hs_last_error": ([], C.c_char_p),
    "hs_plan_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int64), _P, _P,
                        _P, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_uint, _P], C.c_int),
    "hs_plan_create_blocks": ([C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int64), C.c_int,
                               C.POINTER(C.c_int64), _P, _P, _P, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                               C.c_uint, _P], C.c_int),
    "hs_pd_set_adaptive": ([_P, C.POINTER(AdaptParams)], C.c_int),
    "hs_pd_bounds": ([_P, _P, _P, _P, _P], C.c_int),
    "hs_plan_destroy": ([_P], C.c_int),
    "hs_plan_info": ([_P, C.POINTER(PlanInfo)], C.c_int),
    "hs_plan_check": ([_P, _P], C.c_int),
    "hs_set_device_limit": ([C.c_int64], C.c_int),
    "hs_device_bytes": ([C.POINTER(C.c_int64)], C.c_int),
    "hs_phi_fwd": ([_P, _P, _P, _P], C.c_int),
    "hs_phi_adj": ([_P, _P, _P, _P], C.c_int),
    "hs_psi_fwd": ([_P, _P, _P, _P], C.c_int),
    "hs_psi_adj": ([_P, _P, _P, _P], C.c_int),
    "hs_prox_l21": ([_P, _P, _P, C.c_double, C.c_int, _P, _P], C.c_int),
    "hs_prox_nuclear": ([_P, _P, _P, C.c_double, C.c_int, _P, _P, _P], C.c_int),
    "hs_l21_grad": ([_P, _P, _P, _P, _P], C.c_int),
    "hs_gram": ([_P, _P, _P, C.c_int, _P, _P], C.c_int),
    "hs_proj_l2ball": ([_P, _P, _P, _P, C.c_int, _P, _P, _P], C.c_int),
    "hs_proj_l2ball_static": ([C.c_int, _P, _P, _P, _P, C.c_int, C.c_int, _P, _P, _P], C.c_int),
    "hs_norm_l21": ([_P, _P, _P, C.POINTER(C.c_double), _P], C.c_int),
    "hs_op_norm2": ([_P, C.c_int, C.c_double, C.c_uint64, C.POINTER(C.c_double), _P], C.c_int),
    "hs_estimate_mu": ([_P, _P, _P, _P, _P, C.POINTER(C.c_double), _P], C.c_int),
    "hs_pd_state_create": ([_P, _P, _P, C.POINTER(PDParams), C.POINTER(C.c_void_p), _P], C.c_int),
    "hs_pd_state_destroy": ([_P], C.c_int),
    "hs_pd_set_data": ([_P, _P, _P, _P], C.c_int),
    "hs_pd_set_data_host": ([_P, _P, _P, _P], C.c_int),
    "hs_pd_get_host": ([_P, _P, C.POINTER(C.c_double), C.POINTER(C.c_double), _P], C.c_int),
    "hs_pd_step": ([_P, _P], C.c_int),
    "hs_pd_solve": ([_P, C.c_int, C.c_int, _P], C.c_int),
    "hs_pd_get": ([_P, _P, C.POINTER(C.c_double), C.POINTER(C.c_double), _P], C.c_int),
    "hs_pd_iterations": ([_P, C.POINTER(C.c_int64)], C.c_int),
    "hs_pd_reweight": ([_P, C.c_double, C.c_double, _P, _P, _P, _P], C.c_int),
    "hs_pd_graph_kernels": ([_P, C.POINTER(C.c_int)], C.c_int),
    "hs_pd_nuclear_info": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_int), _P], C.c_int),
    "hs_time_stage": ([_P, C.c_int, _P, _P, C.c_int, C.POINTER(C.c_float), _P], C.c_int),
    "hs_daubechies_lowpass": ([C.c_int, C.POINTER(C.c_double)], C.c_int),
    "hs_kb_poly_fit": ([C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double)], C.c_int),
    "hs_kb_poly_coefs": ([C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double)], C.c_int),
    "hs_sweep_lists": ([C.c_int, C.c_int, C.c_int, _P, _P, _P, C.c_int, C.c_int, _P, C.POINTER(C.c_int64), _P,
                        C.POINTER(C.c_int64)], C.c_int),
}
EXPORTED = tuple(_SIGS)


def load(path: Optional[str] = None):
    """Load the library (once). Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; "
                           f"g.build()'` (nvcc, sm_103a)")
    lib = C.CDLL(p)
    for name, (args, res) in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(fn: str, st: int):
    if st != HS_OK:
        msg = load().hs_last_error().decode(errors="replace")
        raise HSError(fn, st, msg)


def version() -> str:
    return load().hs_version().decode()


def last_error() -> str:
    """The calling thread's last error message (hs_last_error)."""
    return load().hs_last_error().decode(errors="replace")


def set_device_limit(nbytes: int):
    """hs_set_device_limit: cap on the device memory plans and states hold (0: none)."""
    _check("hs_set_device_limit", load().hs_set_device_limit(int(nbytes)))


def device_bytes() -> int:
    """hs_device_bytes: device memory the library's plans and states hold now."""
    v = C.c_int64()
    _check("hs_device_bytes", load().hs_device_bytes(C.byref(v)))
    return v.value


def daubechies_lowpass(p: int) -> np.ndarray:
    out = (C.c_double * (2 * p))()
    _check("hs_daubechies_lowpass", load().hs_daubechies_lowpass(p, out))
    return np.array(out[:], dtype=np.float64)


def kb_poly_fit_error(beta: float, terms: int, J: int = 8) -> float:
    e = C.c_double()
    _check("hs_kb_poly_fit", load().hs_kb_poly_fit(J, beta, terms, C.byref(e)))
    return e.value


def kb_poly_coefs(beta: float, terms: int, J: int = 8) -> np.ndarray:
    """hs_kb_poly_coefs: (J, terms) monomial coefficients in s of every unit piece."""
    out = (C.c_double * (J * terms))()
    _check("hs_kb_poly_coefs", load().hs_kb_poly_coefs(J, beta, terms, out))
    return np.array(out[:], dtype=np.float64).reshape(J, terms)


def sweep_lists(Kx: int, Ky: int, offsets, k0x, k0y, hmax: int = 0, cap: int = 0):
    """hs_sweep_lists: the sweep-gridding work lists for windows with start
    cells (k0x, k0y), channel ranges `offsets`, rows cut after hmax rows or cap
    windows (0: defaults). Returns (items (n, 6) int32: channel, strip, row0,
    row1, e0, e1; entries int32, -1 = padding)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    kx = np.ascontiguousarray(k0x, dtype=np.int32)
    ky = np.ascontiguousarray(k0y, dtype=np.int32)
    L = len(off) - 1
    ni, ne = C.c_int64(0), C.c_int64(0)
    args = (Kx, Ky, L, off.ctypes.data, kx.ctypes.data, ky.ctypes.data, int(hmax), int(cap))
    _check("hs_sweep_lists", load().hs_sweep_lists(*args, None, C.byref(ni), None, C.byref(ne)))
    items = np.zeros((max(ni.value, 1), 6), dtype=np.int32)
    ent = np.zeros(max(ne.value, 1), dtype=np.int32)
    _check("hs_sweep_lists", load().hs_sweep_lists(*args, items.ctypes.data, C.byref(ni), ent.ctypes.data,
                                                   C.byref(ne)))
    return items[:ni.value], ent[:ne.value]


# ---------------------------------------------------------------- torch glue
def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _args(*specs):
    """Pointers of checked tensor arguments. Each spec is (tensor, name, dtype,
    numel or None[, optional]): the C functions read and write `numel`
    elements of `dtype` through the pointer and cannot check either, so every
    mismatch is rejected here, for all arguments, before any pointer is taken
    or anything is launched."""
    for spec in specs:
        t, name, dtype, numel = spec[:4]
        optional = len(spec) > 4 and spec[4]
        if t is None:
            if optional:
                continue
            raise ValueError(f"{name} is required")
        if t.dtype != dtype:
            raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return [_ptr(spec[0]) for spec in specs]


def _host_ptr(a, tdtype, numel: int, name: str, np_dtype=None):
    """Pointer of a host buffer (torch CPU tensor or numpy array) after checking
    its element type and count."""
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor")
        if tdtype is not None and a.dtype != tdtype:
            raise ValueError(f"{name} must have dtype {tdtype}, got {a.dtype}")
        if np_dtype is not None and a.dtype != torch.float64:
            raise ValueError(f"{name} must be float64")
        if a.numel() != numel:
            raise ValueError(f"{name} must have {numel} elements, got {a.numel()}")
        return C.c_void_p(a.data_ptr())
    arr = np.asarray(a)
    want = np_dtype if np_dtype is not None else {torch.complex64: np.complex64, torch.complex128: np.complex128,
                                                    torch.float32: np.float32, torch.float64: np.float64}[tdtype]
    if arr.dtype != want or not arr.flags["C_CONTIGUOUS"] or arr.size != numel:
        raise ValueError(f"{name} must be a contiguous {np.dtype(want).name} array of {numel} elements")
    return C.c_void_p(arr.ctypes.data)


class Plan:
    """Measurement plan (hs_plan_create). uv: CUDA tensor (M, 2) of the plan's real dtype."""

    def __init__(self, nx: int, ny: int, offsets: Sequence[int], uv, weights=None, precond=None,
                 oversample: int = 2, J: int = 8, kb_beta: float = 0.0, levels: int = 4,
                 prec: str = "f32", compensated: bool = False, blocks=None, gram_fma: bool = False,
                 autotune: bool = True, fft_chunked: bool = False):
        """blocks: optional offsets (caller order) of intra-channel data blocks, containing
        every channel boundary (hs_plan_create_blocks). gram_fma: form the nuclear prox's
        Gram matrix on the CUDA cores instead of the tensor cores (HS_PLAN_GRAM_FMA).
        autotune=False keeps the default parameters (HS_PLAN_NO_TUNE). fft_chunked: F^H in
        L2-sized channel chunks without timing it (HS_PLAN_FFT_CHUNKED)."""
        torch = _torch()
        lib = load()
        self.nx, self.ny = int(nx), int(ny)
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.offsets = off
        self.L = len(off) - 1
        self.prec = prec
        self.rdtype = torch.float32 if prec == "f32" else torch.float64
        self.cdtype = torch.complex64 if prec == "f32" else torch.complex128
        for name, t in (("uv", uv), ("weights", weights), ("precond", precond)):
            if t is not None and t.dtype != self.rdtype:
                raise ValueError(f"{name} must have dtype {self.rdtype}")
        self._keep = (uv, weights, precond)
        h = C.c_void_p()
        if blocks is None:
            self.blocks = off
            st = lib.hs_plan_create(C.byref(h), self.nx, self.ny, self.L,
                                    off.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(uv), _ptr(weights),
                                    _ptr(precond), oversample, J, float(kb_beta), levels,
                                    HS_F32 if prec == "f32" else HS_F64,
                                    self._flags(compensated, gram_fma, autotune, fft_chunked), _stream())
        else:
            bo = np.ascontiguousarray(np.asarray(blocks, dtype=np.int64))
            self.blocks = bo
            st = lib.hs_plan_create_blocks(C.byref(h), self.nx, self.ny, self.L,
                                           off.ctypes.data_as(C.POINTER(C.c_int64)), len(bo) - 1,
                                           bo.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(uv), _ptr(weights),
                                           _ptr(precond), oversample, J, float(kb_beta), levels,
                                           HS_F32 if prec == "f32" else HS_F64,
                                           self._flags(compensated, gram_fma, autotune, fft_chunked), _stream())
        _check("hs_plan_create", st)
        self.nblocks = len(self.blocks) - 1
        self.h = h
        self._keep = None
        self.M = int(off[-1])

    @staticmethod
    def _flags(compensated: bool, gram_fma: bool, autotune: bool, fft_chunked: bool = False) -> int:
        return ((HS_PLAN_COMPENSATED if compensated else 0) | (HS_PLAN_GRAM_FMA if gram_fma else 0)
                | (0 if autotune else HS_PLAN_NO_TUNE) | (HS_PLAN_FFT_CHUNKED if fft_chunked else 0))

    def check(self):
        """hs_plan_check: synchronise and raise if a bounded device-side wait expired."""
        _check("hs_plan_check", load().hs_plan_check(self.h, _stream()))

    # sizes ----------------------------------------------------------------
    @property
    def info(self) -> dict:
        inf = PlanInfo()
        _check("hs_plan_info", load().hs_plan_info(self.h, C.byref(inf)))
        out = {}
        for k, _ in PlanInfo._fields_:
            v = getattr(inf, k)
            out[k] = list(v) if isinstance(v, C.Array) else v
        return out

    def cube(self, n_bases: int = 0):
        torch = _torch()
        shape = (self.L, self.ny, self.nx) if n_bases == 0 else (n_bases, self.L, self.ny, self.nx)
        return torch.empty(shape, dtype=self.rdtype, device="cuda")

    def vis(self):
        torch = _torch()
        return torch.empty(self.M, dtype=self.cdtype, device="cuda")

    def _img(self, t, name: str, n_bases: int = 0):
        """Argument spec of an image cube (or n_bases coefficient cubes) for _args."""
        return (t, name, self.rdtype, self.L * self.ny * self.nx * (n_bases if n_bases else 1))

    def _vis(self, t, name: str):
        """Argument spec of a visibility vector for _args."""
        return (t, name, self.cdtype, self.M)

    def close(self):
        if getattr(self, "h", None):
            load().hs_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # operators --------------------------------------------------------------
    def phi_fwd(self, X, Y=None):
        Y = self.vis() if Y is None else Y
        pX, pY = _args(self._img(X, "X"), self._vis(Y, "Y"))
        _check("hs_phi_fwd", load().hs_phi_fwd(self.h, pX, pY, _stream()))
        return Y

    def phi_adj(self, Y, X=None):
        X = self.cube() if X is None else X
        pY, pX = _args(self._vis(Y, "Y"), self._img(X, "X"))
        _check("hs_phi_adj", load().hs_phi_adj(self.h, pY, pX, _stream()))
        return X

    def psi_fwd(self, X, A=None):
        A = self.cube(9) if A is None else A
        pX, pA = _args(self._img(X, "X"), self._img(A, "A", 9))
        _check("hs_psi_fwd", load().hs_psi_fwd(self.h, pX, pA, _stream()))
        return A

    def psi_adj(self, A, X=None):
        X = self.cube() if X is None else X
        pA, pX = _args(self._img(A, "A", 9), self._img(X, "X"))
        _check("hs_psi_adj", load().hs_psi_adj(self.h, pA, pX, _stream()))
        return X

    def prox_l21(self, A, thr: float, w_rows=None, dual: bool = False, out=None):
        out = self.cube(9) if out is None else out
        nw = 9 * self.nx * self.ny
        pA, pw, po = _args(self._img(A, "A", 9), (w_rows, "w_rows", self.rdtype, nw, True),
                           self._img(out, "out", 9))
        _check("hs_prox_l21", load().hs_prox_l21(self.h, pA, pw, float(thr), int(dual), po, _stream()))
        return out

    def l21_grad(self, A, w_rows=None, out=None):
        """hs_l21_grad: rows w_n a_n / ||a_n|| (0 for zero rows)."""
        out = self.cube(9) if out is None else out
        nw = 9 * self.nx * self.ny
        pA, pw, po = _args(self._img(A, "A", 9), (w_rows, "w_rows", self.rdtype, nw, True),
                           self._img(out, "out", 9))
        _check("hs_l21_grad", load().hs_l21_grad(self.h, pA, pw, po, _stream()))
        return out

    def prox_nuclear(self, X, thr: float, w_sv=None, dual: bool = False, out=None):
        """Returns (out, singular values as an FP64 CUDA tensor)."""
        torch = _torch()
        out = self.cube() if out is None else out
        pX, pw, po = _args(self._img(X, "X"), (w_sv, "w_sv", torch.float64, self.L, True),
                           self._img(out, "out"))
        sv = torch.empty(self.L, dtype=torch.float64, device="cuda")
        _check("hs_prox_nuclear", load().hs_prox_nuclear(self.h, pX, pw, float(thr), int(dual), po, _ptr(sv),
                                                         _stream()))
        return out, sv

    def gram(self, X, Xadd=None, form: str = "plan"):
        """hs_gram: the L x L Gram matrix of the cube X (+ Xadd), FP64 CUDA tensor.
        form: "plan" (the autotuner's choice), "tensor_cores" or "cuda_cores"."""
        torch = _torch()
        f = {"plan": 0, "tensor_cores": 1, "cuda_cores": 2}[form]
        pX, pA = _args(self._img(X, "X"), self._img(Xadd, "Xadd") + (True,))
        S = torch.empty((self.L, self.L), dtype=torch.float64, device="cuda")
        _check("hs_gram", load().hs_gram(self.h, pX, pA, f, _ptr(S), _stream()))
        return S

    def proj_l2ball(self, Z, Yd, eps, dual: bool = False, out=None):
        """eps: FP64 CUDA tensor (L,). Returns (out, rho) with rho = ||z_l - y_l||."""
        torch = _torch()
        out = self.vis() if out is None else out
        pZ, pY, pe, po = _args(self._vis(Z, "Z"), self._vis(Yd, "Yd"), (eps, "eps", torch.float64, self.L),
                               self._vis(out, "out"))
        rho = torch.empty(self.L, dtype=torch.float64, device="cuda")
        _check("hs_proj_l2ball", load().hs_proj_l2ball(self.h, pZ, pY, pe, int(dual), po, _ptr(rho), _stream()))
        return out, rho

    def norm_l21(self, A, w_rows=None) -> float:
        r = C.c_double()
        pA, pw = _args(self._img(A, "A", 9), (w_rows, "w_rows", self.rdtype, 9 * self.nx * self.ny, True))
        _check("hs_norm_l21", load().hs_norm_l21(self.h, pA, pw, C.byref(r), _stream()))
        return r.value

    def time_stage(self, stage: str, inp=None, out=None, reps: int = 20) -> float:
        """Mean duration (ms) of one stage launched alone (hs_time_stage)."""
        ms = C.c_float()
        _check("hs_time_stage", load().hs_time_stage(self.h, STAGES[stage], _ptr(inp), _ptr(out), int(reps),
                                                     C.byref(ms), _stream()))
        return ms.value

    def estimate_mu(self, Y, A_work=None):
        """hs_estimate_mu: (mu, eta per channel as an FP64 CUDA tensor, dirty cube)."""
        torch = _torch()
        A_work = self.cube(9) if A_work is None else A_work
        pY, pA = _args(self._vis(Y, "Y"), self._img(A_work, "A_work", 9))
        eta = torch.empty(self.L, dtype=torch.float64, device="cuda")
        Xd = self.cube()
        mu = C.c_double()
        _check("hs_estimate_mu", load().hs_estimate_mu(self.h, pY, pA, _ptr(eta), _ptr(Xd), C.byref(mu), _stream()))
        return mu.value, eta, Xd

    def op_norm2(self, iters: int = 500, tol: float = 1e-10, seed: int = 0) -> float:
        r = C.c_double()
        _check("hs_op_norm2", load().hs_op_norm2(self.h, int(iters), float(tol), int(seed), C.byref(r),
                                                 _stream()))
        return r.value


class PDState:
    """Algorithm 2 state (hs_pd_state_create). Y: CUDA complex tensor (caller order);
    eps: FP64 CUDA tensor (L,)."""

    def __init__(self, plan: Plan, Y, eps, *, tau: float = 0.33, kappa1: float = 1.0,
                 kappa2: float = 1.0, kappa3: float = 1.0, mu: float = 0.0, psi_norm2: float = 1.0,
                 use_nuclear: bool = True, use_l21: bool = True, w_nuc=None, w_l21=None,
                 sparsity: str = "l21"):
        """sparsity: "l21" (rows across channels: HyperSARA, JAS) or "l1" (per
        coefficient: SARA; w_l21 is then 9 x L x ny x nx)."""
        if sparsity not in ("l21", "l1"):
            raise ValueError("sparsity must be 'l21' or 'l1'")
        torch = _torch()
        nw = 9 * plan.ny * plan.nx * (plan.L if sparsity == "l1" else 1)
        pY, pe, _, _ = _args(plan._vis(Y, "Y"), (eps, "eps", torch.float64, plan.nblocks),
                             (w_nuc, "w_nuc", torch.float64, plan.L, True), (w_l21, "w_l21", plan.rdtype, nw, True))
        self.plan = plan
        self.sparsity = sparsity
        self._refs = (w_nuc, w_l21)   # the state references these buffers
        prm = PDParams(tau, kappa1, kappa2, kappa3, mu, psi_norm2, int(use_nuclear), int(use_l21),
                       None if w_nuc is None else w_nuc.data_ptr(),
                       None if w_l21 is None else w_l21.data_ptr(), 1 if sparsity == "l1" else 0)
        h = C.c_void_p()
        _check("hs_pd_state_create", load().hs_pd_state_create(plan.h, pY, pe, C.byref(prm),
                                                               C.byref(h), _stream()))
        self.h = h

    def set_data(self, Y, eps):
        torch = _torch()
        pY, pe = _args(self.plan._vis(Y, "Y"), (eps, "eps", torch.float64, self.plan.nblocks))
        _check("hs_pd_set_data", load().hs_pd_set_data(self.h, pY, pe, _stream()))

    def set_data_host(self, Y, eps):
        """hs_pd_set_data_host: Y is a host (preferably pinned) torch tensor or numpy
        array of the plan's complex dtype, eps a host float64 array of one bound per
        data block."""
        yp = _host_ptr(Y, self.plan.cdtype, self.plan.M, "Y")
        ep = _host_ptr(eps, None, self.plan.nblocks, "eps", np.float64)
        _check("hs_pd_set_data_host", load().hs_pd_set_data_host(self.h, yp, ep, _stream()))

    def get_host(self, X):
        """hs_pd_get_host: copies X into the host tensor / array X (plan's real dtype);
        returns (beta, rho per data block)."""
        xp = _host_ptr(X, self.plan.rdtype, self.plan.L * self.plan.ny * self.plan.nx, "X")
        beta = C.c_double()
        rho = (C.c_double * self.plan.nblocks)()
        _check("hs_pd_get_host", load().hs_pd_get_host(self.h, xp, C.byref(beta), rho, _stream()))
        return beta.value, np.array(rho[:])

    def step(self):
        _check("hs_pd_step", load().hs_pd_step(self.h, _stream()))

    def solve(self, iters: int, graph: bool = True):
        _check("hs_pd_solve", load().hs_pd_solve(self.h, int(iters), int(graph), _stream()))

    def get(self, X=None):
        """Returns (X copy, beta, rho per channel as numpy)."""
        X = self.plan.cube() if X is None else X
        beta = C.c_double()
        rho = (C.c_double * self.plan.nblocks)()
        _check("hs_pd_get", load().hs_pd_get(self.h, _ptr(X), C.byref(beta), rho, _stream()))
        return X, beta.value, np.array(rho[:])

    def nuclear_info(self):
        """(singular values of P + X~ at the last step, count above the threshold)."""
        sv = (C.c_double * self.plan.L)()
        n = C.c_int()
        _check("hs_pd_nuclear_info", load().hs_pd_nuclear_info(self.h, sv, C.byref(n), _stream()))
        return np.array(sv[:]), n.value

    def set_adaptive(self, enable: bool = True, lambda1: float = 5e-4, lambda2: float = 0.01,
                     lambda3: float = 0.618, min_gap: int = 100):
        """Adaptive l2 bounds (Algorithm 2 steps 13-19); the paper's defaults."""
        prm = AdaptParams(int(enable), lambda1, lambda2, lambda3, int(min_gap))
        _check("hs_pd_set_adaptive", load().hs_pd_set_adaptive(self.h, C.byref(prm)))

    def bounds(self):
        """(eps, last residuals ||y_b - Phi_b x~||, vartheta) per data block, numpy."""
        nb = self.plan.nblocks
        e, r, t = (C.c_double * nb)(), (C.c_double * nb)(), (C.c_int64 * nb)()
        _check("hs_pd_bounds", load().hs_pd_bounds(self.h, e, r, t, _stream()))
        return np.array(e[:]), np.array(r[:]), np.array(t[:])

    def reweight(self, gamma_l21: float, gamma_nuc: float, w_l21=None, w_nuc=None, sv=None):
        """hs_pd_reweight: Algorithm 1 weights from the current X into w_l21 (9 x ny x nx,
        plan dtype) and w_nuc (L, FP64), and the singular values of X into sv."""
        _check("hs_pd_reweight", load().hs_pd_reweight(self.h, float(gamma_l21), float(gamma_nuc), _ptr(w_l21),
                                                       _ptr(w_nuc), _ptr(sv), _stream()))

    @property
    def graph_kernels(self) -> int:
        n = C.c_int()
        _check("hs_pd_graph_kernels", load().hs_pd_graph_kernels(self.h, C.byref(n)))
        return n.value

    @property
    def iterations(self) -> int:
        n = C.c_int64()
        _check("hs_pd_iterations", load().hs_pd_iterations(self.h, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "h", None):
            load().hs_pd_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reweighted_solve(state: PDState, outer: int, inner: int, decay: float = 0.8, graph: bool = True):
    """Algorithm 1: `outer` re-weights of `inner` PD iterations. The state must
    have been created with weight buffers (w_l21, w_nuc tensors holding ones);
    they are updated in place after every inner loop, gamma and gamma_bar
    starting at 1 and multiplied by `decay` after each update. Without a w_nuc
    buffer only the sparsity weights are updated (JAS, SARA)."""
    w_nuc, w_l21 = state._refs
    if w_l21 is None:
        raise ValueError("reweighted_solve needs a state created with a w_l21 buffer (and w_nuc when the "
                         "nuclear prior is used)")
    gamma = gamma_bar = 1.0
    for _ in range(outer):
        state.solve(inner, graph)
        state.reweight(gamma_bar, gamma, w_l21, w_nuc)
        gamma *= decay
        gamma_bar *= decay
    return state


# Functional names matching the C ABI ----------------------------------------
def phi_fwd(plan: Plan, X, Y=None):
    return plan.phi_fwd(X, Y)


def phi_adj(plan: Plan, Y, X=None):
    return plan.phi_adj(Y, X)


def psi_fwd(plan: Plan, X, A=None):
    return plan.psi_fwd(X, A)


def psi_adj(plan: Plan, A, X=None):
    return plan.psi_adj(A, X)


def prox_l21(plan: Plan, A, thr, w_rows=None, dual=False, out=None):
    return plan.prox_l21(A, thr, w_rows, dual, out)


def prox_nuclear(plan: Plan, X, thr, w_sv=None, dual=False, out=None):
    return plan.prox_nuclear(X, thr, w_sv, dual, out)


def proj_l2ball(plan: Plan, Z, Yd, eps, dual=False, out=None):
    return plan.proj_l2ball(Z, Yd, eps, dual, out)


L2BALL_STATIC_MAX_L = 16384   # HS_L2BALL_STATIC_MAX_L


def proj_l2ball_static(offsets, Z, Yd, eps, dual=False, out=None, prec: str = "f32"):
    """hs_proj_l2ball_static: plan-free projection whose scratch is a fixed
    device array inside the library (no device allocation in the call).
    offsets: int64 CUDA tensor (L + 1,); eps: FP64 CUDA tensor (L,).
    Returns (out, rho)."""
    torch = _torch()
    if prec not in ("f32", "f64"):
        raise ValueError("prec must be 'f32' or 'f64'")
    cdt = torch.complex64 if prec == "f32" else torch.complex128
    L = int(offsets.numel()) - 1
    out = torch.empty_like(Z) if out is None else out
    n = Z.numel()
    args = _args((offsets, "offsets", torch.int64, None), (Z, "Z", cdt, None), (Yd, "Yd", cdt, n),
                 (eps, "eps", torch.float64, max(L, 0)), (out, "out", cdt, n))
    if L >= 1 and int(offsets[-1].item()) != n:   # the kernels index Z, Yd, out up to offsets[L]
        raise ValueError(f"offsets[-1] = {int(offsets[-1].item())} differs from Z.numel() = {n}")
    rho = torch.empty(max(L, 0), dtype=torch.float64, device="cuda")
    _check("hs_proj_l2ball_static",
           load().hs_proj_l2ball_static(L, *args[:4], HS_F32 if prec == "f32" else HS_F64, int(dual), args[4],
                                        _ptr(rho), _stream()))
    return out, rho


def pd_step(state: PDState):
    state.step()


def pd_solve(state: PDState, iters: int, graph: bool = True):
    state.solve(iters, graph)
