"""Python binding of libkron: mu-mode products and Tucker operators on GB300.

A thin ctypes layer over the C ABI of ``include/kron.h``: it marshals torch
tensors (device memory) and the current CUDA stream into the C calls and
allocates workspaces with torch.  Every arithmetic step runs in libkron's
kernels.  There is no CPU fallback: importing this package fails if
``libkron.so`` has not been built (``python paper_2112_11238_gb300/build.py``).

Layout convention (Appendix A, vec operator): tensors are column-major.  A
torch tensor of shape (m_1, ..., m_d) is accepted when its strides are
column-major (stride 1 along the first index); ``colmajor(t)`` returns such a
copy, and outputs are allocated that way.  A matrix L of shape (n, m) needs
stride 1 along its rows and a column stride ``ld >= n``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkron.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libkron.so not found at {LIB_PATH}; build it with "
        "`python paper_2112_11238_gb300/build.py` (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

# ---------------------------------------------------------------- C types
KRON_OK = 0
STATUS = {0: "KRON_OK", 1: "KRON_ERR_INVALID_ARG", 2: "KRON_ERR_UNSUPPORTED",
          3: "KRON_ERR_ALIGNMENT", 4: "KRON_ERR_WORKSPACE", 5: "KRON_ERR_CUDA",
          6: "KRON_ERR_TIMEOUT", 7: "KRON_ERR_NUMERIC"}
F64, F32 = 0, 1
PREC = {"fp64": 0, "fp32": 1, "3xtf32": 2, "bf16x3": 3, "bf16x6": 4, "fx32": 5, "fx32h": 6}
SPLIT_PRECS = ("3xtf32", "bf16x3", "bf16x6")
PLAN_TRANS_L = 0x1
PLAN_NATURAL_ORDER = 0x2
PLAN_UNFUSED = 0x4
MAX_D = 6

_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_ci = ctypes.c_int


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("kron_status_string", [_ci], ctypes.c_char_p)
_sig("kron_version", [], _ci)
_sig("kron_get_device_error", [_vp, ctypes.POINTER(_ci), _ci])
_sig("kron_debug_dependency_timeout", [_ci, ctypes.c_double])
_sig("kron_mump_workspace_size", [_ci, _i64p, _ci, ctypes.c_int64, _ci, _ci, ctypes.POINTER(_sz)])
_sig("kron_mump", [_ci, _i64p, _ci, ctypes.c_int64, _vp, _vp, ctypes.c_int64, _ci, _vp, _ci, _ci, _vp, _sz, _vp])
_sig("kron_mump_noalloc", [_ci, _i64p, _ci, ctypes.c_int64, _vp, _vp, ctypes.c_int64, _ci, _vp, _ci, _ci, _vp])
_sig("kron_plan_create", [ctypes.POINTER(_vp), _ci, _i64p, _i64p, _ci, _ci, ctypes.c_uint])
_sig("kron_plan_destroy", [_vp])
_sig("kron_plan_workspace_size", [_vp, ctypes.POINTER(_sz)])
_sig("kron_plan_order", [_vp, ctypes.POINTER(_ci)])
_sig("kron_plan_launches", [_vp, ctypes.POINTER(_ci), ctypes.POINTER(_ci)])
_sig("kron_plan_flops", [_vp], ctypes.c_double)
_sig("kron_tucker", [_vp, _vp, ctypes.POINTER(_vp), _i64p, _vp, _vp, _sz, _vp])
_sig("kron_ctucker_workspace_size", [_vp, ctypes.POINTER(_sz)])
_sig("kron_gauss_hermite", [ctypes.c_int64, ctypes.c_double, _vp, _vp])
_sig("kron_gauss_laguerre", [ctypes.c_int64, ctypes.c_double, ctypes.c_double, _vp, _vp])
_sig("kron_hermite_functions", [ctypes.c_int64, ctypes.c_double, _vp, ctypes.c_int64, _vp, ctypes.c_int64, _ci, _vp])
_sig("kron_laguerre_functions", [ctypes.c_int64, ctypes.c_double, ctypes.c_double, _vp, ctypes.c_int64, _vp,
                                 ctypes.c_int64, _ci, _vp])
_sig("kron_fourier_resample", [ctypes.c_int64, ctypes.c_int64, _vp, ctypes.c_int64, _vp])
_sig("kron_ctucker", [_vp, _vp, ctypes.POINTER(_vp), _i64p, _ci, _vp, _vp, _sz, _vp])
_sig("kron_kronsumv_workspace_size", [_vp, ctypes.POINTER(_sz)])
_sig("kron_kronsumv", [_vp, _vp, ctypes.POINTER(_vp), _i64p, _vp, _vp, _sz, _vp])
_sig("kron_itucker_workspace_size", [_vp, _ci, ctypes.POINTER(_sz)])
_sig("kron_itucker", [_vp, _vp, ctypes.POINTER(_vp), _i64p, _ci, _vp, _vp, _sz, _vp])
_sig("kron_kronsum_pcg_workspace_size", [_vp, _ci, ctypes.POINTER(_sz)])
_sig("kron_kronsum_pcg", [_vp, ctypes.POINTER(_vp), _i64p, ctypes.POINTER(_vp), _i64p, _vp, _vp, ctypes.c_double,
                          _ci, ctypes.POINTER(_ci), ctypes.POINTER(ctypes.c_double), _vp, _sz, _vp])
_sig("kron_adjoint_workspace_size", [_vp, ctypes.POINTER(_sz)])
_sig("kron_tucker_adjoint", [_vp, _vp, ctypes.POINTER(_vp), _i64p, _vp, _vp, ctypes.POINTER(_vp), _vp, _sz, _vp])
_sig("kron_expm_workspace_size", [ctypes.c_int64, ctypes.POINTER(_sz)])
_sig("kron_expm", [ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_double, _vp, _vp, _sz, _vp])
_sig("kron_expkronsum_workspace_size", [_vp, ctypes.POINTER(_sz)])
_sig("kron_expkronsum_step", [_vp, ctypes.POINTER(_vp), _i64p, ctypes.c_double, _ci, _vp, _vp, _sz, _vp])
_sig("kron_expkronsum_apply", [_vp, ctypes.POINTER(_vp), _i64p, _ci, _vp, _vp, _sz, _vp])
_sig("kron_expkronsum_step_host", [_vp, ctypes.POINTER(_vp), _i64p, ctypes.c_double, _ci, _vp, _vp, _vp, _vp, _sz,
                                   _vp])
_sig("kron_batched_plan_create", [ctypes.POINTER(_vp), _ci, _ci, _i64p, _i64p, _ci, _ci, ctypes.c_uint])
_sig("kron_batched_plan_destroy", [_vp])
_sig("kron_batched_workspace_size", [_vp, ctypes.POINTER(_sz)])
_sig("kron_batched_flops", [_vp], ctypes.c_double)
_sig("kron_batched_bind", [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _sz, _vp])
_sig("kron_batched_run", [_vp, _vp, _sz, _vp])
_sig("kron_batched_autotune", [_vp, _vp, _sz, _vp, ctypes.POINTER(_ci)])
_sig("kron_batched_tuning", [_vp, ctypes.POINTER(_ci), ctypes.POINTER(_ci), ctypes.POINTER(_ci)])
_sig("kron_tucker_batched_workspace_size", [_ci, _ci, _i64p, _i64p, _ci, _ci, ctypes.POINTER(_sz)])
_sig("kron_tucker_batched", [_ci, _ci, _i64p, _i64p, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.POINTER(_vp)),
                             ctypes.POINTER(_vp), _ci, _ci, _vp, _sz, _vp])

EXPORTS = [
    "kron_status_string", "kron_version", "kron_get_device_error", "kron_debug_dependency_timeout",
    "kron_mump_workspace_size",
    "kron_mump", "kron_mump_noalloc", "kron_plan_create", "kron_plan_destroy", "kron_plan_workspace_size",
    "kron_plan_order", "kron_plan_launches", "kron_plan_flops", "kron_tucker", "kron_ctucker_workspace_size", "kron_ctucker",
    "kron_gauss_hermite", "kron_gauss_laguerre", "kron_hermite_functions", "kron_laguerre_functions",
    "kron_fourier_resample", "kron_kronsumv_workspace_size", "kron_kronsumv", "kron_itucker_workspace_size", "kron_itucker", "kron_kronsum_pcg_workspace_size", "kron_kronsum_pcg", "kron_adjoint_workspace_size",
    "kron_tucker_adjoint", "kron_expm_workspace_size", "kron_expm",
    "kron_expkronsum_workspace_size", "kron_expkronsum_step", "kron_expkronsum_apply", "kron_expkronsum_step_host",
    "kron_batched_plan_create", "kron_batched_plan_destroy", "kron_batched_workspace_size",
    "kron_batched_flops", "kron_batched_bind", "kron_batched_run",
    "kron_tucker_batched_workspace_size", "kron_tucker_batched", "kron_batched_autotune", "kron_batched_tuning",
]


class KronError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


def _check(rc: int, what: str) -> None:
    if rc != KRON_OK:
        raise KronError(rc, what)


def version() -> int:
    return int(_lib.kron_version())


def device_error(clear: bool = True, stream=None) -> int:
    """The device error word (bit 0: a kernel's bounded wait timed out; bit 1:
    non-finite input), read in order on `stream` (default: the current
    stream), which it waits for; cleared unless clear=False."""
    code = ctypes.c_int(0)
    rc = _lib.kron_get_device_error(_stream(stream), ctypes.byref(code), int(clear))
    if rc not in (KRON_OK, 6, 7):
        _check(rc, "kron_get_device_error")
    return int(code.value)


def debug_dependency_timeout(hold: bool, limit_ms: float = 0.0) -> None:
    """Test hook: with hold, every in-launch job dependency of the persistent
    kernel waits until its time limit (limit_ms; 0 = 2 s), latches the timeout
    bit and carries on.  hold=False restores normal operation."""
    _check(_lib.kron_debug_dependency_timeout(int(bool(hold)), float(limit_ms)), "kron_debug_dependency_timeout")


# ----------------------------------------------------------------- helpers

def _i64(vals):
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() if t is not None else None for t in ts])


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"libkron supports float64 and float32 tensors, got {t.dtype}")


def colmajor_strides(shape):
    st, acc = [], 1
    for s in shape:
        st.append(acc)
        acc *= max(int(s), 1)
    return tuple(st)


def is_colmajor(t: torch.Tensor) -> bool:
    return all(t.stride(k) == s or t.shape[k] == 1
               for k, s in enumerate(colmajor_strides(t.shape)))


def pinned_colmajor(shape, dtype=torch.float64) -> torch.Tensor:
    """Page-locked host tensor with column-major strides (for step_host)."""
    return torch.empty_strided(tuple(int(s) for s in shape), colmajor_strides(shape), dtype=dtype, pin_memory=True)


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """Copy (if needed) of t with column-major strides."""
    if is_colmajor(t):
        return t
    out = torch.empty_strided(tuple(t.shape), colmajor_strides(t.shape), dtype=t.dtype, device=t.device)
    out.copy_(t)
    return out


def empty_colmajor(shape, dtype, device) -> torch.Tensor:
    return torch.empty_strided(tuple(int(s) for s in shape), colmajor_strides(shape), dtype=dtype, device=device)


def _mat(L: torch.Tensor):
    """(tensor, ld) of a column-major matrix, copying if its layout is not one."""
    if L.dim() != 2:
        raise ValueError("L must be a matrix")
    if L.stride(0) != 1 or L.stride(1) < max(L.shape[0], 1):
        L = colmajor(L)
    return L, max(L.stride(1), L.shape[0], 1)


def _prec(p) -> int:
    if isinstance(p, int):
        return p
    return PREC[p.lower()]


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("libkron works on CUDA tensors only (no CPU fallback)")


# --------------------------------------------------------------- mu-mode

def mump_workspace(T: torch.Tensor, L: torch.Tensor, mu: int, trans: bool = False, prec="fp64") -> torch.Tensor:
    """A workspace large enough for mump_into with these operands."""
    n = L.shape[1] if trans else L.shape[0]
    need = ctypes.c_size_t(0)
    _check(_lib.kron_mump_workspace_size(T.dim(), _i64(list(T.shape)), mu, n, _dtype_code(T), _prec(prec),
                                         ctypes.byref(need)), "kron_mump_workspace_size")
    return _workspace(need.value, T.device)


def mump_into(T: torch.Tensor, L: torch.Tensor, mu: int, S: torch.Tensor, trans: bool = False,
              prec="fp64", ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """S = T x_mu op(L) (Eq. (mmp)) into a preallocated column-major S."""
    _require_cuda(T, L, S)
    L, ld = _mat(L)
    d = T.dim()
    m = list(T.shape)
    n = L.shape[1] if trans else L.shape[0]
    dt, pc = _dtype_code(T), _prec(prec)
    need = ctypes.c_size_t(0)
    _check(_lib.kron_mump_workspace_size(d, _i64(m), mu, n, dt, pc, ctypes.byref(need)), "kron_mump_workspace_size")
    if ws is None or ws.numel() < need.value:
        ws = _workspace(need.value, T.device)
    _check(_lib.kron_mump(d, _i64(m), mu, n, T.data_ptr(), L.data_ptr(), ld, int(trans), S.data_ptr(), dt, pc,
                          ws.data_ptr(), ws.numel(), _stream(stream)), "kron_mump")
    return S


def mump(T: torch.Tensor, L: torch.Tensor, mu: int, trans: bool = False, prec="fp64", stream=None) -> torch.Tensor:
    """T x_mu op(L): op(L) applied to every mu-fibre of T (mu 0-based)."""
    T = colmajor(T)
    n = L.shape[1] if trans else L.shape[0]
    shape = list(T.shape)
    shape[mu] = n
    S = empty_colmajor(shape, T.dtype, T.device)
    return mump_into(T, L.to(T.dtype), mu, S, trans, prec, stream=stream)


# ------------------------------------------------------------------ Tucker

class TuckerPlan:
    """A libkron plan: fixed d, sizes, dtype, precision and mode order."""

    def __init__(self, m, n, dtype=torch.float64, prec="fp64", trans: bool = False,
                 natural_order: bool = False, fused: bool = True):
        self.m = [int(v) for v in m]
        self.n = [int(v) for v in n]
        self.d = len(self.m)
        self.dtype = dtype
        self.prec = prec
        self.trans = trans
        flags = ((PLAN_TRANS_L if trans else 0) | (PLAN_NATURAL_ORDER if natural_order else 0) |
                 (0 if fused else PLAN_UNFUSED))
        h = ctypes.c_void_p()
        # complex plans take the dtype of the real and imaginary parts
        dt = F64 if dtype in (torch.float64, torch.complex128) else F32
        _check(_lib.kron_plan_create(ctypes.byref(h), self.d, _i64(self.m), _i64(self.n), dt, _prec(prec), flags),
               "kron_plan_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.kron_plan_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self) -> int:
        b = ctypes.c_size_t(0)
        _check(_lib.kron_plan_workspace_size(self._h, ctypes.byref(b)), "kron_plan_workspace_size")
        return b.value

    def adjoint_workspace_bytes(self) -> int:
        b = ctypes.c_size_t(0)
        _check(_lib.kron_adjoint_workspace_size(self._h, ctypes.byref(b)), "kron_adjoint_workspace_size")
        return b.value

    def stepper_workspace_bytes(self) -> int:
        b = ctypes.c_size_t(0)
        _check(_lib.kron_expkronsum_workspace_size(self._h, ctypes.byref(b)), "kron_expkronsum_workspace_size")
        return b.value

    def order(self):
        o = (ctypes.c_int * self.d)()
        _check(_lib.kron_plan_order(self._h, o), "kron_plan_order")
        return list(o)

    def launches(self):
        """Mode products per launch of kron_tucker, in the plan's order (2 or 3:
        a fused group of small modes)."""
        sz = (ctypes.c_int * self.d)()
        cnt = ctypes.c_int(0)
        _check(_lib.kron_plan_launches(self._h, sz, ctypes.byref(cnt)), "kron_plan_launches")
        return list(sz)[:cnt.value]

    def flops(self) -> float:
        return float(_lib.kron_plan_flops(self._h))

    def workspace(self, device="cuda") -> torch.Tensor:
        return _workspace(self.workspace_bytes(), device)

    def tucker_into(self, T, Ls, S, ws=None, stream=None):
        """S = T x_1 op(L_1) ... x_d op(L_d) with preallocated column-major S."""
        _require_cuda(T, S, *Ls)
        mats = [_mat(L) for L in Ls]
        if ws is None:
            ws = self.workspace(T.device)
        _check(_lib.kron_tucker(self._h, T.data_ptr(), _ptrs([L for L, _ in mats]), _i64([ld for _, ld in mats]),
                                S.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "kron_tucker")
        return S

    def ctucker_workspace_bytes(self) -> int:
        b = ctypes.c_size_t(0)
        _check(_lib.kron_ctucker_workspace_size(self._h, ctypes.byref(b)), "kron_ctucker_workspace_size")
        return b.value

    def ctucker_into(self, T, Ls, S, conj: bool = False, ws=None, stream=None):
        """Complex Tucker operator S = T x_1 op(L_1) ... x_d op(L_d) with op(L) = L, L^T
        (trans plan) and their conjugates (conj); the paper's cttucker is a trans plan
        with conj.  T, L_mu, S complex (complex128 / complex64), column-major."""
        _require_cuda(T, S, *Ls)
        if not (T.is_complex() and S.is_complex() and all(L.is_complex() for L in Ls)):
            raise ValueError("ctucker takes complex tensors")
        mats = [_mat(L) for L in Ls]
        if ws is None:
            ws = _workspace(self.ctucker_workspace_bytes(), T.device)
        _check(_lib.kron_ctucker(self._h, T.data_ptr(), _ptrs([L for L, _ in mats]), _i64([ld for _, ld in mats]),
                                 int(bool(conj)), S.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)),
               "kron_ctucker")
        return S

    def kronsumv_workspace_bytes(self) -> int:
        b = ctypes.c_size_t(0)
        _check(_lib.kron_kronsumv_workspace_size(self._h, ctypes.byref(b)), "kron_kronsumv_workspace_size")
        return b.value

    def kronsumv_into(self, V, Ls, S, ws=None, stream=None):
        """S = sum_mu V x_mu op(L_mu) with preallocated column-major S (Eq. (actkron))."""
        _require_cuda(V, S, *Ls)
        mats = [_mat(L) for L in Ls]
        if ws is None:
            ws = _workspace(self.kronsumv_workspace_bytes(), V.device)
        _check(_lib.kron_kronsumv(self._h, V.data_ptr(), _ptrs([L for L, _ in mats]), _i64([ld for _, ld in mats]),
                                  S.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "kron_kronsumv")
        return S

    def itucker_workspace_bytes(self, refine: int = 0) -> int:
        b = ctypes.c_size_t(0)
        _check(_lib.kron_itucker_workspace_size(self._h, int(refine), ctypes.byref(b)), "kron_itucker_workspace_size")
        return b.value

    def itucker_into(self, V, Ps, S, refine: int = 0, ws=None, stream=None):
        """S = V x_1 op(P_1)^{-1} ... x_d op(P_d)^{-1} (Eq. (preconnd))."""
        _require_cuda(V, S, *Ps)
        mats = [_mat(P) for P in Ps]
        if ws is None:
            ws = _workspace(self.itucker_workspace_bytes(refine), V.device)
        _check(_lib.kron_itucker(self._h, V.data_ptr(), _ptrs([P for P, _ in mats]), _i64([ld for _, ld in mats]),
                                 int(refine), S.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)),
               "kron_itucker")
        return S

    def pcg_workspace_bytes(self, precondition: bool = True) -> int:
        b = ctypes.c_size_t(0)
        _check(_lib.kron_kronsum_pcg_workspace_size(self._h, int(bool(precondition)), ctypes.byref(b)),
               "kron_kronsum_pcg_workspace_size")
        return b.value

    def kronsum_pcg(self, Ms, B, X, Ps=None, tol: float = 1e-6, maxit: int = 20, ws=None, stream=None):
        """Solve (M_d (+) ... (+) M_1) x = b by CG, preconditioned by
        P_d (x) ... (x) P_1 when Ps is given; X: initial guess, overwritten.
        Returns (X, iterations, relative residual)."""
        _require_cuda(B, X, *Ms, *(Ps or []))
        mats = [_mat(M) for M in Ms]
        pm = [_mat(P) for P in Ps] if Ps is not None else None
        if ws is None:
            ws = _workspace(self.pcg_workspace_bytes(Ps is not None), B.device)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        _check(_lib.kron_kronsum_pcg(self._h, _ptrs([M for M, _ in mats]), _i64([ld for _, ld in mats]),
                                     _ptrs([P for P, _ in pm]) if pm else None,
                                     _i64([ld for _, ld in pm]) if pm else None,
                                     B.data_ptr(), X.data_ptr(), float(tol), int(maxit), ctypes.byref(it),
                                     ctypes.byref(rr), ws.data_ptr(), ws.numel(), _stream(stream)),
               "kron_kronsum_pcg")
        return X, it.value, rr.value

    def adjoint_into(self, T, Ls, dS, dT=None, dLs=None, ws=None, stream=None):
        mats = [_mat(L) for L in Ls]
        if ws is None:
            ws = _workspace(self.adjoint_workspace_bytes(), dS.device)
        dLp = _ptrs(dLs) if dLs is not None else None
        _check(_lib.kron_tucker_adjoint(self._h, T.data_ptr() if T is not None else None,
                                        _ptrs([L for L, _ in mats]), _i64([ld for _, ld in mats]),
                                        dS.data_ptr(), dT.data_ptr() if dT is not None else None, dLp,
                                        ws.data_ptr(), ws.numel(), _stream(stream)), "kron_tucker_adjoint")
        return dT, dLs


def tucker(T: torch.Tensor, Ls, prec="fp64", trans: bool = False, natural_order: bool = False,
           fused: bool = True, stream=None) -> torch.Tensor:
    """Tucker operator T x_1 op(L_1) x_2 ... x_d op(L_d) (Eq. (tuckerop)); fused=False
    runs every mode product of the split forms as its own launch."""
    T = colmajor(T)
    Ls = [L.to(T.dtype) for L in Ls]
    n = [(L.shape[1] if trans else L.shape[0]) for L in Ls]
    plan = TuckerPlan(T.shape, n, T.dtype, prec, trans, natural_order, fused)
    S = empty_colmajor(n, T.dtype, T.device)
    return plan.tucker_into(T, Ls, S, stream=stream)


def ctucker(T: torch.Tensor, Ls, prec="fp64", trans: bool = False, conj: bool = False,
            natural_order: bool = False, stream=None) -> torch.Tensor:
    """Complex Tucker operator T x_1 op(L_1) ... x_d op(L_d) (Eq. (tuckerop) over C),
    op(L) = L, L^T (trans) or their conjugates (conj)."""
    T = colmajor(T)
    if not T.is_complex():
        raise ValueError("ctucker takes a complex tensor")
    Ls = [L.to(T.dtype) for L in Ls]
    n = [(L.shape[1] if trans else L.shape[0]) for L in Ls]
    plan = TuckerPlan(T.shape, n, T.dtype, prec, trans, natural_order)
    S = empty_colmajor(n, T.dtype, T.device)
    return plan.ctucker_into(T, Ls, S, conj=conj, stream=stream)


def cttucker(T: torch.Tensor, Psis, prec="fp64", stream=None) -> torch.Tensor:
    """T x_1 Psi_1^* x_2 ... x_d Psi_d^* (conjugate transposes; the remark after
    Eq. (tensinterp)): evaluation at the quadrature points without forming Psi_mu^*."""
    return ctucker(T, Psis, prec=prec, trans=True, conj=True, stream=stream)


def gauss_hermite(m: int, beta: float):
    """Scaled Gauss-Hermite nodes and function weights (numpy float64 arrays of length m):
    sum_k w_k f(x_k) H_i(x_k) approximates the coefficient of f on H_i."""
    x = np.zeros(int(m))
    w = np.zeros(int(m))
    _check(_lib.kron_gauss_hermite(int(m), float(beta), x.ctypes.data, w.ctypes.data), "kron_gauss_hermite")
    return x, w


def gauss_laguerre(m: int, alpha: float, beta: float):
    """Scaled generalized Gauss-Laguerre nodes and function weights (numpy float64)."""
    x = np.zeros(int(m))
    w = np.zeros(int(m))
    _check(_lib.kron_gauss_laguerre(int(m), float(alpha), float(beta), x.ctypes.data, w.ctypes.data),
           "kron_gauss_laguerre")
    return x, w


def _points(x, device):
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(np.asarray(x, dtype=np.float64))
    return x.to(device=device, dtype=torch.float64).contiguous()


def hermite_functions(m: int, beta: float, x, trans: bool = False, device="cuda", stream=None) -> torch.Tensor:
    """Normalized scaled Hermite functions H_i(x_l), i < m: an n x m column-major
    matrix (the evaluation matrix Phi), or m x n with trans (the transform matrix Psi)."""
    x = _points(x, device)
    n = x.numel()
    F = empty_colmajor((m, n) if trans else (n, m), torch.float64, x.device)
    _check(_lib.kron_hermite_functions(int(m), float(beta), x.data_ptr(), n, F.data_ptr(), max(F.shape[0], 1),
                                       int(bool(trans)), _stream(stream)), "kron_hermite_functions")
    return F


def laguerre_functions(m: int, alpha: float, beta: float, x, trans: bool = False, device="cuda",
                       stream=None) -> torch.Tensor:
    """Normalized scaled generalized Laguerre functions L_i(x_l) (x >= 0), layout as
    hermite_functions."""
    x = _points(x, device)
    n = x.numel()
    F = empty_colmajor((m, n) if trans else (n, m), torch.float64, x.device)
    _check(_lib.kron_laguerre_functions(int(m), float(alpha), float(beta), x.data_ptr(), n, F.data_ptr(),
                                        max(F.shape[0], 1), int(bool(trans)), _stream(stream)),
           "kron_laguerre_functions")
    return F


def fourier_resample(m: int, n: int, device="cuda", stream=None) -> torch.Tensor:
    """The real n x m matrix of the trigonometric interpolation of m equispaced samples of
    a period, evaluated at n equispaced points."""
    F = empty_colmajor((n, m), torch.float64, device)
    _check(_lib.kron_fourier_resample(int(m), int(n), F.data_ptr(), int(n), _stream(stream)),
           "kron_fourier_resample")
    return F


def kronsumv(V: torch.Tensor, Ls, prec="fp64", trans: bool = False, stream=None) -> torch.Tensor:
    """Action of the Kronecker sum: sum_mu V x_mu op(L_mu), i.e.
    vec(S) = (L_d (+) ... (+) L_1) vec(V) (Eq. (actkron)); L_mu square."""
    V = colmajor(V)
    Ls = [L.to(V.dtype) for L in Ls]
    plan = TuckerPlan(V.shape, list(V.shape), V.dtype, prec, trans, natural_order=True)
    S = empty_colmajor(V.shape, V.dtype, V.device)
    return plan.kronsumv_into(V, Ls, S, stream=stream)


def itucker(V: torch.Tensor, Ps, prec="fp64", trans: bool = False, refine: int = 0, stream=None) -> torch.Tensor:
    """Inverse Tucker operator V x_1 op(P_1)^{-1} ... x_d op(P_d)^{-1} (Eq. (preconnd)),
    with `refine` steps of FP64-residual iterative refinement."""
    V = colmajor(V)
    Ps = [P.to(V.dtype) for P in Ps]
    plan = TuckerPlan(V.shape, list(V.shape), V.dtype, prec, trans)
    S = empty_colmajor(V.shape, V.dtype, V.device)
    return plan.itucker_into(V, Ps, S, refine=refine, stream=stream)


def kronsum_pcg(Ms, B: torch.Tensor, X0=None, Ps=None, tol: float = 1e-6, maxit: int = 20, prec="fp64",
                stream=None):
    """(M_d (+) ... (+) M_1) x = b by (preconditioned) CG on the tensor B;
    returns (X, iterations, relative residual) (Sections 3.4 and 4.5)."""
    B = colmajor(B)
    Ms = [M.to(B.dtype) for M in Ms]
    Ps = [P.to(B.dtype) for P in Ps] if Ps is not None else None
    plan = TuckerPlan(B.shape, list(B.shape), B.dtype, prec, natural_order=True)
    X = empty_colmajor(B.shape, B.dtype, B.device)
    if X0 is None:
        X.zero_()
    else:
        X.copy_(X0)
    return plan.kronsum_pcg(Ms, B, X, Ps, tol, maxit, stream=stream)


def tucker_adjoint(T: torch.Tensor, Ls, dS: torch.Tensor, prec="fp64", want_dT: bool = True,
                   want_dL: bool = True, stream=None):
    """(dT, [dL_mu]) of <tucker(T, L), dS> (hand-written adjoint)."""
    T = colmajor(T)
    dS = colmajor(dS.to(T.dtype))
    Ls = [L.to(T.dtype) for L in Ls]
    plan = TuckerPlan(T.shape, [L.shape[0] for L in Ls], T.dtype, prec, natural_order=True)
    dT = empty_colmajor(T.shape, T.dtype, T.device) if want_dT else None
    dLs = [empty_colmajor(L.shape, T.dtype, T.device) for L in Ls] if want_dL else None
    plan.adjoint_into(T, Ls, dS, dT, dLs, stream=stream)
    return dT, dLs


class KronTucker(torch.autograd.Function):
    """S = tucker(T, L_1..L_d) with the hand-written adjoint as backward."""

    @staticmethod
    def forward(ctx, prec, T, *Ls):
        T = colmajor(T)
        Ls = [colmajor(L) for L in Ls]
        ctx.prec = prec
        ctx.save_for_backward(T, *Ls)
        return tucker(T, Ls, prec=prec, natural_order=True)

    @staticmethod
    def backward(ctx, dS):
        T, *Ls = ctx.saved_tensors
        need_T = ctx.needs_input_grad[1]
        need_L = any(ctx.needs_input_grad[2:])
        dT, dLs = tucker_adjoint(T, Ls, dS, prec=ctx.prec, want_dT=need_T, want_dL=need_L)
        grads = [None, dT]
        grads += dLs if dLs is not None else [None] * len(Ls)
        return tuple(grads)


def tucker_autograd(T, Ls, prec="bf16x6"):
    """tucker(T, Ls) differentiable in T and every L_mu (the hand-written
    adjoint as backward).  The default BF16x6 keeps the gradient within 1e-6
    of central differences of the FP64 loss; 3XTF32 comes out about 2e-6 off
    on the d=4 n=48 workload."""
    return KronTucker.apply(prec, T, *Ls)


# ------------------------------------------------------------ exponential

def expm(A: torch.Tensor, tau: float = 1.0, stream=None) -> torch.Tensor:
    """exp(tau A) of a square FP64 CUDA matrix (Pade [13/13], scaling and squaring)."""
    _require_cuda(A)
    A, ld = _mat(A.to(torch.float64))
    n = A.shape[0]
    need = ctypes.c_size_t(0)
    _check(_lib.kron_expm_workspace_size(n, ctypes.byref(need)), "kron_expm_workspace_size")
    ws = _workspace(need.value, A.device)
    E = empty_colmajor((n, n), torch.float64, A.device)
    _check(_lib.kron_expm(n, A.data_ptr(), ld, float(tau), E.data_ptr(), ws.data_ptr(), ws.numel(),
                          _stream(stream)), "kron_expm")
    return E


class StepperPlan:
    """Exponential-of-Kronecker-sum stepper U <- U x_1 exp(tau A_1) ... (Eq. (exptucker))."""

    def __init__(self, n, dtype=torch.float64, prec="fx32h"):
        # default: the fixed-point form, which keeps the 100-step stepper
        # within 2e-6; the FP32-accumulating split forms (3XTF32, BF16X*)
        # drift by about 1e-6 per step over chained steps
        self.plan = TuckerPlan(n, n, dtype, prec)
        self.n = list(n)

    def workspace(self, device="cuda"):
        return _workspace(self.plan.stepper_workspace_bytes(), device)

    def step(self, U, As, tau: float, nsteps: int, ws=None, stream=None):
        """nsteps steps in place on the column-major tensor U; A_mu FP64 matrices."""
        _require_cuda(U, *As)
        mats = [_mat(A) for A in As]
        if ws is None:
            ws = self.workspace(U.device)
        _check(_lib.kron_expkronsum_step(self.plan.handle, _ptrs([A for A, _ in mats]),
                                         _i64([ld for _, ld in mats]), float(tau), int(nsteps), U.data_ptr(),
                                         ws.data_ptr(), ws.numel(), _stream(stream)), "kron_expkronsum_step")
        return U

    def step_host(self, U_in, As, tau: float, nsteps: int, U_out=None, U_dev=None, ws=None, stream=None):
        """nsteps steps of a host state: U_in (CPU, column-major, best page-locked)
        is copied to U_dev while the exponentials are computed, the steps run
        there, and the result lands in U_out (CPU; default U_in).  Enqueued on
        `stream`: U_out is complete once the stream is."""
        _require_cuda(*As)
        if U_in.is_cuda or (U_out is not None and U_out.is_cuda):
            raise ValueError("step_host takes host tensors U_in / U_out")
        U_out = U_in if U_out is None else U_out
        if not (is_colmajor(U_in) and is_colmajor(U_out)):
            raise ValueError("step_host takes column-major host tensors (see pinned_colmajor)")
        if U_out.shape != U_in.shape or U_out.dtype != U_in.dtype:
            raise ValueError("U_out must match U_in")
        dev = As[0].device
        if U_dev is None:
            U_dev = empty_colmajor(U_in.shape, U_in.dtype, dev)
        mats = [_mat(A) for A in As]
        if ws is None:
            ws = self.workspace(dev)
        _check(_lib.kron_expkronsum_step_host(self.plan.handle, _ptrs([A for A, _ in mats]),
                                              _i64([ld for _, ld in mats]), float(tau), int(nsteps),
                                              ctypes.c_void_p(U_in.data_ptr()), ctypes.c_void_p(U_out.data_ptr()),
                                              ctypes.c_void_p(U_dev.data_ptr()), ws.data_ptr(), ws.numel(),
                                              _stream(stream)), "kron_expkronsum_step_host")
        return U_out

    def apply(self, U, Es, nsteps: int, ws=None, stream=None):
        """nsteps steps with given FP64 E_mu = exp(tau A_mu)."""
        _require_cuda(U, *Es)
        mats = [_mat(E) for E in Es]
        if ws is None:
            ws = self.workspace(U.device)
        _check(_lib.kron_expkronsum_apply(self.plan.handle, _ptrs([E for E, _ in mats]),
                                          _i64([ld for _, ld in mats]), int(nsteps), U.data_ptr(),
                                          ws.data_ptr(), ws.numel(), _stream(stream)), "kron_expkronsum_apply")
        return U


def expkronsum_step(U: torch.Tensor, As, tau: float, nsteps: int, prec="fx32h", stream=None) -> torch.Tensor:
    """Returns U after nsteps steps of exp(tau (A_d (+) ... (+) A_1)) (a new tensor)."""
    U = colmajor(U).clone()
    StepperPlan(U.shape, U.dtype, prec).step(U, [A.to(torch.float64) for A in As], tau, nsteps, stream=stream)
    return U


# ----------------------------------------------------------------- batched

class BatchedPlan:
    """Many independent Tucker operators (same d) in one persistent launch."""

    def __init__(self, m, n, dtype=torch.float32, prec="3xtf32"):
        import numpy as np
        m = np.asarray(m, dtype=np.int64)
        n = np.asarray(n, dtype=np.int64)
        self.batch, self.d = m.shape
        self.m, self.n = m, n
        h = ctypes.c_void_p()
        dt = F64 if dtype == torch.float64 else F32
        _check(_lib.kron_batched_plan_create(ctypes.byref(h), self.batch, self.d, _i64(m.ravel()),
                                             _i64(n.ravel()), dt, _prec(prec), 0), "kron_batched_plan_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.kron_batched_plan_destroy(h)
            self._h = None

    def workspace(self, device="cuda"):
        b = ctypes.c_size_t(0)
        _check(_lib.kron_batched_workspace_size(self._h, ctypes.byref(b)), "kron_batched_workspace_size")
        return _workspace(b.value, device)

    def flops(self) -> float:
        return float(_lib.kron_batched_flops(self._h))

    def bind(self, Ts, Ls, Ss, ws, stream=None):
        """Uploads the pointer tables; Ls is a list (per problem) of d matrices (ld = n)."""
        flatL = [L for row in Ls for L in row]
        _check(_lib.kron_batched_bind(self._h, _ptrs(Ts), _ptrs(flatL), _ptrs(Ss), ws.data_ptr(), ws.numel(),
                                      _stream(stream)), "kron_batched_bind")

    def run(self, ws, stream=None):
        _check(_lib.kron_batched_run(self._h, ws.data_ptr(), ws.numel(), _stream(stream)), "kron_batched_run")

    def autotune(self, ws, stream=None) -> bool:
        """Times candidate launch configurations on the bound operands (their
        outputs are overwritten) and keeps the fastest; with
        KRON_AUTOTUNE_CACHE set, reuses / records the choice there.  Returns
        True when the choice came from the cache."""
        hit = ctypes.c_int(0)
        _check(_lib.kron_batched_autotune(self._h, ws.data_ptr(), ws.numel(), _stream(stream), ctypes.byref(hit)),
               "kron_batched_autotune")
        return bool(hit.value)

    def tuning(self):
        """(N-tile width cap, stages, accumulator sets); 0 = built-in rule."""
        a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(_lib.kron_batched_tuning(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "kron_batched_tuning")
        return a.value, b.value, c.value


def tucker_batched(Ts, Ls, prec="3xtf32", stream=None):
    """[T_b x_1 L_b1 ... x_d L_bd for every b] in one persistent launch (the
    one-shot C call); Ts: list of column-major tensors (same d and dtype),
    Ls: list per problem of d matrices."""
    _require_cuda(*Ts)
    batch, d = len(Ts), Ts[0].dim()
    dtype = Ts[0].dtype
    Ts = [colmajor(t) for t in Ts]
    Ls = [[colmajor(L.to(dtype)) for L in row] for row in Ls]
    m = np.array([list(t.shape) for t in Ts], dtype=np.int64)
    n = np.array([[L.shape[0] for L in row] for row in Ls], dtype=np.int64)
    dt, pc = _dtype_code(Ts[0]), _prec(prec)
    need = ctypes.c_size_t(0)
    _check(_lib.kron_tucker_batched_workspace_size(batch, d, _i64(m.ravel()), _i64(n.ravel()), dt, pc,
                                                   ctypes.byref(need)), "kron_tucker_batched_workspace_size")
    ws = _workspace(need.value, Ts[0].device)
    Ss = [empty_colmajor(tuple(int(v) for v in n[b]), dtype, Ts[0].device) for b in range(batch)]
    rows = [_ptrs(row) for row in Ls]
    Lp = (ctypes.POINTER(ctypes.c_void_p) * batch)(*[ctypes.cast(r, ctypes.POINTER(ctypes.c_void_p)) for r in rows])
    _check(_lib.kron_tucker_batched(batch, d, _i64(m.ravel()), _i64(n.ravel()), _ptrs(Ts), Lp, _ptrs(Ss), dt, pc,
                                    ws.data_ptr(), ws.numel(), _stream(stream)), "kron_tucker_batched")
    return Ss
