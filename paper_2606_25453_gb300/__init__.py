"""GB300 (sm_103a) emulated FP64 / FP32 / complex GEMM on INT8 tensor cores.

A thin ctypes binding over the C ABI in ``include/emugemm.h``
(``libemugemm.so``, built by ``paper_2606_25453_gb300.build``).  The names
match the C entry points; arguments are marshalled and nothing is computed
here.  Device memory and streams come from PyTorch.  There is no fallback:
if the CUDA library is missing, importing this package raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build_mod

_LIB_PATH = _build_mod.LIB

EMU_ROW_MAJOR, EMU_COL_MAJOR = 0, 1
EMU_SCHEME_I, EMU_SCHEME_II, EMU_SCHEME_I_F8, EMU_SCHEME_II_NORM = 1, 2, 3, 4
STATUS = {0: "EMU_OK", 1: "EMU_ERR_INVALID_ARG", 2: "EMU_ERR_UNSUPPORTED", 3: "EMU_ERR_NONFINITE",
          4: "EMU_ERR_CUDA", 5: "EMU_ERR_ALLOC", 6: "EMU_ERR_TIMEOUT", 7: "EMU_ERR_TOL_NOT_MET"}
EMU_P_MAX, EMU_NM_MAX, EMU_K_MAX_II = 12, 20, 131071
SEL_NPARAM, SEL_IN, SEL_OUT, SEL_P0 = 8968, 66, 8, 3


class EmuError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__("%s%s" % (STATUS.get(code, "EMU_ERR_%d" % code), (" in " + where) if where else ""))


if not os.path.exists(_LIB_PATH):
    raise ImportError("libemugemm.so is not built (%s); run paper_2606_25453_gb300.build.build() "
                      "or __graft_entry__.build() first" % _LIB_PATH)

lib = ctypes.CDLL(_LIB_PATH)

_i64, _i32, _dbl, _flt, _vp, _sz = (ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_float,
                                    ctypes.c_void_p, ctypes.c_size_t)
class GemmDesc(ctypes.Structure):
    """emu_gemm_desc_t: one row-major product of a grouped call."""
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p),
                ("ldb", ctypes.c_int64), ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


_SIGS = {
    "emu_create": (_i32, [ctypes.POINTER(_vp), _i32]),
    "emu_destroy": (_i32, [_vp]),
    "emu_get_status": (_i32, [_vp, _vp]),
    "emu_status_string": (ctypes.c_char_p, [_i32]),
    "emu_last_cuda_error": (ctypes.c_char_p, []),
    "emu_selftest_wait": (_i32, [_vp, _i64, _vp]),
    "emu_workspace_size": (_i32, [_i32, _i64, _i64, _i64, _i32, _i32, ctypes.POINTER(_sz)]),
    "emu_set_workspace": (_i32, [_vp, _vp, _sz]),
    "emu_dgemm": (_i32, [_vp, _i32, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl, _vp, _i64, _i32,
                         _i32, _vp]),
    "emu_dgemm_host": (_i32, [_vp, _i32, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl, _vp, _i64, _i32,
                              _i32, _vp]),
    "emu_sgemm": (_i32, [_vp, _i32, _i64, _i64, _i64, _flt, _vp, _i64, _vp, _i64, _flt, _vp, _i64, _i32,
                         _i32, _vp]),
    "emu_zgemm": (_i32, [_vp, _i32, _i64, _i64, _i64, _vp, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _i32, _i32,
                         _vp]),
    "emu_cgemm": (_i32, [_vp, _i32, _i64, _i64, _i64, _vp, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _i32, _i32,
                         _vp]),
    "emu_shift_reduce_I": (_i32, [_vp, _i64, _i64, _i32, _i32, _vp, _vp, _vp, _dbl, _dbl, _vp, _i64, _vp]),
    "emu_split_rows": (_i64, [_i64]),
    "emu_split_cols_I": (_i64, [_i64, _i32]),
    "emu_split_cols_II": (_i64, [_i64]),
    "emu_split_I": (_i32, [_vp, _i32, _i32, _i64, _i64, _vp, _i64, _i32, _vp, _vp, _vp]),
    "emu_split_F8": (_i32, [_vp, _i32, _i32, _i64, _i64, _vp, _i64, _i32, _vp, _vp, _vp]),
    "emu_split_II": (_i32, [_vp, _i32, _i32, _i64, _i64, _i64, _vp, _i64, _i32, _vp, _vp, _vp]),
    "emu_partials_I": (_i32, [_vp, _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _vp]),
    "emu_residues_II": (_i32, [_vp, _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _vp]),
    "emu_chunk_len_I": (_i64, [_i32]),
    "emu_chunk_len_F8": (_i64, [_i32]),
    "emu_partials_F8": (_i32, [_vp, _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _vp]),
    "emu_moduli": (_i32, [_i32, _vp]),
    "emu_scale_bits_II": (_i32, [_i32, _i64, _i32]),
    "emu_dgemm_noalloc": (_i32, [_i32, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl, _vp, _i64, _i32, _vp,
                                 _vp]),
    "emu_dgemm_grouped": (_i32, [_vp, _i32, ctypes.POINTER(GemmDesc), _i32, _vp]),
    "emu_dgemm_grouped_loop": (_i32, [_vp, _i32, ctypes.POINTER(GemmDesc), _i32, _vp]),
    "emu_tune_grouped": (_i32, [_vp, _i32, ctypes.POINTER(GemmDesc), _i32, ctypes.c_char_p, ctypes.POINTER(_i32),
                                _vp]),
    "emu_load_tuning": (_i32, [_vp, ctypes.c_char_p]),
    "emu_sel_features": (_i32, [_vp, _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _dbl, _i64, _vp, _vp]),
    "emu_sel_forward": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    "emu_sel_backward": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "emu_sel_adam": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _flt, _flt, _flt, _flt, _vp]),
    "emu_sel_load": (_i32, [_vp, ctypes.POINTER(_flt)]),
    "emu_probe_dd": (_i32, [_vp, _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _vp, _vp, _vp]),
    "emu_dgemm_auto": (_i32, [_vp, _i32, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _vp, _i64, _dbl, _i32,
                              ctypes.POINTER(_i32), _vp]),
    "emu_bound_p": (_i32, [_vp, _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _dbl, ctypes.POINTER(_i32), _vp]),
    "emu_sel_load_II": (_i32, [_vp, ctypes.POINTER(_flt)]),
    "emu_dgemm_auto_II": (_i32, [_vp, _i32, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _vp, _i64, _dbl, _i32,
                                 ctypes.POINTER(_i32), _vp]),
    "emu_bound_nm": (_i32, [_vp, _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _dbl, ctypes.POINTER(_i32), _vp]),
    "emu_trace_enable": (_i32, [_vp, _i32]),
    "emu_trace_read": (_i32, [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


def check(code: int, where: str = "") -> None:
    if code != 0:
        if code == 4:  # EMU_ERR_CUDA: name the runtime error
            where = "%s (%s)" % (where, emu_last_cuda_error().decode())
        raise EmuError(code, where)


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else stream


class Handle:
    """Owns an emu_handle_t bound to one CUDA device."""

    def __init__(self, device: int = 0):
        h = _vp()
        check(emu_create(ctypes.byref(h), device), "emu_create")
        self.h = h
        self.device = device

    def close(self) -> None:
        if self.h:
            emu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None) -> int:
        return int(emu_get_status(self.h, _stream_ptr(stream)))

    def trace(self, enable: bool = True) -> None:
        check(emu_trace_enable(self.h, int(enable)), "emu_trace_enable")

    def trace_read(self) -> dict:
        ms = (_dbl * 4)()
        g, k = _i64(), _i64()
        check(emu_trace_read(self.h, ms, ctypes.byref(g), ctypes.byref(k)), "emu_trace_read")
        return {"ms_scan": ms[0], "ms_split": ms[1], "ms_gemm": ms[2], "ms_other": ms[3],
                "gemm_launches": g.value, "kernel_launches": k.value}


_default = {}


def default_handle(device: int = 0) -> Handle:
    if device not in _default:
        _default[device] = Handle(device)
    return _default[device]


def _scheme(s) -> int:
    if s in (1, "I", "i", EMU_SCHEME_I):
        return EMU_SCHEME_I
    if s in (2, "II", "ii", EMU_SCHEME_II):
        return EMU_SCHEME_II
    if s in (3, "I_F8", "F8", "f8", EMU_SCHEME_I_F8):
        return EMU_SCHEME_I_F8
    if s in (4, "II_NORM", "II_N", "ii_norm", EMU_SCHEME_II_NORM):
        return EMU_SCHEME_II_NORM
    raise ValueError("scheme must be 'I', 'II', 'I_F8' or 'II_NORM'")


def _layout_of(A, B, C):
    """Row-major if all three are C-contiguous, column-major if all are Fortran-ordered."""
    def rowmaj(t):
        return t.dim() == 2 and (t.stride(1) == 1 or t.size(1) <= 1)

    def colmaj(t):
        return t.dim() == 2 and (t.stride(0) == 1 or t.size(0) <= 1)

    if all(rowmaj(t) for t in (A, B, C)):
        ld = lambda t: max(t.stride(0), t.size(1), 1)
        return EMU_ROW_MAJOR, ld(A), ld(B), ld(C)
    if all(colmaj(t) for t in (A, B, C)):
        ld = lambda t: max(t.stride(1), t.size(0), 1)
        return EMU_COL_MAJOR, ld(A), ld(B), ld(C)
    raise ValueError("A, B and C must all be row-major or all column-major")


def dgemm(A, B, C=None, alpha: float = 1.0, beta: float = 0.0, scheme="I", p: int = 7, handle=None,
          stream=None):
    """C = alpha*A@B + beta*C for float64 CUDA tensors through emu_dgemm."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    if C is None:
        C = torch.empty((m, n), dtype=torch.float64, device=A.device)
        beta = 0.0
    layout, lda, ldb, ldc = _layout_of(A, B, C)
    h = handle or default_handle(A.device.index or 0)
    check(emu_dgemm(h.h, layout, m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta, _ptr(C), ldc,
                    _scheme(scheme), p, _stream_ptr(stream)), "emu_dgemm")
    return C


def dgemm_host(A, B, C=None, alpha: float = 1.0, beta: float = 0.0, scheme="I", p: int = 7, handle=None,
               stream=None):
    """C = alpha*A@B + beta*C for float64 host matrices (numpy arrays or CPU
    tensors; pinned CPU tensors let the copies overlap the computation)
    through emu_dgemm_host; all three row-major (C-contiguous rows with any
    leading dimension) or all column-major.  Returns C (a new numpy array if
    C is None)."""
    import numpy as np

    def lay(x):
        """(strides in elements, data pointer, number of elements)"""
        if isinstance(x, np.ndarray):
            return [v // x.itemsize for v in x.strides], x.ctypes.data, x.size
        return list(x.stride()), x.data_ptr(), x.numel()

    m, k = A.shape
    n = B.shape[1]
    if C is None:
        C = np.empty((m, n), dtype=np.float64)
        beta = 0.0
    ops = [(lay(t), t.shape) for t in (A, B, C)]
    pa, pb, pc = (o[0][1] for o in ops)
    # an empty matrix fits either layout (its strides are arbitrary)
    if all(st[1] == 1 or sh[1] <= 1 or sz == 0 for (st, _, sz), sh in ops):
        layout = EMU_ROW_MAJOR
        lds = [max(st[0] if sz else 0, sh[1], 1) for (st, _, sz), sh in ops]
    elif all(st[0] == 1 or sh[0] <= 1 or sz == 0 for (st, _, sz), sh in ops):
        layout = EMU_COL_MAJOR
        lds = [max(st[1] if sz else 0, sh[0], 1) for (st, _, sz), sh in ops]
    else:
        raise ValueError("A, B and C must all be row-major or all column-major")
    h = handle or default_handle(0)
    check(emu_dgemm_host(h.h, layout, m, n, k, alpha, pa, lds[0], pb, lds[1], beta, pc, lds[2], _scheme(scheme), p,
                         _stream_ptr(stream)), "emu_dgemm_host")
    return C


def sgemm(A, B, C=None, alpha: float = 1.0, beta: float = 0.0, scheme="I", p: int = 4, handle=None,
          stream=None):
    """C = alpha*A@B + beta*C for float32 CUDA tensors through emu_sgemm."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    if C is None:
        C = torch.empty((m, n), dtype=torch.float32, device=A.device)
        beta = 0.0
    layout, lda, ldb, ldc = _layout_of(A, B, C)
    h = handle or default_handle(A.device.index or 0)
    check(emu_sgemm(h.h, layout, m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta, _ptr(C), ldc,
                    _scheme(scheme), p, _stream_ptr(stream)), "emu_sgemm")
    return C


def zgemm(A, B, C=None, alpha: complex = 1.0, beta: complex = 0.0, nm: int = 16, handle=None, stream=None,
          scheme="II", p: int | None = None):
    """complex128 C = alpha*A@B + beta*C through emu_zgemm: Scheme II 3M with
    nm moduli (default), or scheme="I" / "I_F8" (4M) with p slices."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    if C is None:
        C = torch.empty((m, n), dtype=torch.complex128, device=A.device)
        beta = 0.0
    layout, lda, ldb, ldc = _layout_of(A, B, C)
    al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
    h = handle or default_handle(A.device.index or 0)
    sc = _scheme(scheme)
    check(emu_zgemm(h.h, layout, m, n, k, al, _ptr(A), lda, _ptr(B), ldb, be, _ptr(C), ldc, sc,
                    nm if sc in (EMU_SCHEME_II, EMU_SCHEME_II_NORM) else p, _stream_ptr(stream)), "emu_zgemm")
    return C


def cgemm(A, B, C=None, alpha: complex = 1.0, beta: complex = 0.0, p: int = 4, scheme="I", handle=None,
          stream=None):
    """complex64 C = alpha*A@B + beta*C through emu_cgemm: Scheme I / I_F8
    (4M, p slices) or Scheme II (3M, p = number of moduli)."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    if C is None:
        C = torch.empty((m, n), dtype=torch.complex64, device=A.device)
        beta = 0.0
    layout, lda, ldb, ldc = _layout_of(A, B, C)
    al = (ctypes.c_float * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_float * 2)(complex(beta).real, complex(beta).imag)
    h = handle or default_handle(A.device.index or 0)
    check(emu_cgemm(h.h, layout, m, n, k, al, _ptr(A), lda, _ptr(B), ldb, be, _ptr(C), ldc, _scheme(scheme), p,
                    _stream_ptr(stream)), "emu_cgemm")
    return C


def shift_reduce_I(Cs, EA, FB, p: int, f8: bool = False, C=None, alpha: float = 1.0, beta: float = 0.0,
                   handle=None, stream=None):
    """Unfused Scheme I epilogue (Eq. 3) on p x m x n int32 partials Cs with
    row exponents EA (int32, m) and column exponents FB (int32, n)."""
    import torch
    _, m, n = Cs.shape
    if C is None:
        C = torch.empty((m, n), dtype=torch.float64, device=Cs.device)
        beta = 0.0
    h = handle or default_handle(Cs.device.index or 0)
    check(emu_shift_reduce_I(h.h, m, n, p, int(f8), _ptr(Cs), _ptr(EA), _ptr(FB), alpha, beta, _ptr(C),
                             max(C.stride(0), n, 1), _stream_ptr(stream)), "emu_shift_reduce_I")
    return C


def moduli(nm: int) -> list[int]:
    out = (ctypes.c_int32 * max(nm, 1))()
    got = emu_moduli(nm, out)
    return [int(out[i]) for i in range(got)]


def split_I(X, p: int, operand: int = 0, handle=None, stream=None, f8: bool = False):
    """Scheme I split of A's rows (operand 0, X is m x k) or B's columns
    (operand 1, X is k x n); returns (hat int8 tensor, exponents int32).
    f8=True: E4M3 slices (emu_split_F8)."""
    import torch
    if operand == 0:
        rows, k = X.shape
    else:
        k, rows = X.shape
    layout = EMU_ROW_MAJOR if X.stride(1) == 1 else EMU_COL_MAJOR
    ldx = X.stride(0) if layout == EMU_ROW_MAJOR else X.stride(1)
    hat = torch.empty((emu_split_rows(rows), emu_split_cols_I(k, p)), dtype=torch.int8, device=X.device)
    E = torch.empty((max(rows, 1),), dtype=torch.int32, device=X.device)
    h = handle or default_handle(X.device.index or 0)
    fn = emu_split_F8 if f8 else emu_split_I
    check(fn(h.h, layout, operand, rows, k, _ptr(X), max(ldx, 1), p, _ptr(hat), _ptr(E), _stream_ptr(stream)),
          fn.__name__)
    return hat, E[:rows]


def split_II(X, nm: int, k_total: int | None = None, operand: int = 0, handle=None, stream=None):
    """Scheme II residues of A's rows / B's columns: (res int8 [nm, rows_pad, kpad], E)."""
    import torch
    if operand == 0:
        rows, k = X.shape
    else:
        k, rows = X.shape
    layout = EMU_ROW_MAJOR if X.stride(1) == 1 else EMU_COL_MAJOR
    ldx = X.stride(0) if layout == EMU_ROW_MAJOR else X.stride(1)
    res = torch.empty((nm, emu_split_rows(rows), emu_split_cols_II(k)), dtype=torch.int8, device=X.device)
    E = torch.empty((max(rows, 1),), dtype=torch.int32, device=X.device)
    h = handle or default_handle(X.device.index or 0)
    check(emu_split_II(h.h, layout, operand, rows, k, k if k_total is None else k_total, _ptr(X),
                       max(ldx, 1), nm, _ptr(res), _ptr(E), _stream_ptr(stream)), "emu_split_II")
    return res, E[:rows]


def partials_I(A, B, p: int, handle=None, stream=None, f8: bool = False):
    """Unfused Scheme I: int32 tensor [p, m, n] of the exact partials C_s
    (f8=True: the E4M3 engine's FP32 accumulators, converted exactly)."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    out = torch.empty((p, m, n), dtype=torch.int32, device=A.device)
    h = handle or default_handle(A.device.index or 0)
    fn = emu_partials_F8 if f8 else emu_partials_I
    check(fn(h.h, EMU_ROW_MAJOR, m, n, k, _ptr(A), A.stride(0), _ptr(B), B.stride(0), p, _ptr(out),
             _stream_ptr(stream)), fn.__name__)
    return out


def residues_II(A, B, nm: int, handle=None, stream=None):
    """Paper-design Scheme II output: uint8 tensor [nm, m, n] of per-modulus residues."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    out = torch.empty((nm, m, n), dtype=torch.uint8, device=A.device)
    h = handle or default_handle(A.device.index or 0)
    check(emu_residues_II(h.h, EMU_ROW_MAJOR, m, n, k, _ptr(A), A.stride(0), _ptr(B), B.stride(0), nm,
                          _ptr(out), _stream_ptr(stream)), "emu_residues_II")
    return out


def grouped_descs(As, Bs, Cs, alphas=None, betas=None):
    """Array of GemmDesc for lists of row-major float64 CUDA tensors."""
    cnt = len(As)
    arr = (GemmDesc * cnt)()
    for i, (A, B, C) in enumerate(zip(As, Bs, Cs)):
        m, k = A.shape
        n = B.shape[1]
        arr[i] = GemmDesc(m, n, k, 1.0 if alphas is None else alphas[i], 0.0 if betas is None else betas[i],
                          A.data_ptr(), max(A.stride(0), k, 1), B.data_ptr(), max(B.stride(0), n, 1), C.data_ptr(),
                          max(C.stride(0), n, 1))
    return arr


def dgemm_grouped(descs, p: int = 6, handle=None, stream=None, loop: bool = False):
    """Run emu_dgemm_grouped (one graph-captured persistent launch) or, with
    loop=True, emu_dgemm_grouped_loop (one emu_dgemm per product)."""
    h = handle or default_handle(0)
    fn = emu_dgemm_grouped_loop if loop else emu_dgemm_grouped
    check(fn(h.h, len(descs), descs, p, _stream_ptr(stream)), fn.__name__)


def tune_grouped(descs, p: int = 6, path: str | None = None, handle=None, stream=None) -> int:
    h = handle or default_handle(0)
    timed = _i32()
    check(emu_tune_grouped(h.h, len(descs), descs, p, None if path is None else path.encode(), ctypes.byref(timed),
                           _stream_ptr(stream)), "emu_tune_grouped")
    return timed.value


def dgemm_auto(A, B, tol: float, alpha: float = 1.0, probe: int = 64, handle=None, stream=None, scheme="I",
               C=None):
    """C = alpha*A@B with the p (scheme="I") or the N moduli (scheme="II":
    Scheme II with norm scaling) chosen by the selector -- the bound if no
    weights are loaded -- checked on `probe` sampled entries; returns
    (C, p or N, status code).  C: optional output tensor (allocated if None)."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    if C is None:
        C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    layout, lda, ldb, ldc = _layout_of(A, B, C)
    h = handle or default_handle(A.device.index or 0)
    p = _i32()
    fn = emu_dgemm_auto_II if scheme in ("II", "II_NORM", 2, 4) else emu_dgemm_auto
    code = fn(h.h, layout, m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, tol, probe, ctypes.byref(p),
              _stream_ptr(stream))
    if code not in (0, 7):
        check(code, fn.__name__)
    return C, p.value, code
