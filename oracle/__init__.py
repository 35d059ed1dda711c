"""CPU oracle for the emulated-GEMM hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product (``paper_2606_25453_gb300``) never imports it, and the two share no
code: this wrapper only marshals numpy arrays into the plain-C oracle in
``emu_oracle.c`` (built with gcc, ``-ffp-contract=off``, OpenMP).

Conventions: matrices are numpy float64 (complex: complex128), row-major, and
the functions take ``A`` (m x k) and ``B`` (k x n) as mathematical matrices;
the wrapper passes ``B.T`` to the C code, whose column operand is stored as
rows.  Paper references: Scheme I -- Sec. II-C-1, Eqs. (1)-(3), (11);
Scheme II -- Sec. II-C-2, Eqs. (4)-(8); 3M -- Sec. IV-B, Eq. (16); Scheme I
on FP8 (E4M3) slices -- the FP8 formulation Sec. VII names as future work,
on the layout of Sec. III-A (reading R7 in emu_oracle.c).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(exact rationals / Python big integers / closed forms); none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emu_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lib = None
_lock = threading.Lock()
# gcc flags of the oracle library (no implicit FMA contraction, no fast math)
CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liborc.so (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc"] + CFLAGS + ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            vp = ctypes.c_void_p
            sig = {
                "orc_num_threads": (i32, []),
                "orc_row_exponents": (i64, [i64, i64, vp, vp]),
                "orc_row_exponents_z": (i64, [i64, i64, vp, vp]),
                "orc_split_I": (None, [i64, i64, vp, vp, i32, vp]),
                "orc_interleave": (None, [i64, i64, i32, i32, vp, vp]),
                "orc_chunk_len_I": (i64, [i32]),
                "orc_partials_I": (None, [i64, i64, i64, i32, i64, vp, vp, vp]),
                "orc_emu_I": (i32, [i64, i64, i64, i32, dbl, vp, vp, dbl, vp, vp, i32]),
                "orc_moduli": (i32, [i32, vp]),
                "orc_log2P_floor": (i32, [i32]),
                "orc_scale_bits_II": (i32, [i32, i64, i32]),
                "orc_residues_II": (None, [i64, i64, vp, vp, i32, i32, i32, i32, vp]),
                "orc_modprod_II": (None, [i64, i64, i64, i32, vp, vp, vp]),
                "orc_crt": (i32, [i32, i64, vp, vp]),
                "orc_emu_II": (i32, [i64, i64, i64, i32, dbl, vp, vp, dbl, vp, vp, i32]),
                "orc_emu_II_ex": (i32, [i64, i64, i64, i32, i32, dbl, vp, vp, dbl, vp, vp, i32]),
                "orc_norm_exponents": (i64, [i64, i64, i32, vp, vp]),
                "orc_norm_halves_II": (None, [i32, vp, vp]),
                "orc_emu_Z3M_norm": (i32, [i64, i64, i64, i32, dbl, dbl, vp, vp, dbl, dbl, vp, vp, i32]),
                "orc_modprod_Z3M": (None, [i64, i64, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
                "orc_emu_Z3M": (i32, [i64, i64, i64, i32, dbl, dbl, vp, vp, dbl, dbl, vp]),
                "orc_emu_C3M": (i32, [i64, i64, i64, i32, dbl, dbl, vp, vp, dbl, dbl, vp]),
                "orc_split_F8": (None, [i64, i64, vp, vp, i32, vp]),
                "orc_chunk_len_F8": (i64, [i32]),
                "orc_emu_F8": (i32, [i64, i64, i64, i32, dbl, vp, vp, dbl, vp, vp, i32]),
                "orc_emu_Z4M_I": (i32, [i64, i64, i64, i32, i32, dbl, dbl, vp, vp, dbl, dbl, vp, vp, i32]),
                "orc_dd_gemm": (None, [i64, i64, i64, vp, vp, vp, vp]),
                "orc_dd_zgemm": (None, [i64, i64, i64, vp, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ---------------------------------------------------------------- scaling
def row_exponents(X) -> np.ndarray:
    """E_i = frexp exponent of max_h |x_ih| (0 for a zero row); Eq. (1) mu."""
    X = _f64(X)
    E = np.zeros(X.shape[0], dtype=np.int32)
    bad = _load().orc_row_exponents(X.shape[0], X.shape[1], _p(X), _p(E))
    if bad:
        raise ValueError("non-finite input")
    return E


def col_exponents(B) -> np.ndarray:
    """F_j for the columns of B (Eq. 1, nu)."""
    return row_exponents(np.ascontiguousarray(np.asarray(B, dtype=np.float64).T))


def row_exponents_z(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.complex128)
    E = np.zeros(X.shape[0], dtype=np.int32)
    bad = _load().orc_row_exponents_z(X.shape[0], X.shape[1], _p(X), _p(E))
    if bad:
        raise ValueError("non-finite input")
    return E


# ---------------------------------------------------------------- Scheme I
def chunk_len_I(p: int) -> int:
    """K_c: the K-chunk over which the INT32 accumulators of Eq. (2) stay exact."""
    return int(_load().orc_chunk_len_I(p))


def split_I_rows(X, p: int, E=None) -> np.ndarray:
    """Slices of the rows of X (Eq. 1): int16 array [p, rows, k]."""
    X = _f64(X)
    if E is None:
        E = row_exponents(X)
    E = np.ascontiguousarray(E, dtype=np.int32)
    D = np.zeros((p,) + X.shape, dtype=np.int16)
    _load().orc_split_I(X.shape[0], X.shape[1], _p(X), _p(E), p, _p(D))
    return D


def interleave(D: np.ndarray, tk: int = 32) -> np.ndarray:
    """Eq. (11) layout of slices D [p, rows, k] -> int8 [rows, ceil(k/tk)*tk*p]."""
    D = np.ascontiguousarray(D, dtype=np.int16)
    p, rows, k = D.shape
    nck = -(-k // tk)
    out = np.zeros((rows, nck * tk * p), dtype=np.int8)
    _load().orc_interleave(rows, k, p, tk, _p(D), _p(out))
    return out


def partials_I(A, B, p: int, kc: int | None = None) -> np.ndarray:
    """Exact chunked partials of Eq. (2): int64 [nchunks, p, m, n]."""
    A, Bt = _f64(A), _f64(np.asarray(B).T)
    m, k = A.shape
    n = Bt.shape[0]
    kc = chunk_len_I(p) if kc is None else kc
    DA = split_I_rows(A, p)
    DB = split_I_rows(Bt, p)
    nch = -(-k // kc) if k else 0
    out = np.zeros((nch, p, m, n), dtype=np.int64)
    _load().orc_partials_I(m, n, k, p, kc, _p(DA), _p(DB), _p(out))
    return out


def emu_I(A, B, p: int, alpha: float = 1.0, beta: float = 0.0, C=None, out_f32: bool = False) -> np.ndarray:
    """Scheme I emulated C = alpha*A@B + beta*C (Eqs. 1-3, exact shift-reduce)."""
    A, Bt = _f64(A), _f64(np.asarray(B).T)
    m, k = A.shape
    n = Bt.shape[0]
    if out_f32:
        Cf = np.zeros((m, n), dtype=np.float32) if C is None else np.array(C, dtype=np.float32, order="C")
        Cd = np.zeros(1)
    else:
        Cd = np.zeros((m, n)) if C is None else np.array(C, dtype=np.float64, order="C")
        Cf = np.zeros(1, dtype=np.float32)
    rc = _load().orc_emu_I(m, n, k, p, float(alpha), _p(A), _p(Bt), float(beta), _p(Cd), _p(Cf),
                           int(out_f32))
    if rc:
        raise ValueError("non-finite input")
    return Cf if out_f32 else Cd


# ---------------------------------------------------------------- Scheme I, FP8 slices
def chunk_len_F8(p: int) -> int:
    """K_c over which FP32 accumulation of E4M3 slice products stays exact."""
    return int(_load().orc_chunk_len_F8(p))


def split_F8_rows(X, p: int, E=None) -> np.ndarray:
    """Balanced base-32 digits of the rows of X (reading R7): int16 [p, rows, k]."""
    X = _f64(X)
    if E is None:
        E = row_exponents(X)
    E = np.ascontiguousarray(E, dtype=np.int32)
    D = np.zeros((p,) + X.shape, dtype=np.int16)
    _load().orc_split_F8(X.shape[0], X.shape[1], _p(X), _p(E), p, _p(D))
    return D


def partials_F8(A, B, p: int, kc: int | None = None) -> np.ndarray:
    """Exact chunked triangle partials of the E4M3 digits: int64 [nchunks, p, m, n]."""
    A, Bt = _f64(A), _f64(np.asarray(B).T)
    m, k = A.shape
    n = Bt.shape[0]
    kc = chunk_len_F8(p) if kc is None else kc
    DA = split_F8_rows(A, p)
    DB = split_F8_rows(Bt, p)
    nch = -(-k // kc) if k else 0
    out = np.zeros((nch, p, m, n), dtype=np.int64)
    _load().orc_partials_I(m, n, k, p, kc, _p(DA), _p(DB), _p(out))
    return out


def emu_F8(A, B, p: int, alpha: float = 1.0, beta: float = 0.0, C=None, out_f32: bool = False) -> np.ndarray:
    """Scheme I with E4M3 slices (beta = 5): C = alpha*A@B + beta*C."""
    A, Bt = _f64(A), _f64(np.asarray(B).T)
    m, k = A.shape
    n = Bt.shape[0]
    if out_f32:
        Cf = np.zeros((m, n), dtype=np.float32) if C is None else np.array(C, dtype=np.float32, order="C")
        Cd = np.zeros(1)
    else:
        Cd = np.zeros((m, n)) if C is None else np.array(C, dtype=np.float64, order="C")
        Cf = np.zeros(1, dtype=np.float32)
    rc = _load().orc_emu_F8(m, n, k, p, float(alpha), _p(A), _p(Bt), float(beta), _p(Cd), _p(Cf), int(out_f32))
    if rc:
        raise ValueError("non-finite input")
    return Cf if out_f32 else Cd


# ---------------------------------------------------------------- Scheme II
def moduli(nm: int) -> list[int]:
    """First nm of the greedy descending pairwise-coprime list 256, 255, 253, ..."""
    out = np.zeros(max(nm, 1), dtype=np.int32)
    got = _load().orc_moduli(nm, _p(out))
    return [int(x) for x in out[:got]]


def log2P_floor(nm: int) -> int:
    return int(_load().orc_log2P_floor(nm))


def scale_bits_II(nm: int, k: int, is_complex: bool = False) -> int:
    return int(_load().orc_scale_bits_II(nm, k, int(is_complex)))


def residues_II_rows(X, nm: int, b: int, E=None) -> np.ndarray:
    """Symmetric residues of trunc(x * 2^(b-E_i)) (Eq. 5): int8 [nm, rows, k]."""
    X = _f64(X)
    if E is None:
        E = row_exponents(X)
    E = np.ascontiguousarray(E, dtype=np.int32)
    R = np.zeros((nm,) + X.shape, dtype=np.int8)
    _load().orc_residues_II(X.shape[0], X.shape[1], _p(X), _p(E), b, nm, 0, 0, _p(R))
    return R


def residues_Z_rows(X, nm: int, b: int, part: int, E=None) -> np.ndarray:
    """Complex residues: part 0 = re, 1 = im, 2 = re+im (3M sum). int8 [nm, rows, k]."""
    X = np.ascontiguousarray(X, dtype=np.complex128)
    if E is None:
        E = row_exponents_z(X)
    E = np.ascontiguousarray(E, dtype=np.int32)
    R = np.zeros((nm,) + X.shape, dtype=np.int8)
    _load().orc_residues_II(X.shape[0], X.shape[1], _p(X), _p(E), b, nm, 1, part, _p(R))
    return R


def modprod_II(RA: np.ndarray, RBt: np.ndarray) -> np.ndarray:
    """Eqs. (6)-(7): uint8 [nm, m, n] residues of the per-modulus products."""
    RA = np.ascontiguousarray(RA, dtype=np.int8)
    RBt = np.ascontiguousarray(RBt, dtype=np.int8)
    nm, m, k = RA.shape
    n = RBt.shape[1]
    out = np.zeros((nm, m, n), dtype=np.uint8)
    _load().orc_modprod_II(m, n, k, nm, _p(RA), _p(RBt), _p(out))
    return out


def crt(res: np.ndarray) -> np.ndarray:
    """Eq. (8) + reading R5: residues uint8 [nm, cnt] -> float64 [cnt]."""
    res = np.ascontiguousarray(res, dtype=np.uint8)
    nm, cnt = res.shape
    out = np.zeros(cnt)
    _load().orc_crt(nm, cnt, _p(res), _p(out))
    return out


def norm_exponents(X, complex_: bool = False) -> np.ndarray:
    """Reading R9: e per row with ||x_row||_2 < 2^e, computed exactly."""
    if complex_:
        Xc = np.ascontiguousarray(X, dtype=np.complex128)
        rows, cols = Xc.shape
        buf = Xc.view(np.float64)
    else:
        buf = _f64(X)
        rows, cols = buf.shape
    E = np.zeros(max(rows, 1), dtype=np.int32)
    if _load().orc_norm_exponents(rows, cols, 2 if complex_ else 1, _p(buf), _p(E)):
        raise ValueError("non-finite input")
    return E[:rows]


def norm_halves_II(nm: int) -> tuple[int, int]:
    a, b = ctypes.c_int(), ctypes.c_int()
    _load().orc_norm_halves_II(nm, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def emu_II(A, B, nm: int, alpha: float = 1.0, beta: float = 0.0, C=None, out_f32: bool = False,
           norm: bool = False):
    """Scheme II emulated C = alpha*A@B + beta*C (Eqs. 5-8); norm=True: the
    norm-based scaling of reading R9 instead of R3."""
    A, Bt = _f64(A), _f64(np.asarray(B).T)
    m, k = A.shape
    n = Bt.shape[0]
    if out_f32:
        Cf = np.zeros((m, n), dtype=np.float32) if C is None else np.array(C, dtype=np.float32, order="C")
        Cd = np.zeros(1)
    else:
        Cd = np.zeros((m, n)) if C is None else np.array(C, dtype=np.float64, order="C")
        Cf = np.zeros(1, dtype=np.float32)
    rc = _load().orc_emu_II_ex(m, n, k, nm, int(norm), float(alpha), _p(A), _p(Bt), float(beta), _p(Cd),
                               _p(Cf), int(out_f32))
    if rc:
        raise ValueError("non-finite input")
    return Cf if out_f32 else Cd


def modprod_Z3M(A3, B3t):
    """Eq. (16) per modulus: A3/B3t = (re, im, sum) residue sets -> (Re, Im) uint8."""
    A3 = [np.ascontiguousarray(x, dtype=np.int8) for x in A3]
    B3t = [np.ascontiguousarray(x, dtype=np.int8) for x in B3t]
    nm, m, k = A3[0].shape
    n = B3t[0].shape[1]
    ore = np.zeros((nm, m, n), dtype=np.uint8)
    oim = np.zeros((nm, m, n), dtype=np.uint8)
    _load().orc_modprod_Z3M(m, n, k, nm, *[_p(x) for x in A3], *[_p(x) for x in B3t], _p(ore), _p(oim))
    return ore, oim


def emu_Z3M(A, B, nm: int, alpha: complex = 1.0, beta: complex = 0.0, C=None, out_f32: bool = False,
            norm: bool = False) -> np.ndarray:
    """Scheme II 3M complex C = alpha*A@B + beta*C (Eqs. 5-8, 16).  out_f32:
    complex64 result (CGEMM; the inputs are used as given, widened exactly)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    Bt = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).T)
    m, k = A.shape
    n = Bt.shape[0]
    alpha, beta = complex(alpha), complex(beta)
    if norm:
        if out_f32:
            out = np.zeros((m, n), dtype=np.complex64) if C is None else np.array(C, dtype=np.complex64, order="C")
            Cz = np.zeros((1, 1), dtype=np.complex128)
            Cf = out
        else:
            out = np.zeros((m, n), dtype=np.complex128) if C is None else np.array(C, dtype=np.complex128, order="C")
            Cz = out
            Cf = np.zeros((1, 1), dtype=np.complex64)
        rc = _load().orc_emu_Z3M_norm(m, n, k, nm, alpha.real, alpha.imag, _p(A), _p(Bt), beta.real, beta.imag,
                                      _p(Cz), _p(Cf), int(out_f32))
    elif out_f32:
        Cf = np.zeros((m, n), dtype=np.complex64) if C is None else np.array(C, dtype=np.complex64, order="C")
        rc = _load().orc_emu_C3M(m, n, k, nm, alpha.real, alpha.imag, _p(A), _p(Bt), beta.real, beta.imag,
                                 _p(Cf))
        out = Cf
    else:
        Cz = np.zeros((m, n), dtype=np.complex128) if C is None else np.array(C, dtype=np.complex128, order="C")
        rc = _load().orc_emu_Z3M(m, n, k, nm, alpha.real, alpha.imag, _p(A), _p(Bt), beta.real, beta.imag,
                                 _p(Cz))
        out = Cz
    if rc:
        raise ValueError("non-finite input")
    return out


def emu_Z4M_I(A, B, p: int, f8: bool = False, alpha: complex = 1.0, beta: complex = 0.0, C=None,
              out_f32: bool = False) -> np.ndarray:
    """Scheme I complex (4M, reading R8) C = alpha*A@B + beta*C with INT8
    (f8=False) or E4M3 (f8=True) slices.  out_f32: complex64 result (CGEMM)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    Bt = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).T)
    m, k = A.shape
    n = Bt.shape[0]
    alpha, beta = complex(alpha), complex(beta)
    if out_f32:
        Cf = np.zeros((m, n), dtype=np.complex64) if C is None else np.array(C, dtype=np.complex64, order="C")
        Cz = np.zeros((1, 1), dtype=np.complex128)
    else:
        Cz = np.zeros((m, n), dtype=np.complex128) if C is None else np.array(C, dtype=np.complex128, order="C")
        Cf = np.zeros((1, 1), dtype=np.complex64)
    rc = _load().orc_emu_Z4M_I(m, n, k, p, int(f8), alpha.real, alpha.imag, _p(A), _p(Bt), beta.real, beta.imag,
                               _p(Cz), _p(Cf), int(out_f32))
    if rc:
        raise ValueError("non-finite input")
    return Cf if out_f32 else Cz


# ---------------------------------------------------------------- reference
def dd_gemm(A, B):
    """Double-double reference product: (hi, lo) float64 arrays."""
    A, Bt = _f64(A), _f64(np.asarray(B).T)
    m, k = A.shape
    n = Bt.shape[0]
    hi = np.zeros((m, n))
    lo = np.zeros((m, n))
    _load().orc_dd_gemm(m, n, k, _p(A), _p(Bt), _p(hi), _p(lo))
    return hi, lo


def dd_zgemm(A, B):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    Bt = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).T)
    m, k = A.shape
    n = Bt.shape[0]
    hi = np.zeros((m, n), dtype=np.complex128)
    lo = np.zeros((m, n), dtype=np.complex128)
    _load().orc_dd_zgemm(m, n, k, _p(A), _p(Bt), _p(hi), _p(lo))
    return hi, lo


def err_metric(C, ref, A, B) -> float:
    """max_ij |C - Cref|_ij / (|A||B|)_ij, |C-Cref| evaluated as |(C-hi)-lo|.

    For complex inputs the modulus of the complex difference is used and the
    denominator is (|A||B|) with elementwise complex moduli.
    """
    hi, lo = ref
    C = np.asarray(C)
    if np.iscomplexobj(C) or np.iscomplexobj(hi):
        d = np.abs((C.astype(np.complex128) - hi) - lo)
    else:
        d = np.abs((C.astype(np.float64) - hi) - lo)
    den = np.abs(np.asarray(A)) @ np.abs(np.asarray(B))
    mask = den > 0
    if not np.any(mask):
        return float(np.max(d)) if d.size else 0.0
    bad = (~mask) & (d > 0)
    if np.any(bad):
        return float("inf")
    return float(np.max(d[mask] / den[mask]))
