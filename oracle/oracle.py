"""numpy front end of the C oracle (test infrastructure only).

Every function takes and returns host numpy arrays.  A compressed matrix is
the structure of arrays of Sec. II: ``f`` (float64 [nb]), ``s`` (float64
[nb]), ``phi`` (uint8 [nb]) and ``code`` (int8 [nb, 28]), blocks in row-major
order over the (rows/8) x (cols/8) block grid.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "blaz_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libblaz_oracle.so")

# No FMA contraction (GCC contracts by default on aarch64), no fast-math.
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC"]

NKEEP = 28


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I8 = ctypes.POINTER(ctypes.c_int8)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64


class Stages(ctypes.Structure):
    """Intermediate stages of compressing one block (Sec. II, Ex. 1-5)."""

    _fields_ = [
        ("delta", ctypes.c_double * 64),
        ("K", ctypes.c_int32),
        ("sum_abs", ctypes.c_double),
        ("s", ctypes.c_double),
        ("dprime", ctypes.c_double * 64),
        ("s_max", ctypes.c_double),
        ("psi", ctypes.c_uint8 * 64),
        ("dct", ctypes.c_double * 64),
        ("m", ctypes.c_double),
        ("phi", ctypes.c_uint8),
        ("f", ctypes.c_double),
        ("code", ctypes.c_int8 * NKEEP),
    ]


def _declare(L):
    L.blazo_dct_tables.argtypes = [_D, _D]
    L.blazo_kept_positions.argtypes = [_I32]
    L.blazo_block_stages.argtypes = [_D, ctypes.POINTER(Stages)]
    L.blazo_compress_block.argtypes = [_D, _D, _D, _U8, _I8]
    L.blazo_decompress_block.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_uint8, _I8, _D]
    L.blazo_compress.argtypes = [_D, _i64, _i64, _i64, _D, _D, _U8, _I8]
    L.blazo_compress_blocks.argtypes = [_D, _i64, _i64, _i64, _I64, _i64, _D, _D, _U8, _I8]
    L.blazo_decompress.argtypes = [_D, _D, _U8, _I8, _i64, _i64, _D, _i64]
    L.blazo_add.argtypes = [_i64, _D, _D, _U8, _I8, _D, _D, _U8, _I8, _D, _D, _U8, _I8]
    L.blazo_sub.argtypes = [_i64, _D, _D, _U8, _I8, _D, _D, _U8, _I8, _D, _D, _U8, _I8]
    L.blazo_scale.argtypes = [_i64, _D, _D, _U8, _I8, ctypes.c_double, _D, _D, _U8, _I8]
    L.blazo_dot.argtypes = [_D, _D, _U8, _I8, _D, _D, _U8, _I8, _i64, _D, _D]
    L.blazo_dot_rowcol.argtypes = [_D, _D, _U8, _I8, _i64, _i64, _D, _D, _U8, _I8, _i64, _i64, _i64, _D, _D]
    L.blazo_matmul_entries.argtypes = [_D, _D, _U8, _I8, _i64, _i64, _D, _i64, _i64, _I64, _I64, _i64, _D, _D]
    L.blazo_matmul.argtypes = [_D, _D, _U8, _I8, _i64, _i64, _D, _i64, _i64, _D, _i64]
    for name in ("blazo_compress", "blazo_compress_blocks", "blazo_decompress", "blazo_add", "blazo_sub", "blazo_scale",
                 "blazo_dot", "blazo_dot_rowcol", "blazo_matmul_entries", "blazo_matmul"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("blazo_dct_tables", "blazo_kept_positions", "blazo_block_stages", "blazo_compress_block",
                 "blazo_decompress_block"):
        getattr(L, name).restype = None
    L.blazo_keep_count.argtypes = [ctypes.c_int]
    L.blazo_keep_count.restype = ctypes.c_int
    L.blazo_compress_rate.argtypes = [_D, _i64, _i64, _i64, ctypes.c_int, _D, _D, _U8, _I8]
    L.blazo_decompress_rate.argtypes = [_D, _D, _U8, _I8, ctypes.c_int, _i64, _i64, _D, _i64]
    L.blazo_add_rate.argtypes = [_i64, ctypes.c_int, ctypes.c_int, _D, _D, _U8, _I8, _D, _D, _U8, _I8,
                                 _D, _D, _U8, _I8]


def _p(a, t):
    return a.ctypes.data_as(t)


def _chk(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


@dataclass
class CMat:
    """A compressed matrix held on the host (structure of arrays)."""

    rows: int
    cols: int
    f: np.ndarray
    s: np.ndarray
    phi: np.ndarray
    code: np.ndarray

    @property
    def nb(self) -> int:
        return (self.rows // 8) * (self.cols // 8)

    @staticmethod
    def empty(rows: int, cols: int) -> "CMat":
        nb = (rows // 8) * (cols // 8)
        return CMat(rows, cols, np.zeros(nb), np.zeros(nb), np.zeros(nb, np.uint8),
                    np.zeros((nb, NKEEP), np.int8))


def dct_tables():
    """(COS[8][8], AA[8][8]) used by the oracle's DCT."""
    c = np.zeros(64)
    a = np.zeros(64)
    lib().blazo_dct_tables(_p(c, _D), _p(a, _D))
    return c.reshape(8, 8), a.reshape(8, 8)


def kept_positions():
    out = np.zeros(56, np.int32)
    lib().blazo_kept_positions(_p(out, _I32))
    return out.reshape(28, 2)


def block_stages(M) -> dict:
    """All stages of compressing one 8x8 block, as numpy arrays."""
    M = np.ascontiguousarray(M, dtype=np.float64).reshape(64)
    st = Stages()
    lib().blazo_block_stages(_p(M, _D), ctypes.byref(st))
    return {
        "delta": np.array(st.delta).reshape(8, 8),
        "K": int(st.K),
        "sum_abs": float(st.sum_abs),
        "s": float(st.s),
        "dprime": np.array(st.dprime).reshape(8, 8),
        "s_max": float(st.s_max),
        "psi": np.array(st.psi, dtype=np.uint8).reshape(8, 8),
        "dct": np.array(st.dct).reshape(8, 8),
        "m": float(st.m),
        "phi": int(st.phi),
        "f": float(st.f),
        "code": np.array(st.code, dtype=np.int8),
    }


def decompress_block(f, s, phi, code):
    code = np.ascontiguousarray(code, dtype=np.int8)
    out = np.zeros(64)
    lib().blazo_decompress_block(float(f), float(s), int(phi), _p(code, _I8), _p(out, _D))
    return out.reshape(8, 8)


def compress(A) -> CMat:
    A = np.ascontiguousarray(A, dtype=np.float64)
    rows, cols = A.shape
    out = CMat.empty(rows, cols)
    _chk(lib().blazo_compress(_p(A, _D), rows, cols, cols, _p(out.f, _D), _p(out.s, _D),
                              _p(out.phi, _U8), _p(out.code, _I8)), "compress")
    return out


def compress_blocks(A, blocks):
    """Compress only the listed block indices; returns (f, s, phi, code)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    rows, cols = A.shape
    blocks = np.ascontiguousarray(blocks, dtype=np.int64)
    n = blocks.size
    f, s = np.zeros(n), np.zeros(n)
    phi, code = np.zeros(n, np.uint8), np.zeros((n, NKEEP), np.int8)
    _chk(lib().blazo_compress_blocks(_p(A, _D), rows, cols, cols, _p(blocks, _I64), n, _p(f, _D),
                                     _p(s, _D), _p(phi, _U8), _p(code, _I8)), "compress_blocks")
    return f, s, phi, code


def decompress(c: CMat):
    out = np.zeros((c.rows, c.cols))
    _chk(lib().blazo_decompress(_p(c.f, _D), _p(c.s, _D), _p(c.phi, _U8), _p(c.code, _I8), c.rows,
                                c.cols, _p(out, _D), c.cols), "decompress")
    return out


def add(a: CMat, b: CMat) -> CMat:
    assert (a.rows, a.cols) == (b.rows, b.cols)
    out = CMat.empty(a.rows, a.cols)
    _chk(lib().blazo_add(a.nb, _p(a.f, _D), _p(a.s, _D), _p(a.phi, _U8), _p(a.code, _I8),
                         _p(b.f, _D), _p(b.s, _D), _p(b.phi, _U8), _p(b.code, _I8),
                         _p(out.f, _D), _p(out.s, _D), _p(out.phi, _U8), _p(out.code, _I8)), "add")
    return out


def sub(a: CMat, b: CMat) -> CMat:
    """Subtraction read from Sec. III (works like Algorithm 1)."""
    assert (a.rows, a.cols) == (b.rows, b.cols)
    out = CMat.empty(a.rows, a.cols)
    _chk(lib().blazo_sub(a.nb, _p(a.f, _D), _p(a.s, _D), _p(a.phi, _U8), _p(a.code, _I8),
                         _p(b.f, _D), _p(b.s, _D), _p(b.phi, _U8), _p(b.code, _I8),
                         _p(out.f, _D), _p(out.s, _D), _p(out.phi, _U8), _p(out.code, _I8)), "sub")
    return out


def scale(a: CMat, c: float) -> CMat:
    out = CMat.empty(a.rows, a.cols)
    _chk(lib().blazo_scale(a.nb, _p(a.f, _D), _p(a.s, _D), _p(a.phi, _U8), _p(a.code, _I8), float(c),
                           _p(out.f, _D), _p(out.s, _D), _p(out.phi, _U8), _p(out.code, _I8)), "scale")
    return out


def dot(a: CMat, b: CMat):
    """Flattened dot <vec A_hat, vec B_hat>; returns (value, sum |A_hat B_hat|)."""
    assert (a.rows, a.cols) == (b.rows, b.cols)
    r = np.zeros(1)
    ar = np.zeros(1)
    _chk(lib().blazo_dot(_p(a.f, _D), _p(a.s, _D), _p(a.phi, _U8), _p(a.code, _I8),
                         _p(b.f, _D), _p(b.s, _D), _p(b.phi, _U8), _p(b.code, _I8), a.nb,
                         _p(r, _D), _p(ar, _D)), "dot")
    return float(r[0]), float(ar[0])


def dot_rowcol(a: CMat, b: CMat, i: int, j: int):
    """Line i of A_hat times column j of B_hat (Algorithm 3); returns (value, abs sum)."""
    assert a.cols == b.rows
    r = np.zeros(1)
    ar = np.zeros(1)
    _chk(lib().blazo_dot_rowcol(_p(a.f, _D), _p(a.s, _D), _p(a.phi, _U8), _p(a.code, _I8), a.rows, a.cols,
                                _p(b.f, _D), _p(b.s, _D), _p(b.phi, _U8), _p(b.code, _I8), b.cols, int(i),
                                int(j), _p(r, _D), _p(ar, _D)), "dot_rowcol")
    return float(r[0]), float(ar[0])


def matmul_entries(a: CMat, B, ii, jj):
    """Entries (ii[q], jj[q]) of A_hat @ B; returns (values, sum_k |A_hat_ik B_kj|)."""
    B = np.ascontiguousarray(B, dtype=np.float64)
    k, m = B.shape
    assert k == a.cols
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    out = np.zeros(ii.size)
    aout = np.zeros(ii.size)
    _chk(lib().blazo_matmul_entries(_p(a.f, _D), _p(a.s, _D), _p(a.phi, _U8), _p(a.code, _I8), a.rows,
                                    a.cols, _p(B, _D), m, m, _p(ii, _I64), _p(jj, _I64), ii.size,
                                    _p(out, _D), _p(aout, _D)), "matmul_entries")
    return out, aout


def matmul(a: CMat, B):
    B = np.ascontiguousarray(B, dtype=np.float64)
    k, m = B.shape
    assert k == a.cols
    C = np.zeros((a.rows, m))
    _chk(lib().blazo_matmul(_p(a.f, _D), _p(a.s, _D), _p(a.phi, _U8), _p(a.code, _I8), a.rows, a.cols,
                            _p(B, _D), m, m, _p(C, _D), m), "matmul")
    return C


def matmul_cc(a: CMat, b: CMat):
    """A_hat @ B_hat of two compressed matrices (Sec. III, "Matrix
    multiplication": the product of the decompressed blocks, each
    decompressed once): B is decompressed by the oracle, then the plain
    i-j-k product of `matmul`."""
    assert a.cols == b.rows
    return matmul(a, decompress(b))



# --- matrices of any shape (padding) ------------------------------------------
# The paper states that the method works for matrices of any dimensions
# without saying how the last partial blocks are formed.  Reading: the matrix
# is extended to the next multiple of 8 in each direction by repeating its
# last row and its last column (edge replication, so the boundary blocks stay
# as smooth as the data); the compressed matrix is that of the extension, and
# every result refers to the logical rows x cols entries only.

def ceil8(n: int) -> int:
    return (n + 7) // 8 * 8


def pad_edge(A):
    """The edge-replicated extension of A to multiples of 8."""
    A = np.asarray(A, dtype=np.float64)
    rows, cols = A.shape
    r8, c8 = ceil8(rows), ceil8(cols)
    if rows == 0 or cols == 0:
        return np.zeros((r8, c8))
    return np.pad(A, ((0, r8 - rows), (0, c8 - cols)), mode="edge")


def compress_padded(A) -> CMat:
    return compress(pad_edge(A))


def decompress_padded(c: CMat, rows: int, cols: int):
    assert (ceil8(rows), ceil8(cols)) == (c.rows, c.cols)
    return decompress(c)[:rows, :cols]


def dot_padded(a: CMat, b: CMat, rows: int, cols: int):
    """<vec A_hat, vec B_hat> over the logical entries; (value, sum |A_hat B_hat|)."""
    import math

    p = decompress_padded(a, rows, cols) * decompress_padded(b, rows, cols)
    return math.fsum(p.ravel().tolist()), math.fsum(np.abs(p).ravel().tolist())


def matmul_padded(a: CMat, B, n: int, k: int):
    """A_hat (logical n x k) @ B (k x m)."""
    return decompress_padded(a, n, k) @ np.asarray(B, dtype=np.float64)


def matmul_cc_padded(a: CMat, b: CMat, n: int, k: int, m: int):
    return decompress_padded(a, n, k) @ decompress_padded(b, k, m)


# --- tunable rate: the first r rows and r columns of the DCT kept -----------------
def keep_count(r: int) -> int:
    """Codes per block at rate r (8 r + (8 - r) r; 28 for r = 2)."""
    n = lib().blazo_keep_count(int(r))
    if n < 0:
        raise ValueError("r must be 1..8")
    return n


def empty_rate(rows: int, cols: int, r: int) -> CMat:
    nb = (rows // 8) * (cols // 8)
    return CMat(rows, cols, np.zeros(nb), np.zeros(nb), np.zeros(nb, np.uint8),
                np.zeros((nb, keep_count(r)), np.int8))


def compress_rate(A, r: int) -> CMat:
    A = np.ascontiguousarray(A, dtype=np.float64)
    rows, cols = A.shape
    out = empty_rate(rows, cols, r)
    _chk(lib().blazo_compress_rate(_p(A, _D), rows, cols, cols, int(r), _p(out.f, _D), _p(out.s, _D),
                                   _p(out.phi, _U8), _p(out.code, _I8)), "compress_rate")
    return out


def decompress_rate(c: CMat, r: int):
    out = np.zeros((c.rows, c.cols))
    _chk(lib().blazo_decompress_rate(_p(c.f, _D), _p(c.s, _D), _p(c.phi, _U8), _p(c.code, _I8), int(r),
                                     c.rows, c.cols, _p(out, _D), c.cols), "decompress_rate")
    return out


def add_rate(a: CMat, b: CMat, r: int, sub: bool = False) -> CMat:
    """Algorithm 1 (sub: the subtraction) on rate-r blocks."""
    assert (a.rows, a.cols) == (b.rows, b.cols)
    out = empty_rate(a.rows, a.cols, r)
    _chk(lib().blazo_add_rate(a.nb, int(r), int(bool(sub)), _p(a.f, _D), _p(a.s, _D), _p(a.phi, _U8),
                              _p(a.code, _I8), _p(b.f, _D), _p(b.s, _D), _p(b.phi, _U8), _p(b.code, _I8),
                              _p(out.f, _D), _p(out.s, _D), _p(out.phi, _U8), _p(out.code, _I8)), "add_rate")
    return out


def scale_rate(a: CMat, c: float) -> CMat:
    """Algorithm 2 on rate-r blocks: f and s times c, phi and the codes kept."""
    return CMat(a.rows, a.cols, a.f * float(c), a.s * float(c), a.phi.copy(), a.code.copy())


def dot_rate(a: CMat, b: CMat, r: int):
    """<vec A_hat, vec B_hat> of rate-r matrices from the oracle's rate-r
    decompression; returns (value, sum |A_hat B_hat|), both summed exactly
    (math.fsum) over the rounded products."""
    import math

    x = (decompress_rate(a, r) * decompress_rate(b, r)).ravel()
    return math.fsum(x), math.fsum(np.abs(x))


def dot_rowcol_rate(a: CMat, b: CMat, r: int, i: int, j: int):
    """Line i of A_hat times column j of B_hat at rate r (Algorithm 3's
    result, by definition from the decompressed matrices); (value, abs sum)."""
    import math

    x = decompress_rate(a, r)[i, :] * decompress_rate(b, r)[:, j]
    return math.fsum(x), math.fsum(np.abs(x))


def matmul_rate(a: CMat, r: int, B):
    """A_hat @ B at rate r, and |A_hat| @ |B| (for componentwise bounds)."""
    Ah = decompress_rate(a, r)
    B = np.asarray(B, dtype=np.float64)
    return Ah @ B, np.abs(Ah) @ np.abs(B)
