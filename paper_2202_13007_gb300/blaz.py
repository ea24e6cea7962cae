"""Thin ctypes binding of libblaz (include/blaz.h), same names as the C ABI.

Argument marshalling only: every step of the compressed-matrix path runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.
There is no fallback: if libblaz.so is missing or no GPU is present, calls
raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _build

NKEEP = 28
MM_FP64 = 0
MM_SPLIT_BF16 = 1
_MODES = {"fp64": MM_FP64, "split_bf16": MM_SPLIT_BF16}


class BlazError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib().blaz_strerror(status).decode()
        if status == -5:
            msg += f" (cudaError {lib().blaz_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [{status}]")
        self.status = status


class _CMatDesc(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("f", ctypes.c_void_p),
                ("s", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("code", ctypes.c_void_p)]


class _Op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("a", _CMatDesc), ("b", _CMatDesc), ("out", _CMatDesc),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("c", ctypes.c_double),
                ("result", ctypes.c_void_p), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("m", ctypes.c_int64), ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


class _BatchCfg(ctypes.Structure):
    _fields_ = [("blocks_per_item", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("autotune", ctypes.c_int32)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_int64), ("items", ctypes.c_int64), ("gemm_tiles", ctypes.c_int64),
                ("blocks_per_item", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("scratch_bytes", ctypes.c_int64), ("tuned_ms", ctypes.c_double)]


OP_COMPRESS, OP_DECOMPRESS, OP_ADD, OP_SUB, OP_SCALE, OP_DOT, OP_MATMUL = range(7)
REQ_RELEASE = 7


class _ServerCfg(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("max_wait_us", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("matmul_mode", ctypes.c_int32)]


class _Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("host_A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("a", ctypes.c_uint64),
                ("b", ctypes.c_uint64), ("c", ctypes.c_double), ("host_B", ctypes.c_void_p),
                ("ldb", ctypes.c_int64), ("m", ctypes.c_int64), ("host_out", ctypes.c_void_p),
                ("ldo", ctypes.c_int64), ("flags", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("handle", ctypes.c_uint64), ("value", ctypes.c_double),
                ("latency_us", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("resident_matrices", ctypes.c_int64),
                ("resident_bytes", ctypes.c_int64), ("peak_bytes", ctypes.c_int64), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_batch", ctypes.c_double), ("throughput_rps", ctypes.c_double)]

_lib = None

# Every entry point of include/blaz.h with its ctypes signature.
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_DESC = ctypes.POINTER(_CMatDesc)
SIGNATURES = {
    "blaz_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "blaz_last_cuda_error": (ctypes.c_int, []),
    "blaz_device_status": (ctypes.c_int, [_P]),
    "blaz_constants": (None, [_P, _P, _P]),
    "blaz_cmat_alloc": (ctypes.c_int, [_DESC, _I64, _I64, _P]),
    "blaz_cmat_free": (ctypes.c_int, [_DESC, _P]),
    "blaz_compress": (ctypes.c_int, [_P, _I64, _DESC, _P]),
    "blaz_decompress": (ctypes.c_int, [_DESC, _P, _I64, _P]),
    "blaz_add": (ctypes.c_int, [_DESC, _DESC, _DESC, _P]),
    "blaz_sub": (ctypes.c_int, [_DESC, _DESC, _DESC, _P]),
    "blaz_scale": (ctypes.c_int, [_DESC, ctypes.c_double, _DESC, _P]),
    "blaz_dot": (ctypes.c_int, [_DESC, _DESC, _P, _P]),
    "blaz_dot_noalloc": (ctypes.c_int, [_DESC, _DESC, _P, _P]),
    "blaz_dot_rowcol": (ctypes.c_int, [_DESC, _DESC, _I64, _I64, _P, _P]),
    "blaz_matmul": (ctypes.c_int, [_DESC, _P, _I64, _I64, _P, _I64, ctypes.c_int, _P]),
    "blaz_matmul_cc": (ctypes.c_int, [_DESC, _DESC, _P, _I64, ctypes.c_int, _P]),
    "blaz_compress_padded": (ctypes.c_int, [_P, _I64, _I64, _I64, _DESC, _P]),
    "blaz_decompress_padded": (ctypes.c_int, [_DESC, _I64, _I64, _P, _I64, _P]),
    "blaz_dot_padded": (ctypes.c_int, [_DESC, _DESC, _I64, _I64, _P, _P]),
    "blaz_matmul_padded": (ctypes.c_int, [_DESC, _I64, _I64, _P, _I64, _I64, _P, _I64, ctypes.c_int, _P]),
    "blaz_matmul_cc_padded": (ctypes.c_int, [_DESC, _DESC, _I64, _I64, _I64, _P, _I64, ctypes.c_int, _P]),
    "blaz_compress_host": (ctypes.c_int, [_P, _I64, _DESC, _P]),
    "blaz_probe_bounded_wait": (ctypes.c_int, [_I64, _P]),
    "blaz_probe_fp64_rate": (ctypes.c_int, [_I64, ctypes.c_int, _P, _I64, _P, _P]),
    "blaz_debug_block_stages": (ctypes.c_int, [_P, _P, _P]),
    "blaz_keep_count": (ctypes.c_int, [ctypes.c_int]),
    "blaz_cmat_alloc_rate": (ctypes.c_int, [_DESC, _I64, _I64, ctypes.c_int, _P]),
    "blaz_compress_rate": (ctypes.c_int, [_P, _I64, ctypes.c_int, _DESC, _P]),
    "blaz_decompress_rate": (ctypes.c_int, [_DESC, ctypes.c_int, _P, _I64, _P]),
    "blaz_add_rate": (ctypes.c_int, [_DESC, _DESC, ctypes.c_int, _DESC, _P]),
    "blaz_sub_rate": (ctypes.c_int, [_DESC, _DESC, ctypes.c_int, _DESC, _P]),
    "blaz_scale_rate": (ctypes.c_int, [_DESC, ctypes.c_double, ctypes.c_int, _DESC, _P]),
    "blaz_dot_rate": (ctypes.c_int, [_DESC, _DESC, ctypes.c_int, _P, _P]),
    "blaz_dot_rowcol_rate": (ctypes.c_int, [_DESC, _DESC, ctypes.c_int, _I64, _I64, _P, _P]),
    "blaz_matmul_rate": (ctypes.c_int, [_DESC, ctypes.c_int, _P, _I64, _I64, _P, _I64, ctypes.c_int, _P]),
    "blaz_matmul_cc_rate": (ctypes.c_int, [_DESC, _DESC, ctypes.c_int, _P, _I64, ctypes.c_int, _P]),
    "blaz_cmat_download": (ctypes.c_int, [_DESC, _P, _P]),
    "blaz_cmat_upload": (ctypes.c_int, [_P, _DESC, _P]),
    "blaz_cmat_save": (ctypes.c_int, [_DESC, ctypes.c_char_p, _P]),
    "blaz_cmat_file_info": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "blaz_cmat_load": (ctypes.c_int, [ctypes.c_char_p, _DESC, _P]),
    "blaz_batch_plan": (ctypes.c_int, [ctypes.POINTER(_Op), _I64, ctypes.POINTER(_BatchCfg),
                                       ctypes.POINTER(ctypes.c_void_p), _P]),
    "blaz_batch_run": (ctypes.c_int, [_P, _P]),
    "blaz_batch_info_get": (ctypes.c_int, [_P, ctypes.POINTER(_BatchInfo)]),
    "blaz_batch_free": (ctypes.c_int, [_P]),
    "blaz_server_create": (ctypes.c_int, [ctypes.POINTER(_ServerCfg), ctypes.POINTER(ctypes.c_void_p)]),
    "blaz_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]),
    "blaz_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(_Result)]),
    "blaz_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(_Result), _I64]),
    "blaz_server_cmat": (ctypes.c_int, [_P, ctypes.c_uint64, _DESC]),
    "blaz_server_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(_ServerStats)]),
    "blaz_server_destroy": (ctypes.c_int, [_P]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libblaz.so (build it first with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libblaz.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc: int, what: str):
    if rc != 0:
        raise BlazError(rc, what)


def _dev_f64(t: torch.Tensor, name: str):
    if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 2):
        raise TypeError(f"{name} must be a 2-D float64 CUDA tensor")
    if t.numel() and t.stride(1) != 1:
        raise TypeError(f"{name} must have unit column stride")


def _ld(t: torch.Tensor) -> int:
    """Leading dimension of a row-major matrix view (the row length when empty,
    where torch may report any stride)."""
    return t.stride(0) if t.numel() else t.shape[1]


@dataclass
class CMat:
    """A compressed matrix in device memory (structure of arrays, Sec. II)."""

    rows: int
    cols: int
    f: torch.Tensor      # float64 [nb]
    s: torch.Tensor      # float64 [nb]
    phi: torch.Tensor    # uint8   [nb]
    code: torch.Tensor   # int8    [nb, keep(rate)] (28 at the default rate 2)
    shape: tuple | None = None  # logical (rows, cols) when compressed by blaz_compress_padded
    rate: int = 2        # first `rate` DCT rows and columns kept (the blaz_*_rate entry points)

    @property
    def nb(self) -> int:
        return (self.rows // 8) * (self.cols // 8)

    @property
    def nbytes(self) -> int:
        return self.nb * (8 + 8 + 1 + keep_count(self.rate))

    @staticmethod
    def empty(rows: int, cols: int, device=None, rate: int = 2) -> "CMat":
        device = device or torch.device("cuda", torch.cuda.current_device())
        if rows % 8 or cols % 8 or rows < 0 or cols < 0:
            raise ValueError("sides must be non-negative multiples of 8")
        nb = (rows // 8) * (cols // 8)
        return CMat(rows, cols, torch.empty(nb, dtype=torch.float64, device=device),
                    torch.empty(nb, dtype=torch.float64, device=device),
                    torch.empty(nb, dtype=torch.uint8, device=device),
                    torch.empty((nb, keep_count(rate)), dtype=torch.int8, device=device), rate=rate)

    def desc(self) -> _CMatDesc:
        return _CMatDesc(self.rows, self.cols, self.f.data_ptr(), self.s.data_ptr(), self.phi.data_ptr(),
                         self.code.data_ptr())

    def to_host(self):
        return (self.f.cpu().numpy(), self.s.cpu().numpy(), self.phi.cpu().numpy(), self.code.cpu().numpy())


def device_status(stream=None) -> int:
    """Synchronize `stream` and return (and clear) the device status word:
    0, or -7 (BLAZ_ERR_TIMEOUT) if a kernel's bounded wait ran out."""
    return lib().blaz_device_status(_stream(stream))


class BlockStages(ctypes.Structure):
    """blaz_block_stages of include/blaz.h: the stages of compressing one block."""

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


def debug_block_stages(M, stream=None) -> dict:
    """Every stage of compressing one 8x8 block (M: 64 binary64 values on the
    GPU, row-major), computed by the library's kernel; numpy arrays back."""
    M = M.contiguous()
    if M.dtype != torch.float64 or M.numel() != 64 or not M.is_cuda:
        raise ValueError("M must be 64 float64 values on a CUDA device")
    buf = torch.zeros(ctypes.sizeof(BlockStages), dtype=torch.uint8, device=M.device)
    _check(lib().blaz_debug_block_stages(M.data_ptr(), buf.data_ptr(), _stream(stream)), "blaz_debug_block_stages")
    host = buf.cpu().numpy()
    st = BlockStages.from_buffer_copy(host.tobytes())
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


def probe_fp64_rate(iters: int, out, warps_per_sm: int = 16, stream=None) -> int:
    """Launch the binary64 issue-rate probe on `stream` (out: float64 device
    tensor of at least 32 x warps_per_sm x SM count elements); returns the
    number of binary64 additions launched (time the launch with CUDA events)."""
    ops = ctypes.c_int64(0)
    _check(lib().blaz_probe_fp64_rate(int(iters), int(warps_per_sm), out.data_ptr(), out.numel(), ctypes.byref(ops),
                                      _stream(stream)), "blaz_probe_fp64_rate")
    return ops.value


def constants():
    """(cos table [8,8], alpha_i alpha_j table [8,8], kept positions [28,2]) of the library."""
    import numpy as np

    c = np.zeros(64)
    a = np.zeros(64)
    k = np.zeros(56, np.int32)
    lib().blaz_constants(c.ctypes.data, a.ctypes.data, k.ctypes.data)
    return c.reshape(8, 8), a.reshape(8, 8), k.reshape(28, 2)


def blaz_compress(A: torch.Tensor, out: CMat | None = None, stream=None) -> CMat:
    _dev_f64(A, "A")
    rows, cols = A.shape
    out = out or CMat.empty(rows, cols, A.device)
    if (out.rows, out.cols) != (rows, cols):
        raise ValueError("out shape mismatch")
    d = out.desc()
    _check(lib().blaz_compress(A.data_ptr(), _ld(A), ctypes.byref(d), _stream(stream)), "blaz_compress")
    return out


def blaz_decompress(a: CMat, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty((a.rows, a.cols), dtype=torch.float64, device=a.f.device)
    _dev_f64(out, "out")
    d = a.desc()
    _check(lib().blaz_decompress(ctypes.byref(d), out.data_ptr(), _ld(out), _stream(stream)),
           "blaz_decompress")
    return out


def _binary(name, a: CMat, b: CMat, out: CMat | None, stream):
    out = out or CMat.empty(a.rows, a.cols, a.f.device)
    da, db, do = a.desc(), b.desc(), out.desc()
    _check(getattr(lib(), name)(ctypes.byref(da), ctypes.byref(db), ctypes.byref(do), _stream(stream)), name)
    return out


def blaz_add(a: CMat, b: CMat, out: CMat | None = None, stream=None) -> CMat:
    return _binary("blaz_add", a, b, out, stream)


def blaz_sub(a: CMat, b: CMat, out: CMat | None = None, stream=None) -> CMat:
    return _binary("blaz_sub", a, b, out, stream)


def blaz_scale(a: CMat, c: float, out: CMat | None = None, stream=None) -> CMat:
    out = out or CMat.empty(a.rows, a.cols, a.f.device)
    da, do = a.desc(), out.desc()
    _check(lib().blaz_scale(ctypes.byref(da), float(c), ctypes.byref(do), _stream(stream)), "blaz_scale")
    return out


def keep_count(r: int) -> int:
    """Codes kept per block at rate r (8r + (8-r)r; ValueError outside 1..8)."""
    if not 1 <= int(r) <= 8:
        raise ValueError("rate must be in 1..8")
    return 8 * int(r) + (8 - int(r)) * int(r)


def _same_rate(*ms: CMat) -> int:
    r = ms[0].rate
    for m in ms:
        if m.rate != r or m.code.shape != (m.nb, keep_count(r)):
            raise ValueError("operands must have the same rate and [nb, keep(rate)] codes")
    return r


def blaz_compress_rate(A: torch.Tensor, r: int, out: CMat | None = None, stream=None) -> CMat:
    """Compression keeping the first r rows and columns of each block's DCT."""
    _dev_f64(A, "A")
    rows, cols = A.shape
    out = out or CMat.empty(rows, cols, A.device, rate=r)
    if (out.rows, out.cols) != (rows, cols) or out.rate != r:
        raise ValueError("out shape or rate mismatch")
    _same_rate(out)
    d = out.desc()
    _check(lib().blaz_compress_rate(A.data_ptr(), _ld(A), int(r), ctypes.byref(d), _stream(stream)),
           "blaz_compress_rate")
    return out


def blaz_decompress_rate(a: CMat, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    r = _same_rate(a)
    if out is None:
        out = torch.empty((a.rows, a.cols), dtype=torch.float64, device=a.f.device)
    _dev_f64(out, "out")
    d = a.desc()
    _check(lib().blaz_decompress_rate(ctypes.byref(d), r, out.data_ptr(), _ld(out), _stream(stream)),
           "blaz_decompress_rate")
    return out


def _binary_rate(name, a: CMat, b: CMat, out: CMat | None, stream):
    out = out or CMat.empty(a.rows, a.cols, a.f.device, rate=a.rate)
    r = _same_rate(a, b, out)
    da, db, do = a.desc(), b.desc(), out.desc()
    _check(getattr(lib(), name)(ctypes.byref(da), ctypes.byref(db), r, ctypes.byref(do), _stream(stream)), name)
    return out


def blaz_add_rate(a: CMat, b: CMat, out: CMat | None = None, stream=None) -> CMat:
    return _binary_rate("blaz_add_rate", a, b, out, stream)


def blaz_sub_rate(a: CMat, b: CMat, out: CMat | None = None, stream=None) -> CMat:
    return _binary_rate("blaz_sub_rate", a, b, out, stream)


def blaz_scale_rate(a: CMat, c: float, out: CMat | None = None, stream=None) -> CMat:
    out = out or CMat.empty(a.rows, a.cols, a.f.device, rate=a.rate)
    r = _same_rate(a, out)
    da, do = a.desc(), out.desc()
    _check(lib().blaz_scale_rate(ctypes.byref(da), float(c), r, ctypes.byref(do), _stream(stream)),
           "blaz_scale_rate")
    return out


def blaz_dot_rate(a: CMat, b: CMat, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """<vec A_hat, vec B_hat> of two matrices of the same rate."""
    r = _same_rate(a, b)
    out = out if out is not None else torch.empty((), dtype=torch.float64, device=a.f.device)
    da, db = a.desc(), b.desc()
    _check(lib().blaz_dot_rate(ctypes.byref(da), ctypes.byref(db), r, out.data_ptr(), _stream(stream)),
           "blaz_dot_rate")
    return out


def blaz_dot_rowcol_rate(a: CMat, b: CMat, i: int, j: int, out: torch.Tensor | None = None, stream=None):
    """Line i of A_hat times column j of B_hat (Algorithm 3) at the operands' rate."""
    r = _same_rate(a, b)
    out = out if out is not None else torch.empty((), dtype=torch.float64, device=a.f.device)
    da, db = a.desc(), b.desc()
    _check(lib().blaz_dot_rowcol_rate(ctypes.byref(da), ctypes.byref(db), r, int(i), int(j), out.data_ptr(),
                                      _stream(stream)), "blaz_dot_rowcol_rate")
    return out


def blaz_matmul_rate(a: CMat, B: torch.Tensor, mode: str = "fp64", out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    r = _same_rate(a)
    _dev_f64(B, "B")
    if B.shape[0] != a.cols:
        raise ValueError("inner dimensions differ")
    m = B.shape[1]
    if out is None:
        out = torch.empty((a.rows, m), dtype=torch.float64, device=B.device)
    _dev_f64(out, "out")
    da = a.desc()
    _check(lib().blaz_matmul_rate(ctypes.byref(da), r, B.data_ptr(), _ld(B), m, out.data_ptr(), _ld(out),
                                  _MODES[mode], _stream(stream)), "blaz_matmul_rate")
    return out


def blaz_matmul_cc_rate(a: CMat, b: CMat, mode: str = "fp64", out: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
    r = _same_rate(a, b)
    if a.cols != b.rows:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = torch.empty((a.rows, b.cols), dtype=torch.float64, device=a.f.device)
    _dev_f64(out, "out")
    da, db = a.desc(), b.desc()
    _check(lib().blaz_matmul_cc_rate(ctypes.byref(da), ctypes.byref(db), r, out.data_ptr(), _ld(out),
                                     _MODES[mode], _stream(stream)), "blaz_matmul_cc_rate")
    return out


def blaz_dot(a: CMat, b: CMat, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    out = out if out is not None else torch.empty((), dtype=torch.float64, device=a.f.device)
    da, db = a.desc(), b.desc()
    _check(lib().blaz_dot(ctypes.byref(da), ctypes.byref(db), out.data_ptr(), _stream(stream)), "blaz_dot")
    return out


def blaz_dot_noalloc(a: CMat, b: CMat, out: torch.Tensor, stream=None) -> torch.Tensor:
    """blaz_dot for callers that cannot let the library allocate: scratch is a
    fixed array inside the library; ``out`` must be given (one float64 on the
    device).  Calls that may overlap on the GPU must not be issued."""
    da, db = a.desc(), b.desc()
    _check(lib().blaz_dot_noalloc(ctypes.byref(da), ctypes.byref(db), out.data_ptr(), _stream(stream)),
           "blaz_dot_noalloc")
    return out


def blaz_dot_rowcol(a: CMat, b: CMat, i: int, j: int, out: torch.Tensor | None = None, stream=None):
    out = out if out is not None else torch.empty((), dtype=torch.float64, device=a.f.device)
    da, db = a.desc(), b.desc()
    _check(lib().blaz_dot_rowcol(ctypes.byref(da), ctypes.byref(db), int(i), int(j), out.data_ptr(),
                                 _stream(stream)), "blaz_dot_rowcol")
    return out


def blaz_matmul(a: CMat, B: torch.Tensor, mode: str = "fp64", out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    _dev_f64(B, "B")
    if B.shape[0] != a.cols:
        raise ValueError("inner dimensions differ")
    m = B.shape[1]
    if out is None:
        out = torch.empty((a.rows, m), dtype=torch.float64, device=B.device)
    _dev_f64(out, "out")
    da = a.desc()
    _check(lib().blaz_matmul(ctypes.byref(da), B.data_ptr(), _ld(B), m, out.data_ptr(), _ld(out),
                             _MODES[mode], _stream(stream)), "blaz_matmul")
    return out


def blaz_matmul_cc(a: CMat, b: CMat, mode: str = "fp64", out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """C = A_hat * B_hat of two compressed matrices (dense binary64 n x m)."""
    if a.cols != b.rows:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = torch.empty((a.rows, b.cols), dtype=torch.float64, device=a.f.device)
    _dev_f64(out, "out")
    da, db = a.desc(), b.desc()
    _check(lib().blaz_matmul_cc(ctypes.byref(da), ctypes.byref(db), out.data_ptr(), _ld(out),
                                _MODES[mode], _stream(stream)), "blaz_matmul_cc")
    return out


def _ceil8(n: int) -> int:
    return (n + 7) // 8 * 8


def blaz_compress_padded(A: torch.Tensor, out: CMat | None = None, stream=None) -> CMat:
    """Compress a matrix of any shape (edge-replicated to multiples of 8);
    the result's ``shape`` attribute keeps the logical (rows, cols)."""
    _dev_f64(A, "A")
    rows, cols = A.shape
    if out is None:
        out = CMat.empty(_ceil8(rows), _ceil8(cols), device=A.device)
    d = out.desc()
    _check(lib().blaz_compress_padded(A.data_ptr(), _ld(A), rows, cols, ctypes.byref(d), _stream(stream)),
           "blaz_compress_padded")
    out.shape = (rows, cols)
    return out


def _logical(a: CMat, shape):
    return tuple(shape) if shape is not None else (a.shape or (a.rows, a.cols))


def blaz_decompress_padded(a: CMat, shape=None, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    rows, cols = _logical(a, shape)
    if out is None:
        out = torch.empty((rows, cols), dtype=torch.float64, device=a.f.device)
    _dev_f64(out, "out")
    d = a.desc()
    _check(lib().blaz_decompress_padded(ctypes.byref(d), rows, cols, out.data_ptr(), _ld(out), _stream(stream)),
           "blaz_decompress_padded")
    return out


def blaz_dot_padded(a: CMat, b: CMat, shape=None, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    rows, cols = _logical(a, shape)
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=a.f.device)
    da, db = a.desc(), b.desc()
    _check(lib().blaz_dot_padded(ctypes.byref(da), ctypes.byref(db), rows, cols, out.data_ptr(), _stream(stream)),
           "blaz_dot_padded")
    return out


def blaz_matmul_padded(a: CMat, B: torch.Tensor, shape=None, mode: str = "fp64", out: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
    n, k = _logical(a, shape)
    _dev_f64(B, "B")
    if B.shape[0] != k:
        raise ValueError("inner dimensions differ")
    m = B.shape[1]
    if out is None:
        out = torch.empty((n, m), dtype=torch.float64, device=B.device)
    _dev_f64(out, "out")
    da = a.desc()
    _check(lib().blaz_matmul_padded(ctypes.byref(da), n, k, B.data_ptr(), _ld(B), m, out.data_ptr(), _ld(out),
                                    _MODES[mode], _stream(stream)), "blaz_matmul_padded")
    return out


def blaz_matmul_cc_padded(a: CMat, b: CMat, a_shape=None, b_shape=None, mode: str = "fp64",
                          out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n, k = _logical(a, a_shape)
    k2, m = _logical(b, b_shape)
    if k != k2:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = torch.empty((n, m), dtype=torch.float64, device=a.f.device)
    _dev_f64(out, "out")
    da, db = a.desc(), b.desc()
    _check(lib().blaz_matmul_cc_padded(ctypes.byref(da), ctypes.byref(db), n, k, m, out.data_ptr(), _ld(out),
                                       _MODES[mode], _stream(stream)), "blaz_matmul_cc_padded")
    return out


def blaz_compress_host(A: torch.Tensor, out: CMat | None = None, stream=None) -> CMat:
    """Compress a float64 matrix held in host memory (page-locked for full
    speed); transfer and compression are pipelined by the library.  `A` must
    not change until the stream has passed the call."""
    if A.is_cuda or A.dtype != torch.float64 or A.dim() != 2:
        raise TypeError("A must be a 2-D float64 host tensor")
    if A.numel() and A.stride(1) != 1:
        raise TypeError("A must have unit column stride")
    rows, cols = A.shape
    out = out or CMat.empty(rows, cols)
    if (out.rows, out.cols) != (rows, cols):
        raise ValueError("out shape mismatch")
    d = out.desc()
    _check(lib().blaz_compress_host(A.data_ptr(), _ld(A), ctypes.byref(d), _stream(stream)), "blaz_compress_host")
    return out


def blaz_cmat_download(a: CMat, host: torch.Tensor, stream=None) -> torch.Tensor:
    """Copy the packed payload (45 bytes per block) into a uint8 host tensor."""
    if host.is_cuda or host.dtype != torch.uint8 or host.numel() < a.nbytes or not host.is_contiguous():
        raise TypeError("host must be a contiguous uint8 host tensor of at least a.nbytes bytes")
    d = a.desc()
    _check(lib().blaz_cmat_download(ctypes.byref(d), host.data_ptr(), _stream(stream)), "blaz_cmat_download")
    return host


def blaz_cmat_upload(host: torch.Tensor, a: CMat, stream=None) -> CMat:
    """Fill `a` from a packed payload in a uint8 host tensor."""
    if host.is_cuda or host.dtype != torch.uint8 or host.numel() < a.nbytes or not host.is_contiguous():
        raise TypeError("host must be a contiguous uint8 host tensor of at least a.nbytes bytes")
    d = a.desc()
    _check(lib().blaz_cmat_upload(host.data_ptr(), ctypes.byref(d), _stream(stream)), "blaz_cmat_upload")
    return a


def blaz_cmat_save(a: CMat, path, stream=None) -> None:
    """Write `a` to `path` (format in include/blaz.h); blocks until written."""
    da = a.desc()
    _check(lib().blaz_cmat_save(ctypes.byref(da), os.fsencode(path), _stream(stream)), "blaz_cmat_save")


def blaz_cmat_file_info(path) -> tuple[int, int]:
    """(rows, cols) stored in a compressed-matrix file (host only)."""
    r, c = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().blaz_cmat_file_info(os.fsencode(path), ctypes.byref(r), ctypes.byref(c)), "blaz_cmat_file_info")
    return r.value, c.value


def blaz_cmat_load(path, out: CMat | None = None, stream=None) -> CMat:
    """Read a compressed matrix from `path` into `out` (allocated here if None)."""
    if out is None:
        out = CMat.empty(*blaz_cmat_file_info(path))
    do = out.desc()
    _check(lib().blaz_cmat_load(os.fsencode(path), ctypes.byref(do), _stream(stream)), "blaz_cmat_load")
    return out


class Batch:
    """A planned batch of mixed operations (one persistent, graph-captured launch).

    ``ops`` is a list of dicts: {"op": "compress", "A": tensor, "out": CMat},
    {"op": "decompress", "a": CMat, "C": tensor}, {"op": "add"|"sub", "a", "b",
    "out"}, {"op": "scale", "a", "c", "out"}, {"op": "dot", "a", "b", "result":
    float64 tensor (one element)}, {"op": "matmul", "a": CMat, "B": tensor,
    "C": tensor}.  The tensors must stay alive while the plan exists."""

    _KIND = {"compress": OP_COMPRESS, "decompress": OP_DECOMPRESS, "add": OP_ADD, "sub": OP_SUB,
             "scale": OP_SCALE, "dot": OP_DOT, "matmul": OP_MATMUL}

    def __init__(self, ops, blocks_per_item: int = 0, ctas_per_sm: int = 0, autotune: bool = False, stream=None):
        arr = (_Op * max(1, len(ops)))()
        self._keep = []
        for i, d in enumerate(ops):
            o = arr[i]
            o.kind = self._KIND[d["op"]]
            for key in ("a", "b", "out"):
                if key in d:
                    setattr(o, key, d[key].desc())
            if "A" in d:
                _dev_f64(d["A"], "A")
                o.A, o.lda = d["A"].data_ptr(), _ld(d["A"])
            if "c" in d:
                o.c = float(d["c"])
            if "result" in d:
                o.result = d["result"].data_ptr()
            if "B" in d:
                _dev_f64(d["B"], "B")
                o.B, o.ldb, o.m = d["B"].data_ptr(), _ld(d["B"]), d["B"].shape[1]
            if "C" in d:
                _dev_f64(d["C"], "C")
                o.C, o.ldc = d["C"].data_ptr(), _ld(d["C"])
            self._keep.append(d)
        cfg = _BatchCfg(blocks_per_item, ctas_per_sm, 1 if autotune else 0)
        h = ctypes.c_void_p()
        _check(lib().blaz_batch_plan(arr, len(ops), ctypes.byref(cfg), ctypes.byref(h), _stream(stream)),
               "blaz_batch_plan")
        self._h = h

    def run(self, stream=None):
        _check(lib().blaz_batch_run(self._h, _stream(stream)), "blaz_batch_run")

    def info(self) -> dict:
        inf = _BatchInfo()
        _check(lib().blaz_batch_info_get(self._h, ctypes.byref(inf)), "blaz_batch_info_get")
        return {k: getattr(inf, k) for k, _ in _BatchInfo._fields_}

    def free(self):
        if self._h:
            lib().blaz_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Request server: resident compressed matrices on the current device,
    admission by a device-memory budget, continuous batching (C++ scheduler
    thread inside libblaz).  Host inputs are numpy float64 arrays (copied at
    submission); outputs are written into numpy arrays the caller passes and
    keeps alive until the request completes."""

    _KIND = dict(Batch._KIND, release=REQ_RELEASE)

    def __init__(self, budget_bytes: int, streams: int = 0, max_batch: int = 0, max_wait_us: int = 0,
                 queue_capacity: int = 0, matmul_mode: str = "fp64"):
        cfg = _ServerCfg(int(budget_bytes), streams, max_batch, max_wait_us, queue_capacity, _MODES[matmul_mode])
        h = ctypes.c_void_p()
        _check(lib().blaz_server_create(ctypes.byref(cfg), ctypes.byref(h)), "blaz_server_create")
        self._h = h

    def submit(self, op: str, *, A=None, a: int = 0, b: int = 0, c: float = 0.0, B=None, out=None,
               pinned: bool = False) -> int:
        """Queue a request; with pinned=True every host array passed is page-locked
        and must stay valid and unmodified until the request completes."""
        import numpy as np

        r = _Request()
        r.flags = 1 if pinned else 0
        r.kind = self._KIND[op]
        if A is not None:
            assert A.dtype == np.float64 and A.ndim == 2 and A.strides[1] == 8
            r.rows, r.cols = A.shape
            r.host_A, r.lda = A.ctypes.data, A.strides[0] // 8
        r.a, r.b, r.c = a, b, float(c)
        if B is not None:
            assert B.dtype == np.float64 and B.ndim == 2 and B.strides[1] == 8
            r.host_B, r.ldb, r.m = B.ctypes.data, B.strides[0] // 8, B.shape[1]
        if out is not None:
            assert out.dtype == np.float64 and out.strides[-1] == 8
            r.host_out = out.ctypes.data
            r.ldo = out.strides[0] // 8 if out.ndim == 2 else 1
        t = ctypes.c_uint64()
        rc = lib().blaz_server_submit(self._h, ctypes.byref(r), ctypes.byref(t))
        if rc != 0:
            raise BlazError(rc, "blaz_server_submit")
        return t.value

    def poll(self, ticket: int):
        res = _Result()
        _check(lib().blaz_server_poll(self._h, ticket, ctypes.byref(res)), "blaz_server_poll")
        return {k: getattr(res, k) for k, _ in _Result._fields_}

    def wait(self, ticket: int, timeout_s: float = 60.0):
        res = _Result()
        _check(lib().blaz_server_wait(self._h, ticket, ctypes.byref(res), int(timeout_s * 1e6)), "blaz_server_wait")
        return {k: getattr(res, k) for k, _ in _Result._fields_}

    def cmat(self, handle: int) -> "CMat":
        """A copy of a resident matrix as a CMat (device tensors)."""
        d = _CMatDesc()
        _check(lib().blaz_server_cmat(self._h, handle, ctypes.byref(d)), "blaz_server_cmat")
        nb = (d.rows // 8) * (d.cols // 8)
        dev = torch.device("cuda", torch.cuda.current_device())

        def view(ptr, n, dtype, shape):
            if n == 0:
                return torch.empty(shape, dtype=dtype, device=dev)
            nbytes = n * torch.empty((), dtype=dtype).element_size()
            return _from_ptr(ptr, nbytes, dtype, shape, dev)

        return CMat(d.rows, d.cols, view(d.f, nb, torch.float64, (nb,)), view(d.s, nb, torch.float64, (nb,)),
                    view(d.phi, nb, torch.uint8, (nb,)), view(d.code, nb * NKEEP, torch.int8, (nb, NKEEP)))

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib().blaz_server_stats_get(self._h, ctypes.byref(st)), "blaz_server_stats_get")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def destroy(self):
        if self._h:
            lib().blaz_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class _DevArray:
    """Minimal __cuda_array_interface__ exporter for a raw device pointer."""

    _TYPESTR = {torch.float64: "<f8", torch.uint8: "|u1", torch.int8: "|i1"}

    def __init__(self, ptr: int, dtype, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": self._TYPESTR[dtype],
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _from_ptr(ptr: int, nbytes: int, dtype, shape, dev):
    """Copy device memory at `ptr` into a new tensor (reading a server-owned
    matrix; the copy keeps the server's lifetime rules simple)."""
    return torch.as_tensor(_DevArray(ptr, dtype, shape), device=dev).clone()


# short aliases
compress, decompress, add, sub, scale = blaz_compress, blaz_decompress, blaz_add, blaz_sub, blaz_scale
dot, dot_rowcol, matmul, matmul_cc = blaz_dot, blaz_dot_rowcol, blaz_matmul, blaz_matmul_cc
save, load, file_info = blaz_cmat_save, blaz_cmat_load, blaz_cmat_file_info
compress_padded, decompress_padded, dot_padded = blaz_compress_padded, blaz_decompress_padded, blaz_dot_padded
matmul_padded, matmul_cc_padded = blaz_matmul_padded, blaz_matmul_cc_padded
compress_host, download, upload = blaz_compress_host, blaz_cmat_download, blaz_cmat_upload
compress_rate, decompress_rate = blaz_compress_rate, blaz_decompress_rate
add_rate, sub_rate, scale_rate = blaz_add_rate, blaz_sub_rate, blaz_scale_rate
dot_rate, dot_rowcol_rate = blaz_dot_rate, blaz_dot_rowcol_rate
matmul_rate, matmul_cc_rate = blaz_matmul_rate, blaz_matmul_cc_rate
