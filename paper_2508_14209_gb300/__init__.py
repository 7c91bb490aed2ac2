"""Python binding of libmsketch (include/msketch.h): GPU CountSketch,
Count-Gauss multisketch and sketched least squares on GB300.

Argument marshalling only: every numeric step runs in the CUDA library.  The
functions take torch CUDA tensors (PyTorch provides device memory and
streams), check shapes/layouts, allocate the caller-side workspace the C ABI
asks for, and raise MskError on a non-zero status.  There is no CPU path: if
libmsketch.so is missing, importing the library raises.

Layouts: A is d x n column-major (a tensor with stride (1, lda), e.g. the
transpose of a contiguous (n, lda) tensor sliced to d columns); Y is k x ncol
row-major (stride (ldy, 1)); Z is p x ncol column-major.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# The library the binding loads: libmsketch.so, or another build of it (the
# checked build, libmsketch_checked.so) named by MSK_LIB.
LIB_PATH = os.environ.get("MSK_LIB") or os.path.join(_HERE, "libmsketch.so")

MSK_F64, MSK_F32 = 0, 1
GEMM_F64, GEMM_F32, GEMM_BF16, GEMM_F16, GEMM_BF16X3 = 0, 1, 2, 3, 4
CS_ATOMIC, CS_SORTED = 0, 1
MSK_OK, MSK_ENOCONV, MSK_ENOMEM, MSK_ETIMEOUT, MSK_ECUDA, MSK_ENOTSUP, MSK_EBUSY = (
    0, 1001, 1002, 1003, 1004, 1005, 1006)

GEMM_PRECS = {"f64": GEMM_F64, "f32": GEMM_F32, "bf16": GEMM_BF16, "f16": GEMM_F16,
              "bf16x3": GEMM_BF16X3}

# Names of every function include/msketch.h declares (checked by the tests).
EXPORTS = ("msk_version", "msk_last_error", "msk_checked_build", "msk_check_status", "msk_stage_events", "msk_take_timeout", "msk_selftest_wait", "cs_hash", "ms_gaussian", "msk_cs_workspace",
           "cs_sketch", "msk_ms_workspace", "ms_sketch", "msk_gemm_workspace", "msk_gemm",
           "msk_householder_qr", "msk_trsv_upper", "msk_lstsq_workspace", "ms_lstsq",
           "msk_ne_workspace", "ne_lstsq", "msk_normal_apply_workspace", "msk_normal_apply", "msk_rcq_workspace", "rcq_lstsq", "rcq_qr",
           "msk_sns_workspace", "sns_lstsq", "msk_srht_workspace", "srht_sketch",
           "msk_ms_host_workspace", "ms_sketch_host", "ms_sketch_rows",
           "msk_gemm_noalloc", "msk_tune_set", "msk_tune_get",
           "msk_tune_clear", "msk_batch_workspace", "msk_batch_item_bound", "msk_batch_lstsq", "ms_server_create",
           "ms_server_submit", "ms_server_poll", "ms_server_wait_all", "ms_server_stats",
           "ms_server_destroy", "ms_server_error", "msk_autotune_workspace", "msk_autotune")

NOALLOC_SCRATCH_BYTES = 64 << 20


class MskError(RuntimeError):
    def __init__(self, fn, code, detail=""):
        self.code = code
        super().__init__(f"{fn} returned {code}{(': ' + detail) if detail else ''}")


class BatchItem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("d", ctypes.c_int64), ("n", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("b", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("x", ctypes.c_void_p)]


class LstsqInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("relres", ctypes.c_double), ("relres_sns", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libmsketch.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"libmsketch.so not built at {path}; run paper_2508_14209_gb300.build.build()")
        L = ctypes.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


_p, _i64, _u64, _int, _sz, _dbl, _i32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                         ctypes.c_int, ctypes.c_size_t, ctypes.c_double,
                                         ctypes.c_int32)


def _declare(L):
    sig = {
        "msk_version": (ctypes.c_char_p, []),
        "msk_last_error": (ctypes.c_char_p, []),
        "msk_take_timeout": (_int, [_p]),
        "msk_checked_build": (_int, []),
        "msk_stage_events": (_int, [_p, _p]),
        "msk_check_status": (_int, [_p]),
        "msk_selftest_wait": (_int, [_p]),
        "cs_hash": (_int, [_u64, _i64, _i64, _i64, _p, _p, _p]),
        "ms_gaussian": (_int, [_u64, _i64, _i64, _int, _p, _i64, _p]),
        "msk_cs_workspace": (_sz, [_i64, _i64, _i64, _int, _int]),
        "cs_sketch": (_int, [_p, _int, _i64, _i64, _i64, _p, _i64, _u64, _p, _i64, _int, _p, _sz, _p]),
        "msk_ms_workspace": (_sz, [_i64, _i64, _int, _i64, _i64, _int, _int, _int]),
        "ms_sketch": (_int, [_p, _int, _i64, _i64, _i64, _p, _i64, _i64, _u64, _int, _p, _i64, _int,
                             _p, _sz, _p]),
        "msk_gemm_workspace": (_sz, [_i64, _i64, _i64, _int]),
        "msk_gemm": (_int, [_u64, _i64, _i64, _i64, _p, _i64, _int, _p, _i64, _p, _sz, _p]),
        "msk_tune_set": (_int, [ctypes.c_char_p, ctypes.c_longlong]),
        "msk_tune_get": (ctypes.c_longlong, [ctypes.c_char_p, ctypes.c_longlong]),
        "msk_tune_clear": (_int, [ctypes.c_char_p]),
        "msk_gemm_noalloc": (_int, [_u64, _i64, _i64, _i64, _p, _i64, _int, _p, _i64, _p]),
        "msk_householder_qr": (_int, [_p, _i64, _i64, _i64, _p]),
        "msk_trsv_upper": (_int, [_p, _i64, _i64, _p, _p, _p]),
        "msk_lstsq_workspace": (_sz, [_i64, _i64, _i64, _i64, _int, _int, _int]),
        "ms_lstsq": (_int, [_p, _int, _i64, _i64, _i64, _p, _i64, _i64, _u64, _int, _int, _dbl, _i32,
                            _p, ctypes.POINTER(LstsqInfo), _p, _sz, _p]),
        "msk_ne_workspace": (_sz, [_i64, _i64]),
        "ne_lstsq": (_int, [_p, _i64, _i64, _i64, _p, _p, _p, _sz, _p]),
        "msk_normal_apply_workspace": (_sz, [_i64, _i64]),
        "msk_normal_apply": (_int, [_p, _i64, _i64, _i64, _p, _p, _p, _sz, _p]),
        "msk_rcq_workspace": (_sz, [_i64, _i64, _i64, _i64, _int, _int, _int]),
        "msk_sns_workspace": (_sz, [_i64, _i64, _int, _i64, _i64, _int]),
        "msk_srht_workspace": (_sz, [_i64, _i64, _int, _i64]),
        "msk_ms_host_workspace": (_sz, [_i64, _i64, _int, _i64, _i64, _int, _int, _i64]),
        "ms_sketch_rows": (_int, [_p, _int, _i64, _i64, _i64, _p, _i64, _i64, _i64, _u64, _int, _p, _i64, _p,
                                  _sz, _p]),
        "ms_sketch_host": (_int, [_p, _int, _i64, _i64, _i64, _p, _i64, _i64, _u64, _int, _p, _i64, _i64,
                                  _p, _sz, _p]),
        "srht_sketch": (_int, [_p, _int, _i64, _i64, _i64, _p, _i64, _u64, _p, _i64, _p, _sz, _p]),
        "sns_lstsq": (_int, [_p, _int, _i64, _i64, _i64, _p, _int, _i64, _i64, _u64, _p, _p, _p, _sz,
                             _p]),
        "rcq_lstsq": (_int, [_p, _int, _i64, _i64, _i64, _p, _i64, _i64, _u64, _int, _p, _p, _p, _sz,
                             _p]),
        "rcq_qr": (_int, [_p, _int, _i64, _i64, _i64, _i64, _i64, _u64, _int, _p, _i64, _p, _i64, _p,
                          _sz, _p]),
        "msk_batch_workspace": (_sz, [ctypes.POINTER(BatchItem), _int, _int]),
        "msk_batch_item_bound": (_sz, [ctypes.POINTER(BatchItem), _int]),
        "ms_server_create": (_int, [_sz, _int, _int, _int, _dbl, _i32, ctypes.POINTER(_p)]),
        "ms_server_submit": (_int, [_p, ctypes.POINTER(BatchItem), ctypes.POINTER(_u64)]),
        "ms_server_poll": (_int, [_p, _u64, ctypes.POINTER(_int), ctypes.POINTER(LstsqInfo),
                                  ctypes.POINTER(_dbl)]),
        "ms_server_wait_all": (_int, [_p]),
        "ms_server_stats": (_int, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
        "ms_server_destroy": (_int, [_p]),
        "ms_server_error": (ctypes.c_char_p, [_p]),
        "msk_batch_lstsq": (_int, [ctypes.POINTER(BatchItem), _int, _int, _dbl, _i32,
                                   ctypes.POINTER(LstsqInfo), _p, _sz, _p]),
        "msk_autotune_workspace": (_sz, [ctypes.POINTER(BatchItem), _int, _int]),
        "msk_autotune": (_int, [ctypes.POINTER(BatchItem), _int, _int, _dbl, _i32, _int, ctypes.c_char_p,
                                _sz, _p, _sz, _p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def tune_set(name: str, value: int) -> None:
    _check("msk_tune_set", load().msk_tune_set(name.encode(), int(value)))


def tune_get(name: str, default: int = -1) -> int:
    return int(load().msk_tune_get(name.encode(), int(default)))


def tune_clear(name: str | None = None) -> None:
    load().msk_tune_clear(None if name is None else name.encode())


def version() -> str:
    return load().msk_version().decode()


def msk_take_timeout(stream=None) -> int:
    """Synchronise the stream; MSK_ETIMEOUT if a pipelined kernel gave up a
    bounded wait since the last call (the record is cleared), else MSK_OK."""
    return int(load().msk_take_timeout(_stream(stream)))


def msk_checked_build() -> bool:
    """True when the loaded library was built with device-side index checks."""
    return bool(load().msk_checked_build())


def msk_check_status(stream=None) -> int:
    """Site of the first failed index check since the last call (0: none)."""
    rc = load().msk_check_status(_stream(stream))
    if rc < 0 or rc == MSK_ECUDA:
        _check("msk_check_status", rc)
    return rc


def msk_selftest_wait(stream=None) -> None:
    """Launch the bounded-wait test kernel (its wait expires after 1 s)."""
    _check("msk_selftest_wait", load().msk_selftest_wait(_stream(stream)))


def _check(fn, rc, ok=(MSK_OK,)):
    if rc not in ok:
        raise MskError(fn, rc, load().msk_last_error().decode())
    return rc


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dtype_code(t):
    if t.dtype == torch.float64:
        return MSK_F64
    if t.dtype == torch.float32:
        return MSK_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _colmajor(A):
    """(lda) of a d x n column-major tensor view."""
    if A.dim() != 2:
        raise ValueError("A must be 2-D")
    d, n = A.shape
    if d > 1 and A.stride(0) != 1:
        raise ValueError("A must be column-major (stride(0) == 1)")
    lda = A.stride(1) if n > 1 else max(d, 1)
    return max(lda, max(d, 1))


def _cuda(t, name):
    if t is not None and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


def workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def colmajor(d, n, dtype, device, lda=None):
    """Uninitialised d x n column-major tensor (leading dimension lda)."""
    lda = d if lda is None else lda
    buf = torch.empty((max(n, 1), max(lda, 1)), dtype=dtype, device=device)
    return buf[:n, :d].t()


# ---------------------------------------------------------------------------

def cs_hash(seed, i0, count, k, h=None, s=None, stream=None, device="cuda"):
    """Buckets h(i) (uint32 stored in int32 tensor) and signs s(i) of rows
    i0..i0+count-1."""
    if h is None:
        h = torch.empty(count, dtype=torch.int32, device=device)
    if s is None:
        s = torch.empty(count, dtype=torch.int8, device=device)
    _check("cs_hash", load().cs_hash(seed & (2**64 - 1), i0, count, k, _ptr(h), _ptr(s), _stream(stream)))
    return h, s


_PREC_DTYPE = {GEMM_F64: torch.float64, GEMM_F32: torch.float32, GEMM_BF16: torch.bfloat16,
               GEMM_F16: torch.float16}


def ms_gaussian(seed, p, k, out_prec=GEMM_F32, G=None, stream=None, device="cuda"):
    """The p x k Gaussian (row-major) of the multisketch's second stage."""
    if G is None:
        G = torch.empty((p, k), dtype=_PREC_DTYPE[out_prec], device=device)
    _check("ms_gaussian", load().ms_gaussian(seed & (2**64 - 1), p, k, out_prec, _ptr(G), G.stride(0),
                                             _stream(stream)))
    return G


def msk_cs_workspace(d, n, k, dtype, strategy):
    return load().msk_cs_workspace(d, n, k, dtype, strategy)


def cs_sketch(A, k, seed, b=None, Y=None, strategy=CS_ATOMIC, ws=None, stream=None):
    """Y = S [A b] (k x ncol, row-major, A's dtype)."""
    _cuda(A, "A"), _cuda(b, "b")
    d, n = A.shape
    lda = _colmajor(A)
    dt = _dtype_code(A)
    ncol = n + (0 if b is None else 1)
    if b is not None and (b.dtype != torch.float64 or b.numel() != d):
        raise ValueError("b must be float64 of length d")
    if Y is None:
        Y = torch.empty((k, ncol), dtype=A.dtype, device=A.device)
    need = msk_cs_workspace(d, n, k, dt, strategy)
    if ws is None and need:
        ws = workspace(need, A.device)
    _check("cs_sketch", load().cs_sketch(_ptr(A), dt, d, n, lda, _ptr(b), k, seed & (2**64 - 1), _ptr(Y),
                                         Y.stride(0), strategy, _ptr(ws),
                                         0 if ws is None else ws.numel(), _stream(stream)))
    return Y


def ms_sketch_rows(A, row0, k, p, seed, b=None, gemm_prec=GEMM_F64, Z=None, ws=None, stream=None):
    """Z = G S [A b] for the row block A (device, column-major) holding rows
    row0 .. row0+d-1 of a taller matrix: hashed with global row indices, so
    the blocks' Z add up to the whole matrix's."""
    _cuda(A, "A"), _cuda(b, "b")
    d, n = A.shape
    dt = _dtype_code(A)
    ncol = n + (0 if b is None else 1)
    if Z is None:
        Z = colmajor(p, ncol, torch.float64, A.device)
    if ws is None:
        ws = workspace(msk_ms_workspace(d, n, b is not None, k, p, dt, gemm_prec), A.device)
    _check("ms_sketch_rows", load().ms_sketch_rows(_ptr(A), dt, d, n, _colmajor(A), _ptr(b), row0, k, p,
                                                   seed & (2**64 - 1), gemm_prec, _ptr(Z), _colmajor(Z),
                                                   _ptr(ws), ws.numel(), _stream(stream)))
    return Z


def msk_ms_host_workspace(d, n, with_b, k, p, dtype, gemm_prec, chunk_rows=0):
    return load().msk_ms_host_workspace(d, n, int(with_b), k, p, dtype, gemm_prec, chunk_rows)


def ms_sketch_host(A, k, p, seed, b=None, gemm_prec=GEMM_F64, Z=None, chunk_rows=0, ws=None,
                   stream=None, device=None):
    """Z = G S [A b] for a HOST column-major A (and host float64 b): row
    blocks are copied to the device while the previous block is sketched;
    returns Z on the host (column-major p x ncol float64).  Page-locked A
    (and b) let the copies overlap the sketch."""
    if A.is_cuda or (b is not None and b.is_cuda):
        raise TypeError("ms_sketch_host takes host tensors")
    d, n = A.shape
    lda = _colmajor(A)
    dt = _dtype_code(A)
    ncol = n + (0 if b is None else 1)
    if b is not None and (b.dtype != torch.float64 or b.numel() != d or not b.is_contiguous()):
        raise ValueError("b must be contiguous float64 of length d")
    if Z is None:
        Z = colmajor(p, ncol, torch.float64, "cpu")
    if Z.is_cuda or Z.dtype != torch.float64:
        raise TypeError("Z must be a host float64 tensor")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    if ws is None:
        ws = workspace(msk_ms_host_workspace(d, n, b is not None, k, p, dt, gemm_prec, chunk_rows), dev)
    _check("ms_sketch_host", load().ms_sketch_host(_ptr(A), dt, d, n, lda, _ptr(b), k, p,
                                                   seed & (2**64 - 1), gemm_prec, _ptr(Z), _colmajor(Z),
                                                   chunk_rows, _ptr(ws), ws.numel(), _stream(stream)))
    return Z


def msk_ms_workspace(d, n, with_b, k, p, dtype, gemm_prec, strategy=CS_ATOMIC):
    return load().msk_ms_workspace(d, n, int(with_b), k, p, dtype, gemm_prec, strategy)


def _event_handle(ev, stream):
    """The cudaEvent_t of a torch.cuda.Event (created by one record if new)."""
    if not ev.cuda_event:
        ev.record(stream)
    return ctypes.c_void_p(ev.cuda_event)


def ms_sketch(A, k, p, seed, b=None, gemm_prec=GEMM_F64, Z=None, strategy=CS_ATOMIC, ws=None,
              stream=None, cs_events=None):
    """Z = G S [A b] (p x ncol, column-major FP64).  cs_events: optional pair
    of torch.cuda.Event recorded around the call's CountSketch."""
    _cuda(A, "A"), _cuda(b, "b")
    d, n = A.shape
    lda = _colmajor(A)
    dt = _dtype_code(A)
    ncol = n + (0 if b is None else 1)
    if Z is None:
        Z = colmajor(p, ncol, torch.float64, A.device)
    need = msk_ms_workspace(d, n, b is not None, k, p, dt, gemm_prec, strategy)
    if ws is None:
        ws = workspace(need, A.device)
    if cs_events is not None:
        s = torch.cuda.current_stream() if stream is None else stream
        load().msk_stage_events(_event_handle(cs_events[0], s), _event_handle(cs_events[1], s))
    _check("ms_sketch", load().ms_sketch(_ptr(A), dt, d, n, lda, _ptr(b), k, p, seed & (2**64 - 1),
                                         gemm_prec, _ptr(Z), _colmajor(Z), strategy, _ptr(ws), ws.numel(),
                                         _stream(stream)))
    return Z


def msk_gemm_workspace(p, k, ncol, gemm_prec):
    return load().msk_gemm_workspace(p, k, ncol, gemm_prec)


def _gemm_operands(p, Y, Z, gemm_prec):
    """Check the Gaussian-stage operands the C side cannot see through its
    void pointers: Y row-major k x ncol on the GPU (unit column stride),
    float64 for GEMM_F64 and float32 for every other precision; Z, when
    given, a column-major p x ncol float64 GPU tensor."""
    if gemm_prec not in _PREC_DTYPE and gemm_prec != GEMM_BF16X3:
        raise ValueError(f"unknown gemm_prec {gemm_prec}")
    if Y.dim() != 2:
        raise ValueError("Y must be 2-D (k x ncol)")
    k, ncol = Y.shape
    want = torch.float64 if gemm_prec == GEMM_F64 else torch.float32
    if Y.dtype != want:
        raise ValueError(f"Y must be {want} for gemm_prec {gemm_prec}, got {Y.dtype}")
    if ncol > 1 and Y.stride(1) != 1:
        raise ValueError("Y must be row-major (stride(1) == 1)")
    if k > 1 and Y.stride(0) < ncol:
        raise ValueError("Y's row pitch stride(0) must be >= ncol")
    if Z is not None:
        if Z.dtype != torch.float64 or tuple(Z.shape) != (p, ncol):
            raise ValueError(f"Z must be float64 of shape ({p}, {ncol})")
        if p > 1 and Z.stride(0) != 1:
            raise ValueError("Z must be column-major (stride(0) == 1)")
        _cuda(Z, "Z")
    _cuda(Y, "Y")
    return k, ncol


def msk_gemm(seed, p, Y, gemm_prec=GEMM_F64, Z=None, ws=None, stream=None):
    """Z = G Y with G the seed's p x k Gaussian; Y row-major k x ncol
    (float64 for GEMM_F64, float32 otherwise)."""
    k, ncol = _gemm_operands(p, Y, Z, gemm_prec)
    _cuda(ws, "ws")
    if Z is None:
        Z = colmajor(p, ncol, torch.float64, Y.device)
    if ws is None:
        ws = workspace(msk_gemm_workspace(p, k, ncol, gemm_prec), Y.device)
    _check("msk_gemm", load().msk_gemm(seed & (2**64 - 1), p, k, ncol, _ptr(Y), Y.stride(0), gemm_prec,
                                       _ptr(Z), _colmajor(Z), _ptr(ws), ws.numel(), _stream(stream)))
    return Z


def msk_gemm_noalloc(seed, p, Y, gemm_prec=GEMM_F64, Z=None, stream=None):
    """msk_gemm with the library's fixed scratch array instead of a caller
    workspace (for callers that may not allocate device memory; Z is still the
    caller's).  Calls share the array: serialise them."""
    k, ncol = _gemm_operands(p, Y, Z, gemm_prec)
    if Z is None:
        Z = colmajor(p, ncol, torch.float64, Y.device)
    _check("msk_gemm_noalloc", load().msk_gemm_noalloc(seed & (2**64 - 1), p, k, ncol, _ptr(Y), Y.stride(0),
                                                       gemm_prec, _ptr(Z), _colmajor(Z), _stream(stream)))
    return Z


def msk_householder_qr(W, stream=None):
    """In-place Householder QR of the m x c column-major FP64 W; returns W."""
    m, c = W.shape
    _check("msk_householder_qr", load().msk_householder_qr(_ptr(W), m, c, _colmajor(W), _stream(stream)))
    return W


def msk_trsv_upper(R, rhs, x=None, stream=None):
    n = R.shape[0]
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=R.device)
    rc = load().msk_trsv_upper(_ptr(R), n, _colmajor(R), _ptr(rhs), _ptr(x), _stream(stream))
    if rc < 0 or rc >= 1000:
        _check("msk_trsv_upper", rc)
    return x, rc


def msk_lstsq_workspace(d, n, k, p, dtype, gemm_prec, refine):
    return load().msk_lstsq_workspace(d, n, k, p, dtype, gemm_prec, int(refine))


def ms_lstsq(A, b, k, p, seed, gemm_prec=GEMM_F64, refine=False, tol=1e-10, max_iter=50, x=None,
             ws=None, stream=None, want_info=True):
    """Multisketched least squares; returns (x, info dict, status)."""
    _cuda(A, "A"), _cuda(b, "b")
    d, n = A.shape
    dt = _dtype_code(A)
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=A.device)
    if ws is None:
        ws = workspace(msk_lstsq_workspace(d, n, k, p, dt, gemm_prec, refine), A.device)
    info = LstsqInfo()
    rc = load().ms_lstsq(_ptr(A), dt, d, n, _colmajor(A), _ptr(b), k, p, seed & (2**64 - 1), gemm_prec,
                         int(refine), tol, max_iter, _ptr(x), ctypes.byref(info) if want_info else None,
                         _ptr(ws), ws.numel(), _stream(stream))
    if rc < 0 or rc in (MSK_ENOMEM, MSK_ECUDA, MSK_ENOTSUP, MSK_ETIMEOUT):
        _check("ms_lstsq", rc)
    return x, {"iters": info.iters, "converged": info.converged, "relres": info.relres,
               "relres_sns": info.relres_sns}, rc


def msk_ne_workspace(d, n):
    return load().msk_ne_workspace(d, n)


def ne_lstsq(A, b, x=None, ws=None, stream=None):
    """Normal-equations least squares; returns (x, status) — status j+1 > 0
    when the Cholesky pivot j is not positive."""
    d, n = A.shape
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=A.device)
    if ws is None:
        ws = workspace(msk_ne_workspace(d, n), A.device)
    rc = load().ne_lstsq(_ptr(A), d, n, _colmajor(A), _ptr(b), _ptr(x), _ptr(ws), ws.numel(), _stream(stream))
    if rc < 0 or rc >= 1000:
        _check("ne_lstsq", rc)
    return x, rc


def msk_normal_apply_workspace(d, n):
    return load().msk_normal_apply_workspace(d, n)


def msk_normal_apply(A, p, v=None, ws=None, stream=None):
    """v = A^T (A p) for FP32 A in double-single arithmetic: the refinement's
    operator pass (after the residual pass that bounds its terms)."""
    _cuda(A, "A")
    d, n = A.shape
    if v is None:
        v = torch.empty(n, dtype=torch.float64, device=A.device)
    if ws is None:
        ws = workspace(msk_normal_apply_workspace(d, n), A.device)
    rc = load().msk_normal_apply(_ptr(A), d, n, _colmajor(A), _ptr(p), _ptr(v), _ptr(ws), ws.numel(),
                                 _stream(stream))
    _check("msk_normal_apply", rc)
    return v


SKETCH_MULTI, SKETCH_COUNT, SKETCH_GAUSS, SKETCH_SRHT = 0, 1, 2, 3


def msk_srht_workspace(d, n, with_b, k):
    return load().msk_srht_workspace(d, n, int(bool(with_b)), k)


def srht_sketch(A, k, seed, b=None, Y=None, ws=None, stream=None):
    """Y = (1/sqrt(k)) P H D [A b] (Section 5), row-major k x (n+1) FP64
    (d a power of two)."""
    _cuda(A, "A")
    d, n = A.shape
    ncol = n + (0 if b is None else 1)
    if Y is None:
        Y = torch.empty((k, ncol), dtype=torch.float64, device=A.device)
    if ws is None:
        ws = workspace(msk_srht_workspace(d, n, b is not None, k), A.device)
    rc = load().srht_sketch(_ptr(A), _dtype_code(A), d, n, _colmajor(A), _ptr(b), k, seed & (2**64 - 1),
                            _ptr(Y), Y.stride(0), _ptr(ws), ws.numel(), _stream(stream))
    _check("srht_sketch", rc)
    return Y


def msk_sns_workspace(d, n, kind, k, p, dtype):
    return load().msk_sns_workspace(d, n, kind, k, p, dtype)


def sns_lstsq(A, b, kind, k, p, seed, x=None, ws=None, stream=None):
    """FP64 sketch-and-solve with S = G C (SKETCH_MULTI), C alone
    (SKETCH_COUNT, k rows) or G alone (SKETCH_GAUSS, p rows); returns
    (x, info dict, status)."""
    _cuda(A, "A"), _cuda(b, "b")
    d, n = A.shape
    dt = _dtype_code(A)
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=A.device)
    if ws is None:
        ws = workspace(msk_sns_workspace(d, n, kind, k, p, dt), A.device)
    info = LstsqInfo()
    rc = load().sns_lstsq(_ptr(A), dt, d, n, _colmajor(A), _ptr(b), kind, k, p, seed & (2**64 - 1),
                          _ptr(x), ctypes.byref(info), _ptr(ws), ws.numel(), _stream(stream))
    if rc < 0 or rc >= 1000:
        _check("sns_lstsq", rc)
    return x, {"iters": info.iters, "converged": info.converged, "relres": info.relres,
               "relres_sns": info.relres_sns}, rc


def msk_rcq_workspace(d, n, k, p, dtype, gemm_prec, want_q=False):
    return load().msk_rcq_workspace(d, n, k, p, dtype, gemm_prec, int(bool(want_q)))


def rcq_lstsq(A, b, k, p, seed, gemm_prec=GEMM_F64, x=None, ws=None, stream=None):
    """rand_cholQR least squares (Algorithm 5); returns (x, info dict, status).
    status j+1 > 0: R0[j][j] == 0 or pivot j of chol(Q0^T Q0) not positive
    (x is NaN)."""
    _cuda(A, "A"), _cuda(b, "b")
    d, n = A.shape
    dt = _dtype_code(A)
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=A.device)
    if ws is None:
        ws = workspace(msk_rcq_workspace(d, n, k, p, dt, gemm_prec), A.device)
    info = LstsqInfo()
    rc = load().rcq_lstsq(_ptr(A), dt, d, n, _colmajor(A), _ptr(b), k, p, seed & (2**64 - 1),
                          gemm_prec, _ptr(x), ctypes.byref(info), _ptr(ws), ws.numel(),
                          _stream(stream))
    if rc < 0 or rc >= 1000:
        _check("rcq_lstsq", rc)
    return x, {"iters": info.iters, "converged": info.converged, "relres": info.relres,
               "relres_sns": info.relres_sns}, rc


def rcq_qr(A, k, p, seed, gemm_prec=GEMM_F64, Q=None, R=None, ws=None, stream=None):
    """rand_cholQR (Algorithm 4): A = Q R.  Q is d x n column-major FP64 (may
    be A itself when A is FP64 column-major); R is n x n column-major upper
    triangular.  Returns (Q, R, status)."""
    _cuda(A, "A")
    d, n = A.shape
    dt = _dtype_code(A)
    if Q is None:
        Q = colmajor(d, n, torch.float64, A.device)
    if R is None:
        R = colmajor(n, n, torch.float64, A.device)
    if ws is None:
        ws = workspace(msk_rcq_workspace(d, n, k, p, dt, gemm_prec, True), A.device)
    rc = load().rcq_qr(_ptr(A), dt, d, n, _colmajor(A), k, p, seed & (2**64 - 1), gemm_prec, _ptr(Q),
                       _colmajor(Q), _ptr(R), _colmajor(R), _ptr(ws), ws.numel(), _stream(stream))
    if rc < 0 or rc >= 1000:
        _check("rcq_qr", rc)
    return Q, R, rc


def _batch_items(problems, xs):
    arr = (BatchItem * len(problems))()
    for j, ((A, bb, seed), x) in enumerate(zip(problems, xs)):
        if A.dtype != torch.float32:
            raise TypeError("batched problems take FP32 A")
        d, n = A.shape
        arr[j] = BatchItem(A.data_ptr(), d, n, _colmajor(A), bb.data_ptr(), seed & (2**64 - 1),
                           x.data_ptr())
    return arr


def msk_batch_workspace(problems, refine=True):
    xs = [None] * len(problems)
    arr = (BatchItem * len(problems))()
    for j, (A, bb, seed) in enumerate(problems):
        d, n = A.shape
        arr[j] = BatchItem(A.data_ptr(), d, n, _colmajor(A), bb.data_ptr(), seed & (2**64 - 1), 0)
    return load().msk_batch_workspace(arr, len(problems), int(refine))


def msk_batch_item_bound(problem, refine=True):
    """Additive upper bound of one problem's part of msk_batch_workspace."""
    A, bb, seed = problem
    d, n = A.shape
    item = BatchItem(A.data_ptr(), d, n, _colmajor(A), bb.data_ptr(), seed & (2**64 - 1), 0)
    return load().msk_batch_item_bound(ctypes.byref(item), int(refine))


def msk_batch_lstsq(problems, refine=True, tol=1e-10, max_iter=10, ws=None, stream=None):
    """Solve [(A, b, seed), ...] (FP32 column-major A, FP64 b on the GPU) in one
    batch.  Returns (xs, infos, status)."""
    dev = problems[0][0].device
    xs = [torch.empty(A.shape[1], dtype=torch.float64, device=dev) for A, _, _ in problems]
    arr = _batch_items(problems, xs)
    if ws is None:
        ws = workspace(load().msk_batch_workspace(arr, len(problems), int(refine)), dev)
    infos = (LstsqInfo * len(problems))()
    rc = load().msk_batch_lstsq(arr, len(problems), int(refine), tol, max_iter, infos, _ptr(ws),
                                ws.numel(), _stream(stream))
    if rc < 0 or rc in (MSK_ENOMEM, MSK_ECUDA, MSK_ENOTSUP, MSK_ETIMEOUT):
        _check("msk_batch_lstsq", rc)
    out = [{"iters": i.iters, "converged": i.converged, "relres": i.relres,
            "relres_sns": i.relres_sns} for i in infos]
    return xs, out, rc


def msk_autotune(problems, refine=True, tol=1e-6, max_iter=4, reps=3, stream=None):
    """Time the registry knobs on the batch [(A, b, seed), ...] and leave the
    fastest values set (msk_autotune); returns the report as a dict."""
    import json

    dev = problems[0][0].device
    xs = [torch.empty(A.shape[1], dtype=torch.float64, device=dev) for A, _, _ in problems]
    arr = _batch_items(problems, xs)
    ws = workspace(load().msk_autotune_workspace(arr, len(problems), int(refine)), dev)
    buf = ctypes.create_string_buffer(1 << 16)
    rc = load().msk_autotune(arr, len(problems), int(refine), tol, max_iter, reps, buf, len(buf), _ptr(ws),
                             ws.numel(), _stream(stream))
    _check("msk_autotune", rc)
    return json.loads(buf.value.decode())


class Server:
    """Thin wrapper of the C request server (ms_server_*)."""

    def __init__(self, mem_budget, workers=2, max_batch=64, refine=True, tol=1e-10, max_iter=10):
        h = ctypes.c_void_p()
        _check("ms_server_create", load().ms_server_create(int(mem_budget), workers, max_batch, int(refine),
                                                           tol, max_iter, ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, A, b, seed, x):
        """Queue (A, b, seed) with output x; returns the ticket."""
        d, n = A.shape
        item = BatchItem(A.data_ptr(), d, n, _colmajor(A), b.data_ptr(), seed & (2**64 - 1), x.data_ptr())
        t = ctypes.c_uint64()
        _check("ms_server_submit", load().ms_server_submit(self._h, ctypes.byref(item), ctypes.byref(t)))
        self._keep[t.value] = (A, b, x)
        return t.value

    def poll(self, ticket):
        """(done, info dict or None, latency seconds or None, status)."""
        done = ctypes.c_int()
        info = LstsqInfo()
        lat = ctypes.c_double()
        rc = load().ms_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(info), ctypes.byref(lat))
        if rc < 0:
            _check("ms_server_poll", rc)
        if not done.value:
            return False, None, None, rc
        self._keep.pop(ticket, None)
        return True, {"iters": info.iters, "converged": info.converged, "relres": info.relres,
                      "relres_sns": info.relres_sns}, lat.value, rc

    def error(self):
        return load().ms_server_error(self._h).decode()

    def wait_all(self):
        _check("ms_server_wait_all", load().ms_server_wait_all(self._h))

    def stats(self):
        s, bt, q = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        load().ms_server_stats(self._h, ctypes.byref(s), ctypes.byref(bt), ctypes.byref(q))
        return {"solved": s.value, "batches": bt.value, "queued": q.value}

    def close(self):
        if self._h:
            load().ms_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
