"""Plain, slow FP64 CPU oracle for the CountSketch / multisketch / least-squares
path of arXiv 2508.14209 (Higgins, Boman, Yamazaki).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library; the two meet only through
the seeded input generators in ``inputs/`` and through the written definition
of the counter generator (splitmix64) and of the Gaussian sampler.

The streaming loops (hash, CountSketch, Gaussian matrix, G*Y, Gram, residual)
are plain C in ``msk_oracle.c``; the small dense steps (Householder QR,
triangular solves, Cholesky, the refinement loop) are plain numpy here.  Each
function names the passage of the paper it follows.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  hash / draw          splitmix64 reference stream, chi^2 uniformity, sign balance
  gaussian             moments, Kolmogorov-Smirnov against N(0,1/p), ln accuracy
  countsketch          brute force with the explicit dense S, sum invariant,
                       integer-exact sums
  countsketch_rows     the blocks of a row partition add up to countsketch
                       (integer-exact); row0 = 0 is countsketch itself
  gemm                 integer-exact products, bf16/fp16 rounding definition
  householder_r/solve  R^T R = Z^T Z, |R| against LAPACK's QR, numpy lstsq
  residual / relres /  integer problems whose residual is exact (r = e, norms
    residual_and_g.    as exact integers), x = 0 and b = A x, numpy's FP64
                       evaluation of r, A^T r and the norms, A^T r = 0 at
                       LAPACK's least-squares minimiser
  normal_apply         brute force in exact rational arithmetic (each w_i
                       rounded once), a cancellation case plain FP64 loses
  sns_lstsq            exact recovery for b = A x, distortion bound of Section 2
  ne_lstsq             agrees with QR when well conditioned, fails for
                       kappa > 1e8 (Section 6.3)
  refine               converges to the exact LS minimiser
  fwht / srht          the Hadamard matrix of the recursive definition
                       (scipy.linalg.hadamard), brute force with the explicit
                       dense S, E||S x||^2 = ||x||^2, uniform rows, balanced
                       signs
  sns_lstsq_count/     exact recovery for b = A x, distortion bound, E||S y||^2
    _gauss             = ||y||^2 (sketch scaling), same minimiser class as
                       sns_lstsq
  rand_cholqr          Q^T Q = I, Q R = A, |R| against LAPACK's QR of A
                       (Algorithm 4)
  rand_cholqr_lstsq    the exact LS minimiser (Algorithm 5), at kappa up to
                       1e10 where the normal equations fail
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile msk_oracle.c into liboracle.so next to it (gcc, no -march)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_int = ctypes.c_int


def _declare(L):
    L.or_stream_key.restype = _u64
    L.or_stream_key.argtypes = [_u64, _u64]
    L.or_draw.restype = _u64
    L.or_draw.argtypes = [_u64, _u64]
    L.or_hash.restype = None
    L.or_hash.argtypes = [_u64, _i64, _i64, _i64, _p, _p]
    L.or_srht_signs.restype = None
    L.or_srht_signs.argtypes = [_u64, _i64, _p]
    L.or_srht_rows.restype = None
    L.or_srht_rows.argtypes = [_u64, _i64, _i64, _p]
    L.or_ln_f32.restype = ctypes.c_float
    L.or_ln_f32.argtypes = [ctypes.c_float]
    L.or_gauss_std.restype = ctypes.c_float
    L.or_gauss_std.argtypes = [_u64, _u64]
    L.or_gaussian.restype = None
    L.or_gaussian.argtypes = [_u64, _i64, _i64, _p, _i64]
    L.or_countsketch.restype = _int
    L.or_countsketch.argtypes = [_p, _int, _i64, _i64, _i64, _p, _i64, _u64, _p, _i64]
    L.or_countsketch_buckets.restype = _int
    L.or_countsketch_buckets.argtypes = [_p, _int, _i64, _i64, _i64, _p, _i64, _u64,
                                         _i64, _p, _p, _p, _p]
    L.or_gemm.restype = None
    L.or_gemm.argtypes = [_p, _i64, _p, _i64, _i64, _i64, _i64, _p, _i64]
    L.or_gram.restype = None
    L.or_gram.argtypes = [_p, _int, _i64, _i64, _i64, _p, _p, _p]
    L.or_residual.restype = None
    L.or_residual.argtypes = [_p, _int, _i64, _i64, _i64, _p, _p, _p, _p, _p]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _colmajor(A):
    """Return (array, dtype code, lda) for a column-major (Fortran) view of A."""
    A = np.asarray(A)
    if A.dtype not in (np.float64, np.float32):
        A = A.astype(np.float64)
    if not A.flags.f_contiguous:
        A = np.asfortranarray(A)
    return A, (0 if A.dtype == np.float64 else 1), max(A.shape[0], 1)


# --------------------------------------------------------------------------
# Counter generator and sketch randomness (Definition 3, Section 4; the
# on-the-fly hashed form the paper names as future work in Section 8).

def stream_key(seed: int, tag: int) -> int:
    return int(lib().or_stream_key(seed & (2**64 - 1), tag))


def draw(key: int, i: int) -> int:
    return int(lib().or_draw(key & (2**64 - 1), i))


def hash_rows(seed: int, i0: int, count: int, k: int):
    """Buckets h(i) in [0,k) (uint32) and signs s(i) in {-1,+1} (int8)."""
    h = np.empty(count, dtype=np.uint32)
    s = np.empty(count, dtype=np.int8)
    if count:
        lib().or_hash(seed & (2**64 - 1), i0, count, k, _ptr(h), _ptr(s))
    return h, s


# --------------------------------------------------------------------------
# Gaussian matrix of the multisketch's second stage (Section 1, Section 6.2).

def ln_f32(x: float) -> float:
    return float(lib().or_ln_f32(ctypes.c_float(x)))


def gaussian(seed: int, p: int, k: int) -> np.ndarray:
    """p x k row-major float32 matrix with N(0, 1/p) entries (polar method)."""
    G = np.empty((p, k), dtype=np.float32)
    if p and k:
        lib().or_gaussian(seed & (2**64 - 1), p, k, _ptr(G), k)
    return G


def round_bf16(x) -> np.ndarray:
    """IEEE round-to-nearest-even of float32 values to bfloat16, returned as
    float32 values.  bfloat16 keeps the top 16 bits of binary32; rounding adds
    0x7FFF plus the lowest kept bit, then truncates (ties go to even)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + keep_lsb) >> 16) << 16
    nan = np.isnan(a)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    out = np.where(nan, np.float32(np.nan), out)
    return out.reshape(np.shape(x))


def split_bf16x3(y32) -> np.ndarray:
    """y1 + y2 + y3 for the split of float32 y into three bfloat16 parts
    (Henry, Tang, Heinecke, ARITH 2019): y1 = bf16(y), y2 = bf16(y - y1),
    y3 = bf16(y - y1 - y2), each difference exact in binary32.  Returned as the
    float64 sum (exact: the parts have disjoint significant bits)."""
    y = np.asarray(y32, dtype=np.float32)
    y1 = round_bf16(y)
    r1 = (y - y1).astype(np.float32)
    y2 = round_bf16(r1)
    r2 = (r1 - y2).astype(np.float32)
    y3 = round_bf16(r2)
    return y1.astype(np.float64) + y2.astype(np.float64) + y3.astype(np.float64)


def round_fp16(x) -> np.ndarray:
    """IEEE round-to-nearest-even of float32 values to binary16 (numpy's
    conversion), returned as float32 values."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


# --------------------------------------------------------------------------
# CountSketch (Definition 3 and its row form, Section 4; Algorithm 2 computes
# the same sums with atomics).

def countsketch(A, k: int, seed: int, b=None) -> np.ndarray:
    """Y = S [A b] as a k x ncol row-major FP64 array (ncol = n, or n+1 with b)."""
    A, dt, lda = _colmajor(A)
    d, n = A.shape
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    ncol = n + (0 if bb is None else 1)
    Y = np.empty((k, ncol), dtype=np.float64)
    rc = lib().or_countsketch(_ptr(A), dt, d, n, lda, _ptr(bb), k, seed & (2**64 - 1), _ptr(Y), ncol)
    if rc != 0:
        raise MemoryError("oracle countsketch: out of memory")
    return Y


def countsketch_rows(A, k: int, seed: int, row0: int, b=None) -> np.ndarray:
    """S_r [A b] for a block of rows row0 .. row0+d-1 of a taller matrix,
    hashed with their global indices (Definition 3 restricted to the block;
    the distribution of Section 7): k x ncol FP64, rows added in order."""
    A64 = np.asarray(A, dtype=np.float64)
    X = A64 if b is None else np.hstack([A64, np.asarray(b, dtype=np.float64).reshape(-1, 1)])
    h, s = hash_rows(seed, row0, X.shape[0], k)
    Y = np.zeros((k, X.shape[1]))
    np.add.at(Y, h.astype(np.int64), s.astype(np.float64)[:, None] * X)
    return Y


def countsketch_buckets(A, k: int, seed: int, buckets, b=None):
    """Rows `buckets` of S [A b], their absolute sums and row counts."""
    A, dt, lda = _colmajor(A)
    d, n = A.shape
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    ncol = n + (0 if bb is None else 1)
    lst = np.ascontiguousarray(buckets, dtype=np.int64)
    nb = lst.size
    Yb = np.empty((nb, ncol), dtype=np.float64)
    ab = np.empty((nb, ncol), dtype=np.float64)
    cnt = np.empty(nb, dtype=np.int64)
    rc = lib().or_countsketch_buckets(_ptr(A), dt, d, n, lda, _ptr(bb), k, seed & (2**64 - 1),
                                      nb, _ptr(lst), _ptr(Yb), _ptr(ab), _ptr(cnt))
    if rc != 0:
        raise MemoryError("oracle countsketch_buckets: out of memory")
    return Yb, ab, cnt


def bucket_abs_sums(A, k: int, seed: int, b=None) -> np.ndarray:
    """sum over rows i with h(i)=m of |[A b][i, j]| (k x ncol), the scale of
    the per-entry sketch tolerance."""
    A = np.asarray(A)
    cols = [np.abs(A.astype(np.float64))]
    if b is not None:
        cols.append(np.abs(np.asarray(b, dtype=np.float64)).reshape(-1, 1))
    absAb = np.hstack(cols)
    h, _ = hash_rows(seed, 0, A.shape[0], k)
    out = np.zeros((k, absAb.shape[1]))
    np.add.at(out, h.astype(np.int64), absAb)
    return out


# --------------------------------------------------------------------------
# Gaussian stage Z = G Y (the "Count-Gauss" multisketch, Sections 1 and 6.2).

def gemm(G, Y) -> np.ndarray:
    """Z = G Y with compensated FP64 dot products; returns p x ncol (C order
    array holding the values; the layout of the result is the caller's)."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    p, k = G.shape
    k2, ncol = Y.shape
    assert k == k2
    Zf = np.empty((ncol, p), dtype=np.float64)  # column-major p x ncol
    lib().or_gemm(_ptr(G), k, _ptr(Y), ncol, p, k, ncol, _ptr(Zf), p)
    return np.ascontiguousarray(Zf.T)


def multisketch(A, k: int, p: int, seed: int, b=None, gemm_prec: str = "f64"):
    """Z = G (S [A b]) with the Gaussian and the sketch rounded to the GEMM's
    input precision first ("f64": G widened exactly from float32, Y as is;
    "f32": Y rounded to float32; "bf16"/"f16": G and Y rounded to the 16-bit
    type; "bf16x3": G rounded to bfloat16, float32 Y split into three
    bfloat16 parts).  Returns (Z, G_used, Y_used) as FP64 arrays."""
    Y = countsketch(A, k, seed, b)
    G = gaussian(seed, p, k)
    if gemm_prec == "f64":
        Gu, Yu = G.astype(np.float64), Y
    elif gemm_prec == "f32":
        Gu, Yu = G.astype(np.float64), Y.astype(np.float32).astype(np.float64)
    elif gemm_prec == "bf16":
        Gu = round_bf16(G).astype(np.float64)
        Yu = round_bf16(Y.astype(np.float32)).astype(np.float64)
    elif gemm_prec == "f16":
        Gu = round_fp16(G).astype(np.float64)
        Yu = round_fp16(Y.astype(np.float32)).astype(np.float64)
    elif gemm_prec == "bf16x3":
        Gu = round_bf16(G).astype(np.float64)
        Yu = split_bf16x3(Y.astype(np.float32)).astype(np.float64)
    else:
        raise ValueError(gemm_prec)
    return gemm(Gu, Yu), Gu, Yu


# --------------------------------------------------------------------------
# Small dense steps of Algorithm 1 and of the normal equations (Section 6.3).

def householder_r(Z) -> np.ndarray:
    """R factor of the economy QR of Z (m x c, m >= c) by Householder
    reflections (the GeQRF step of Section 6.1).  Column j: x = W[j:, j],
    v = x + sign(x_0) ||x|| e_0 with sign(0) = +1, W[j:, j:] -= v (2/v^T v)
    (v^T W[j:, j:]); hence R[j, j] = -sign(x_0) ||x||.  Returns c x c upper
    triangular."""
    W = np.array(Z, dtype=np.float64, copy=True)
    m, c = W.shape
    assert m >= c
    for j in range(c):
        x = W[j:, j].copy()
        alpha = float(np.sqrt(np.dot(x, x)))
        sgn = 1.0 if x[0] >= 0 else -1.0
        v = x
        v[0] += sgn * alpha
        vtv = float(np.dot(v, v))
        if vtv > 0.0:
            W[j:, j:] -= np.outer(v, (2.0 / vtv) * (v @ W[j:, j:]))
        W[j, j] = -sgn * alpha
        W[j + 1:, j] = 0.0
    return np.triu(W[:c, :c])


def back_substitution(R, c) -> np.ndarray:
    """x with R x = c, R upper triangular (the TRSV of Algorithm 1, step 3)."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (c[i] - np.dot(R[i, i + 1:], x[i + 1:])) / R[i, i]
    return x


def forward_substitution_transposed(R, c) -> np.ndarray:
    """y with R^T y = c, R upper triangular."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (c[i] - np.dot(R[:i, i], y[:i])) / R[i, i]
    return y


def cholesky_upper(Gm):
    """Upper R with R^T R = Gm (the POTRF of Section 6.3), column by column.
    Returns (R, info): info = 0, or j+1 when pivot j is not positive."""
    Gm = np.asarray(Gm, dtype=np.float64)
    n = Gm.shape[0]
    R = np.zeros((n, n))
    for j in range(n):
        s = Gm[j, j] - np.dot(R[:j, j], R[:j, j])
        if not (s > 0.0):
            return R, j + 1
        R[j, j] = np.sqrt(s)
        for c in range(j + 1, n):
            R[j, c] = (Gm[j, c] - np.dot(R[:j, j], R[:j, c])) / R[j, j]
    return R, 0


def lstsq_from_sketch(W):
    """Algorithm 1 steps 2-3 on a sketched [SA Sb] (m x (n+1)): the R of the
    augmented matrix holds R11 = R[:n, :n] and Q^T z = R[:n, n] (applying the
    reflectors of SA to Sb, the OrMQR step), then x = R11^{-1} (Q^T z)."""
    R = householder_r(W)
    n = W.shape[1] - 1
    return back_substitution(R[:n, :n], R[:n, n]), R


def residual(A, b, x):
    """(||b - A x||, ||b||) with compensated sums (relres definition of
    Section 6.3)."""
    A, dt, lda = _colmajor(A)
    d, n = A.shape
    bb = np.ascontiguousarray(b, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(2)
    lib().or_residual(_ptr(A), dt, d, n, lda, _ptr(bb), _ptr(xx), None, None, _ptr(out))
    return float(np.sqrt(out[0])), float(np.sqrt(out[1]))


def relres(A, b, x) -> float:
    r, bn = residual(A, b, x)
    return r / bn


def residual_and_gradient(A, b, x):
    """r = b - A x and g = A^T r, both compensated."""
    A, dt, lda = _colmajor(A)
    d, n = A.shape
    bb = np.ascontiguousarray(b, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    r = np.empty(d)
    g = np.empty(n)
    out = np.zeros(2)
    lib().or_residual(_ptr(A), dt, d, n, lda, _ptr(bb), _ptr(xx), _ptr(r), _ptr(g), _ptr(out))
    return r, g, float(np.sqrt(out[0])), float(np.sqrt(out[1]))


def _split26(x):
    """x = hi + lo exactly, each part with at most 26 significant bits
    (Veltkamp's splitting with the factor 2^27 + 1), so that a binary32
    times either part is exact in FP64."""
    x = np.asarray(x, dtype=np.float64)
    c = (2.0 ** 27 + 1.0) * x
    hi = c - (c - x)
    return hi, x - hi


def normal_apply(A, p):
    """v = A^T (A p) for a binary32 A: the operator of the preconditioned
    normal equations the refinement iterates on (Section 6.3).  w_i = sum_j
    a_ij p_j and then v_j = sum_i a_ij w_i, each sum the correctly rounded
    FP64 value of its exact terms: a times the two 26-bit parts of the FP64
    factor are exact products, and math.fsum rounds their exact sum once.
    The only error left is the rounding of each w_i."""
    import math

    A64 = np.asarray(A, dtype=np.float32).astype(np.float64)
    d, n = A64.shape
    ph, pl = _split26(p)
    P = np.concatenate((A64 * ph, A64 * pl), axis=1)
    w = np.array([math.fsum(row) for row in P.tolist()])
    wh, wl = _split26(w)
    Q = np.concatenate((A64 * wh[:, None], A64 * wl[:, None]), axis=0)
    return np.array([math.fsum(col) for col in Q.T.tolist()])


def sns_lstsq(A, b, k: int, p: int, seed: int, gemm_prec: str = "f64"):
    """Multisketched sketch-and-solve least squares (Algorithm 1 with
    S = G C: CountSketch C to k rows, Gaussian G to p rows).  Returns
    (x, relres, R) with R the (n+1) x (n+1) factor of [SA Sb]."""
    Z, _, _ = multisketch(A, k, p, seed, b=b, gemm_prec=gemm_prec)
    x, R = lstsq_from_sketch(Z)
    return x, relres(A, b, x), R


# --------------------------------------------------------------------------
# Randomized Cholesky QR (Section 6.3, Algorithms 4 and 5).

def _right_solve_upper(X, U):
    """X U^{-1} for upper-triangular U (a triangular solve per row of X)."""
    import scipy.linalg

    return scipy.linalg.solve_triangular(np.asarray(U, dtype=np.float64),
                                         np.asarray(X, dtype=np.float64).T,
                                         trans="T", lower=False).T


def rand_cholqr(A, k: int, p: int, seed: int, gemm_prec: str = "f64"):
    """Algorithm 4 with the multisketch S = G C: Y = S A; R0 = R of the
    economy QR of Y (Householder, as householder_r); Q0 = A R0^{-1};
    G = Q0^T Q0; R1 = chol(G); Q = Q0 R1^{-1}; R = R1 R0.
    Returns (Q, R, info) with info = j+1 when pivot j of chol(G) is not
    positive (Q and R are then None)."""
    A64 = np.asarray(A, dtype=np.float64)
    Y, _, _ = multisketch(A, k, p, seed, gemm_prec=gemm_prec)
    R0 = householder_r(Y)
    Q0 = _right_solve_upper(A64, R0)
    R1, info = cholesky_upper(Q0.T @ Q0)
    if info:
        return None, None, info
    Q = _right_solve_upper(Q0, R1)
    return Q, np.triu(R1 @ R0), 0


def rand_cholqr_lstsq(A, b, k: int, p: int, seed: int, gemm_prec: str = "f64"):
    """Algorithm 5: Y = S A; R0 from qr(Y); Q0 = A R0^{-1}; G = Q0^T Q0 and
    z = Q0^T b; R1 = chol(G); R = R1 R0; y = R1^{-T} z; x = R^{-1} y.
    Returns (x, info); x is NaN when chol(G) fails (info = j+1)."""
    A64 = np.asarray(A, dtype=np.float64)
    bb = np.asarray(b, dtype=np.float64)
    Y, _, _ = multisketch(A, k, p, seed, gemm_prec=gemm_prec)
    R0 = householder_r(Y)
    Q0 = _right_solve_upper(A64, R0)
    R1, info = cholesky_upper(Q0.T @ Q0)
    if info:
        return np.full(A64.shape[1], np.nan), info
    z = Q0.T @ bb
    R = np.triu(R1 @ R0)
    y = forward_substitution_transposed(R1, z)
    return back_substitution(R, y), 0


# --------------------------------------------------------------------------
# SRHT (Section 5): S = (1/sqrt(k)) P H_d D.

def srht_signs(seed: int, d: int) -> np.ndarray:
    """Diagonal of D (int8 +-1): -1 when bit 0 of draw i of stream tag 5 is set."""
    s = np.empty(d, dtype=np.int8)
    lib().or_srht_signs(seed & (2**64 - 1), d, _ptr(s))
    return s


def srht_rows(seed: int, k: int, d: int) -> np.ndarray:
    """Rows of H D x that P samples (uint32, uniform in [0, d), with
    replacement): multiply-shift of draw l of stream tag 6."""
    j = np.empty(k, dtype=np.uint32)
    lib().or_srht_rows(seed & (2**64 - 1), k, d, _ptr(j))
    return j


def fwht(X) -> np.ndarray:
    """H_d X for the Hadamard matrix of the recursive definition
    (H_2 = [[1, 1], [1, -1]], H_2l = [[H_l, H_l], [H_l, -H_l]]): the fast
    Walsh-Hadamard transform, one radix-2 butterfly stage per power of two,
    applied to every column of X (d x n, d a power of two)."""
    X = np.array(X, dtype=np.float64, copy=True)
    d = X.shape[0]
    assert d >= 1 and d & (d - 1) == 0
    rest = X.shape[1:]
    h = 1
    while h < d:
        V = X.reshape((d // (2 * h), 2, h) + rest)
        a = V[:, 0].copy()
        V[:, 0] += V[:, 1]
        V[:, 1] = a - V[:, 1]
        X = V.reshape((d,) + rest)
        h *= 2
    return X


def srht(A, k: int, seed: int, b=None) -> np.ndarray:
    """Y = (1/sqrt(k)) P H_d D [A b] (Section 5), k x (n+1), FP64: D's signs
    applied to the rows, the fast Walsh-Hadamard transform of every column,
    the sampled rows divided by sqrt(k)."""
    A64 = np.asarray(A, dtype=np.float64)
    X = A64 if b is None else np.hstack([A64, np.asarray(b, dtype=np.float64).reshape(-1, 1)])
    d = X.shape[0]
    X = srht_signs(seed, d).astype(np.float64)[:, None] * X
    return fwht(X)[srht_rows(seed, k, d).astype(np.int64)] / np.sqrt(np.float64(k))


def sns_lstsq_srht(A, b, k: int, seed: int):
    """Algorithm 1 with S the SRHT.  Returns (x, relres, R)."""
    x, R = lstsq_from_sketch(srht(A, k, seed, b))
    return x, relres(A, b, x), R


def sns_lstsq_count(A, b, k: int, seed: int):
    """Algorithm 1 with S = C alone: the k x d CountSketch (Definition 3) of
    [A b], then the Householder QR and triangular solve of the k x (n+1)
    result.  Returns (x, relres, R)."""
    W = countsketch(A, k, seed, b)
    x, R = lstsq_from_sketch(W)
    return x, relres(A, b, x), R


def gaussian_sketch(A, p: int, seed: int, b=None) -> np.ndarray:
    """G [A b] for the p x d Gaussian sketch (Section 1) whose entries are the
    multisketch's Gaussian at k = d: gaussian(seed, p, d)."""
    A64 = np.asarray(A, dtype=np.float64)
    X = A64 if b is None else np.hstack([A64, np.asarray(b, dtype=np.float64).reshape(-1, 1)])
    return gemm(gaussian(seed, p, A64.shape[0]).astype(np.float64), X)


def sns_lstsq_gauss(A, b, p: int, seed: int):
    """Algorithm 1 with S = G alone (p x d Gaussian).  Returns (x, relres, R)."""
    x, R = lstsq_from_sketch(gaussian_sketch(A, p, seed, b))
    return x, relres(A, b, x), R


def gram(A, b):
    """(A^T A, A^T b) with compensated dot products."""
    A, dt, lda = _colmajor(A)
    d, n = A.shape
    bb = np.ascontiguousarray(b, dtype=np.float64)
    Gm = np.empty((n, n), dtype=np.float64, order="F")
    y = np.empty(n)
    lib().or_gram(_ptr(A), dt, d, n, lda, _ptr(bb), _ptr(Gm), _ptr(y))
    return np.array(Gm), y


def ne_lstsq(A, b):
    """Normal equations (Section 6.3): A^T A = R^T R (Cholesky), then
    x = R^{-1} (R^{-T} A^T b).  Returns (x, info); info > 0 when the Gram
    matrix is not numerically positive definite."""
    Gm, y = gram(A, b)
    R, info = cholesky_upper(Gm)
    if info:
        return np.full(Gm.shape[0], np.nan), info
    return back_substitution(R, forward_substitution_transposed(R, y)), 0


def lstsq_exact(A, b):
    """Least-squares minimiser of the stored A by Householder QR of the full
    [A b] (the textbook QR solver the paper compares against, Section 6.3)."""
    A = np.asarray(A, dtype=np.float64)
    W = np.hstack([A, np.asarray(b, dtype=np.float64).reshape(-1, 1)])
    x, _ = lstsq_from_sketch(W)
    return x


def refine(A, b, R, x0, max_iter: int = 100, tol: float = 1e-10):
    """Sketch-and-precondition refinement: preconditioned conjugate gradients
    on the normal equations (CGLS) with right preconditioner R from the sketch
    (the Blendenpik/LSRN family the paper cites in Section 6).  In FP64 with
    compensated residuals:
        r = b - A x;  s = R^{-T} A^T r;  q = s;  gamma = s.s
        repeat:  t = R^{-1} q;  w = A t;  alpha = gamma / w.w
                 x += alpha t;  r = b - A x  (recomputed, compensated)
                 s = R^{-T} A^T r;  gamma' = s.s;  q = s + (gamma'/gamma) q
    until relres changes by at most tol * relres.  Returns (x, relres
    history)."""
    A64 = np.asarray(A, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    r, g, rn, bn = residual_and_gradient(A, b, x)
    s = forward_substitution_transposed(R, g)
    q = s.copy()
    gamma = float(np.dot(s, s))
    hist = [rn / bn]
    for _ in range(max_iter):
        if gamma == 0.0:
            break
        t = back_substitution(R, q)
        w = A64 @ t
        alpha = gamma / float(np.dot(w, w))
        x = x + alpha * t
        r, g, rn, _ = residual_and_gradient(A, b, x)
        hist.append(rn / bn)
        s = forward_substitution_transposed(R, g)
        gamma_new = float(np.dot(s, s))
        q = s + (gamma_new / gamma) * q
        gamma = gamma_new
        if abs(hist[-2] - hist[-1]) <= tol * hist[-1]:
            break
    return x, hist
