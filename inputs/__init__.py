"""Seeded synthetic inputs shared by the oracle tests, the parity tests and the
benchmark.  This module holds none of the sketching or solving arithmetic:
it only draws the matrices and right-hand sides the method is applied to
(the experiments of Section 6: tall N(0,1) matrices, least-squares problems
with a prescribed singular-value spread, b = A e + noise).

Everything is generated with torch's seeded generators on the requested device,
so the CUDA path and the oracle consume the very same bytes (the oracle gets a
host copy).  The values depend on (seed, shape, device type); a CPU draw and a
CUDA draw of the same seed differ, which is fine because each test or bench
run feeds one draw to both sides.
"""
from __future__ import annotations

import math

import torch

# Row-chunk size of the chunked generators (fixed, so the values do not depend
# on how much memory the caller has).
_CHUNK = 1 << 20


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed) & ((1 << 63) - 1))
    return g


def colmajor_empty(d: int, n: int, dtype, device, lda: int | None = None) -> torch.Tensor:
    """Uninitialised d x n column-major matrix with leading dimension lda."""
    lda = d if lda is None else lda
    assert lda >= d
    buf = torch.empty((max(n, 1), max(lda, 1)), dtype=dtype, device=device)
    return buf[:n, :d].t()


def normal_matrix(d: int, n: int, seed: int, dtype=torch.float64, device="cpu",
                  lda: int | None = None) -> torch.Tensor:
    """d x n column-major matrix of i.i.d. N(0,1) entries (the random test
    matrices of Section 6.2), drawn column by column, rounded to dtype."""
    A = colmajor_empty(d, n, dtype, device, lda)
    g = _gen(seed, device)
    for j in range(n):
        A[:, j] = torch.randn(d, generator=g, device=device, dtype=torch.float64).to(dtype)
    return A


def integer_matrix(d: int, n: int, seed: int, lo: int = -8, hi: int = 8,
                   dtype=torch.float64, device="cpu") -> torch.Tensor:
    """d x n column-major matrix of uniform integers in [lo, hi] (sums of such
    values are exact in floating point)."""
    A = colmajor_empty(d, n, dtype, device)
    g = _gen(seed, device)
    A.copy_(torch.randint(lo, hi + 1, (d, n), generator=g, device=device).to(dtype))
    return A


def haar_orthogonal(n: int, seed: int, device="cpu") -> torch.Tensor:
    """n x n Haar-distributed orthogonal matrix: QR of a Gaussian matrix with
    the signs of diag(R) moved into Q (Mezzadri, Notices AMS 2007).  Drawn and
    factored on the host (it is small), then moved to `device`."""
    g = _gen(seed ^ 0x5A5A5A5A, "cpu")
    M = torch.randn(n, n, generator=g, dtype=torch.float64)
    Q, R = torch.linalg.qr(M)
    sgn = torch.sign(torch.diagonal(R))
    sgn[sgn == 0] = 1
    return (Q * sgn).to(device)


def log_spaced_sigma(n: int, log10_min: float, device="cpu") -> torch.Tensor:
    """sigma_j = 10^(log10_min * j / (n-1)), j = 0..n-1 (1 down to 10^log10_min)."""
    if n == 1:
        return torch.ones(1, dtype=torch.float64, device=device)
    j = torch.arange(n, dtype=torch.float64, device=device)
    return torch.pow(torch.tensor(10.0, dtype=torch.float64, device=device), log10_min * j / (n - 1))


def ls_problem(d: int, n: int, log10_sigma_min: float, seed: int, dtype=torch.float64,
               device="cpu", noise: float = 1e-6, x_true=None):
    """Least-squares test problem A = G diag(sigma) V^T (G with N(0,1/d)
    entries, V Haar orthogonal, sigma log-spaced from 1 to 10^log10_sigma_min)
    stored column-major in dtype, and b = A x_true + noise ||A x_true|| xi/sqrt(d)
    with xi ~ N(0,1) and x_true = e = (1,...,1) (Section 6.3 sets x = e).
    b and A x_true are formed in FP64 from the stored (rounded) A.
    Returns (A, b, x_true)."""
    V = haar_orthogonal(n, seed, device)
    sig = log_spaced_sigma(n, log10_sigma_min, device)
    M = sig.reshape(-1, 1) * V.t()  # diag(sigma) V^T
    A = colmajor_empty(d, n, dtype, device)
    if x_true is None:
        x_true = torch.ones(n, dtype=torch.float64, device=device)
    Ax = torch.empty(d, dtype=torch.float64, device=device)
    g = _gen(seed, device)
    for r0 in range(0, d, _CHUNK):
        r1 = min(d, r0 + _CHUNK)
        Gc = torch.randn(r1 - r0, n, generator=g, device=device, dtype=torch.float64)
        Gc.mul_(1.0 / math.sqrt(d))
        Ac = (Gc @ M).to(dtype)
        A[r0:r1, :] = Ac
        Ax[r0:r1] = Ac.to(torch.float64) @ x_true
    gn = _gen(seed ^ 0x3C3C3C3C, device)
    xi = torch.randn(d, generator=gn, device=device, dtype=torch.float64)
    b = Ax + noise * torch.linalg.vector_norm(Ax) * xi / math.sqrt(d)
    return A, b, x_true


def noisy_rhs(A: torch.Tensor, mu: float, var: float, seed: int):
    """b = A e + eta with eta_i ~ N(mu, var): the "easy" (mu=0, var=0.01) and
    "hard" (mu=3, var=2) right-hand sides of Section 6.3."""
    d, n = A.shape
    e = torch.ones(n, dtype=torch.float64, device=A.device)
    g = _gen(seed ^ 0x77777777, A.device)
    eta = mu + math.sqrt(var) * torch.randn(d, generator=g, device=A.device, dtype=torch.float64)
    return A.to(torch.float64) @ e + eta
