"""GPU parity of the dense steps and the least-squares solvers against the
oracle: Householder R, triangular solves, sketch-and-solve (same S and G as the
oracle: relative residual within 1e-8 relative), refinement (relative residual
within 1e-8 of the oracle's exact least-squares minimiser, and never above
FP64 sketch-and-solve), normal equations and their breakdown (Section 6.3)."""
import math

import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
EPS64 = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def msk():
    import paper_2508_14209_gb300 as m
    from paper_2508_14209_gb300 import build

    assert torch.cuda.is_available()
    build.build()
    m.load()
    return m


def dev_colmajor(M, msk):
    M = torch.as_tensor(M)
    d, n = M.shape
    out = msk.colmajor(d, n, M.dtype, "cuda")
    out.copy_(M)
    return out


# Shapes whose owned columns fit in shared memory run the on-chip cluster QR;
# (2048, 400) exceeds it and runs the global-memory form; (8192, 65) and
# (40000, 17) are taller than the global form's shared-memory staging of v.
@pytest.mark.parametrize("m,c", [(8, 1), (9, 9), (64, 7), (129, 65), (512, 129), (1024, 257),
                                 (2048, 100), (300, 17), (2048, 400), (8192, 65), (40000, 17)])
def test_householder_r_matches_oracle(msk, orc, m, c):
    Z = np.random.default_rng(m * 7 + c).standard_normal((m, c))
    W = dev_colmajor(Z, msk)
    msk.msk_householder_qr(W)
    Wh = W.cpu().numpy()
    R = Wh[:c, :c]
    Ro = orc.householder_r(Z)
    nz = np.linalg.norm(Z)
    assert np.all(Wh[np.tril_indices(m, -1, c)] == 0.0)
    assert np.allclose(R, Ro, rtol=0, atol=4 * m * EPS64 * nz)
    assert np.allclose(R.T @ R, Z.T @ Z, rtol=0, atol=8 * m * EPS64 * nz * nz)


# The cluster QR's two on-chip forms: the flow form (per-reflector mbarriers,
# deferred updates; the default) and the look-ahead form behind one split
# cluster barrier per column (knob qr.flow = 0) both match the oracle.
@pytest.mark.parametrize("m,c", [(9, 9), (64, 17), (129, 65), (512, 129), (1024, 257), (300, 17),
                                 (40, 40)])
@pytest.mark.parametrize("flow", [0, 1])
def test_householder_forms_match_oracle(msk, orc, m, c, flow):
    Z = np.random.default_rng(m * 13 + c).standard_normal((m, c))
    W = dev_colmajor(Z, msk)
    msk.tune_set("qr.flow", flow)
    try:
        msk.msk_householder_qr(W)
        torch.cuda.synchronize()
    finally:
        msk.tune_clear("qr.flow")
    assert msk.msk_take_timeout() == 0
    Wh = W.cpu().numpy()
    R = Wh[:c, :c]
    nz = np.linalg.norm(Z)
    assert np.all(Wh[np.tril_indices(m, -1, c)] == 0.0)
    assert np.allclose(R, orc.householder_r(Z), rtol=0, atol=4 * m * EPS64 * nz)
    assert np.allclose(R.T @ R, Z.T @ Z, rtol=0, atol=8 * m * EPS64 * nz * nz)


def test_trsv_and_zero_pivot(msk):
    rng = np.random.default_rng(3)
    n = 200
    R = np.triu(rng.standard_normal((n, n))) + 8 * np.eye(n)
    c = rng.standard_normal(n)
    x, rc = msk.msk_trsv_upper(dev_colmajor(R, msk), torch.tensor(c, device="cuda"))
    assert rc == 0
    assert np.allclose(x.cpu().numpy(), np.linalg.solve(R, c), rtol=1e-12, atol=1e-12)
    R[57, 57] = 0.0
    _, rc = msk.msk_trsv_upper(dev_colmajor(R, msk), torch.tensor(c, device="cuda"))
    assert rc == 58


def _problem(d, n, lsig, seed, dtype):
    A, b, _ = inputs.ls_problem(d, n, lsig, seed=seed, dtype=dtype)
    return A, b


@pytest.mark.parametrize("d,n,lsig", [(4096 + 17, 8, -2), (65536, 32, -6), (20000, 64, -10),
                                      (1 << 17, 16, -2)])
def test_sns_f64_matches_oracle(msk, orc, d, n, lsig):
    A, b = _problem(d, n, lsig, 100 + n, torch.float64)
    k, p, seed = 2 * n * n, 4 * n, 0x5EED0003
    x, info, rc = msk.ms_lstsq(dev_colmajor(A, msk), b.cuda(), k, p, seed, msk.GEMM_F64)
    assert rc == 0
    xg = x.cpu().numpy()
    An, bn = A.numpy(), b.numpy()
    xo, ro, _ = orc.sns_lstsq(An, bn, k, p, seed, "f64")
    rg = orc.relres(An, bn, xg)
    assert abs(rg - ro) <= 1e-8 * ro
    assert abs(info["relres"] - rg) <= 1e-8 * rg
    kappa = 10.0 ** (-lsig)
    assert np.linalg.norm(xg - xo) <= 1e3 * kappa * EPS64 * np.linalg.norm(xo) + 1e-300


def test_sns_exact_recovery(msk):
    d, n = 1 << 14, 12
    A, _ = _problem(d, n, -3, 7, torch.float64)
    xt = torch.arange(1, n + 1, dtype=torch.float64)
    b = A @ xt
    x, info, rc = msk.ms_lstsq(dev_colmajor(A, msk), b.cuda(), 2 * n * n, 4 * n, 9, msk.GEMM_F64)
    assert rc == 0
    assert torch.allclose(x.cpu(), xt, rtol=1e-10, atol=0)


# Cases also cover the refinement passes' edges: one partial row tile (d below
# the tile height), d not a multiple of 4, odd leading dimensions (4-byte
# copies instead of 16-byte ones), n not a power of two, and n = 400 (two
# columns per thread in the column phase).
@pytest.mark.parametrize("d,n,lsig,prec,lda_pad,k", [
    (1 << 15, 16, -4, "f32", 0, None), (1 << 15, 32, -8, "f32", 0, None),
    (40000, 64, -6, "f32", 0, None), (500, 16, -5, "f32", 0, None),
    (40003, 100, -7, "bf16x3", 3, None), (30001, 48, -8, "f32", 1, None),
    (6001, 400, -3, "f32", 0, 4000)])
def test_refined_mixed_reaches_minimiser(msk, orc, d, n, lsig, prec, lda_pad, k):
    A, b = _problem(d, n, lsig, 300 + n, torch.float32)
    k, p, seed = k or 2 * n * n, 4 * n, 0x5EED0004
    Ad = msk.colmajor(d, n, torch.float32, "cuda", lda=d + lda_pad)
    Ad.copy_(A)
    x, info, rc = msk.ms_lstsq(Ad, b.cuda(), k, p, seed, msk.GEMM_PRECS[prec],
                               refine=True, tol=1e-12, max_iter=20)
    assert rc == 0, info
    An, bn = A.numpy(), b.numpy()
    xo = orc.lstsq_exact(An, bn)
    ro = orc.relres(An, bn, xo)
    rg = orc.relres(An, bn, x.cpu().numpy())
    assert abs(rg - ro) <= 1e-8 * ro                      # two-sided, against the minimiser
    _, r_sns64, _ = orc.sns_lstsq(An.astype(np.float64), bn, k, p, seed, "f64")
    assert rg <= (1 + 1e-8) * r_sns64                     # never worse than FP64 sketch-and-solve
    assert info["iters"] >= 1 and info["converged"] == 1


@pytest.mark.parametrize("n", [8, 100])
def test_residual_pass_exact_with_subnormal_and_zero_entries(msk, orc, n):
    """The FP64 residual pass widens FP32 entries to FP64 exactly: a column of
    subnormal entries (integers below 2^20 times 2^-149) carrying a solution
    component of 2^130 contributes O(1) to b, so a flushed or misconverted
    subnormal would change the residual the pass reports; zero entries ride
    along."""
    d = 4099
    A, _ = _problem(d, n, -2, 77 + n, torch.float32)
    g = torch.Generator().manual_seed(5)
    A[:, 0] = torch.randint(-2**20, 2**20, (d,), generator=g).to(torch.float32) * 2.0**-149
    A[::3, 1] = 0.0
    assert (A[:, 0].abs() < torch.finfo(torch.float32).tiny).float().mean() > 0.9
    xt = torch.ones(n, dtype=torch.float64)
    xt[0] = 2.0**130
    An = A.numpy().astype(np.float64)
    b = torch.tensor(An @ xt.numpy()) + 1e-3 * torch.randn(d, generator=g, dtype=torch.float64)
    Ad = msk.colmajor(d, n, torch.float32, "cuda", lda=d)
    Ad.copy_(A)
    x, info, rc = msk.ms_lstsq(Ad, b.cuda(), 2 * n * n, 4 * n, 11, msk.GEMM_F64)
    assert rc == 0
    r_orc = orc.relres(An, b.numpy(), x.cpu().numpy())
    assert abs(info["relres"] - r_orc) <= 1e-10 * r_orc


@pytest.mark.parametrize("d,n", [(20000 + 3, 128), (9001, 255), (6000, 256), (3000, 520), (4000, 1),
                                 (9001, 24), (9001, 32), (9001, 10), (9001, 16)])
def test_ne_shapes_match_oracle(msk, orc, d, n):
    """Normal equations across the Gram kernels' layouts: one panel of 2x2
    blocks (129 columns), several panels (256, 257 columns), an odd column
    count with a zero pad column, the 64x64-tile form past 513 columns, a
    single column, and the narrow panels (two slots per thread) with 8, 4 and
    2 row groups per CTA (11 and 17 columns: 8 groups; 25 columns: 4; 33
    columns: 2); kappa = 1e2, so both sides sit at the minimiser."""
    A, b = _problem(d, n, -2, 300 + n, torch.float64)
    x, rc = msk.ne_lstsq(dev_colmajor(A, msk), b.cuda())
    assert rc == 0
    xo, info = orc.ne_lstsq(A.numpy(), b.numpy())
    assert info == 0
    xg = x.cpu().numpy()
    assert np.allclose(xg, xo, rtol=1e-8, atol=1e-8 * np.abs(xo).max())
    rg = orc.relres(A.numpy(), b.numpy(), xg)
    ro = orc.relres(A.numpy(), b.numpy(), xo)
    assert abs(rg - ro) <= 1e-8 * ro


def test_ne_matches_oracle_and_breaks_down(msk, orc):
    d, n = 1 << 14, 10
    A, b = _problem(d, n, -4, 41, torch.float64)
    x, rc = msk.ne_lstsq(dev_colmajor(A, msk), b.cuda())
    assert rc == 0
    xo, info = orc.ne_lstsq(A.numpy(), b.numpy())
    assert info == 0
    assert np.allclose(x.cpu().numpy(), xo, rtol=1e-6, atol=1e-6 * np.abs(xo).max())
    # Section 6.3 sensitivity experiment: d = 2^17, n = 16, b = A e, kappa = 1e10
    d, n = 1 << 17, 16
    A, _ = _problem(d, n, -10, 42, torch.float64)
    b = A @ torch.ones(n, dtype=torch.float64)
    Ad = dev_colmajor(A, msk)
    xn, rc = msk.ne_lstsq(Ad, b.cuda())
    xs, info, rcs = msk.ms_lstsq(Ad, b.cuda(), 2 * n * n, 4 * n, 5, msk.GEMM_F64)
    rs = orc.relres(A.numpy(), b.numpy(), xs.cpu().numpy())
    assert rcs == 0 and rs < 1e-12
    if rc == 0:
        rn = orc.relres(A.numpy(), b.numpy(), xn.cpu().numpy())
        assert rn > 1e3 * rs
    else:
        assert rc > 0 and torch.isnan(xn).all()


# The mixed-precision configuration's Gaussian-stage arms (FP32 A and FP32
# CountSketch; the Gaussian stage in BF16, in FP16, or split-BF16 with
# draining; FP64 QR and residuals), on its shape family scaled down
# (k = 2n^2, p = 4n) at kappa = 1e4 and 1e8.  A single 16-bit rounding of the
# sketch perturbs the preconditioner R by O(u16 kappa(A)), so the refinement
# may run out of steps; each result must then be reported as MSK_ENOCONV and
# still be no worse than FP64 sketch-and-solve of the same request.  A
# converged result sits at the oracle's minimiser (two-sided, 1e-8).
@pytest.mark.parametrize("prec", ["bf16", "f16", "bf16x3"])
@pytest.mark.parametrize("lsig", [-4, -8])
def test_refined_gaussian_stage_arms(msk, orc, prec, lsig):
    d, n = 1 << 16, 64
    A, b = _problem(d, n, lsig, 500 + n, torch.float32)
    k, p, seed = 2 * n * n, 4 * n, 0x5EED0004
    Ad = dev_colmajor(A, msk)
    x, info, rc = msk.ms_lstsq(Ad, b.cuda(), k, p, seed, msk.GEMM_PRECS[prec], refine=True,
                               tol=1e-12, max_iter=20)
    An, bn = A.numpy(), b.numpy()
    ro = orc.relres(An, bn, orc.lstsq_exact(An, bn))
    rg = orc.relres(An, bn, x.cpu().numpy())
    _, r_sns64, _ = orc.sns_lstsq(An.astype(np.float64), bn, k, p, seed, "f64")
    print(f"arm {prec} kappa=1e{-lsig}: status {rc} inner iterations {info['iters']} "
          f"|relres - relres*|/relres* = {abs(rg - ro) / ro:.3e} relres/relres_SnS64 = {rg / r_sns64:.6f}")
    assert abs(info["relres"] - rg) <= 1e-10 * rg
    assert rg <= (1 + 1e-8) * r_sns64
    if rc == msk.MSK_OK:
        assert info["converged"] == 1
        assert abs(rg - ro) <= 1e-8 * ro
    else:
        assert rc == msk.MSK_ENOCONV and info["converged"] == 0, (rc, info)
    if prec == "bf16x3":
        assert rc == msk.MSK_OK   # the draining split-BF16 stage converges at both kappa
