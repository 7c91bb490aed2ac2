"""Run by tests/test_gpu_checked.py in a child process whose MSK_LIB names the
checked build: a few calls of every checked kernel family on odd shapes,
each compared with the oracle, and msk_check_status() == 0 after each.
Prints one line per case; exits non-zero on the first mismatch."""
import sys

import numpy as np
import torch

import inputs
import oracle
import paper_2508_14209_gb300 as msk

EPS64 = np.finfo(np.float64).eps


def check(name):
    st = msk.msk_check_status()
    print(f"{name}: check status {st}", flush=True)
    if st != 0:
        sys.exit(3)


def main():
    oracle.build()
    msk.load()
    assert msk.msk_checked_build(), "MSK_LIB does not name the checked build"
    # CountSketch, FP64 and FP32, odd sizes and widths (fixed-width, narrow and
    # generic kernels)
    for d, n, k, dt in [(5001, 7, 98, torch.float64), (40000, 64, 8192, torch.float64),
                        (30001, 16, 512, torch.float64), (20000, 33, 2178, torch.float32),
                        (9000, 128, 4096, torch.float32)]:
        A = inputs.normal_matrix(d, n, 7 + n, dtype=dt)
        Ad = msk.colmajor(d, n, dt, "cuda")
        Ad.copy_(A)
        Y = msk.cs_sketch(Ad, k, 11).double().cpu().numpy()
        Yo = oracle.countsketch(A.numpy(), k, 11)
        absY = oracle.bucket_abs_sums(A.numpy(), k, 11)
        u = 64 * EPS64 if dt == torch.float64 else 1e-5
        assert np.all(np.abs(Y - Yo) <= u * absY), (d, n, k)
        check(f"cs_sketch {d}x{n} k={k} {dt}")
    # FP64 multisketch through the sliced tensor-core stage (k >= 1024)
    d, n, k, p = 12000, 64, 2048, 130
    A = inputs.normal_matrix(d, n, 3, dtype=torch.float64)
    Ad = msk.colmajor(d, n, torch.float64, "cuda")
    Ad.copy_(A)
    Z = msk.ms_sketch(Ad, k, p, 5, gemm_prec=msk.GEMM_F64).cpu().numpy()
    Zo, Gu, Yu = oracle.multisketch(A.numpy(), k, p, 5, gemm_prec="f64")
    absY = oracle.bucket_abs_sums(A.numpy(), k, 5)
    bound = (k + 2) * EPS64 * (np.abs(Gu) @ np.abs(Yu)) + np.abs(Gu) @ (64 * EPS64 * absY)
    assert np.all(np.abs(Z - Zo) <= bound)
    check(f"ms_sketch f64 {d}x{n} k={k} p={p}")
    # refined mixed-precision solve and a small batch
    A, b, _ = inputs.ls_problem(20001, 32, -6, seed=9, dtype=torch.float32)
    Ad = msk.colmajor(20001, 32, torch.float32, "cuda")
    Ad.copy_(A)
    x, info, rc = msk.ms_lstsq(Ad, b.cuda(), 2048, 128, 13, msk.GEMM_BF16X3, refine=True, tol=1e-12,
                               max_iter=20)
    An, bn = A.numpy(), b.numpy()
    ro = oracle.relres(An, bn, oracle.lstsq_exact(An, bn))
    assert rc == 0 and abs(oracle.relres(An, bn, x.cpu().numpy()) - ro) <= 1e-8 * ro
    check("ms_lstsq refined 20001x32")
    probs = []
    for j, (d, n) in enumerate([(5000, 16), (9001, 64), (7000, 32)]):
        A, b, _ = inputs.ls_problem(d, n, -4, seed=20 + j, dtype=torch.float32)
        Ad = msk.colmajor(d, n, torch.float32, "cuda")
        Ad.copy_(A)
        probs.append((Ad, b.cuda(), 30 + j, A.numpy(), b.numpy()))
    xs, infos, rc = msk.msk_batch_lstsq([(A, b, s) for A, b, s, _, _ in probs], refine=True, tol=1e-12,
                                        max_iter=10)
    assert rc == 0
    for (A, b, s, An, bn), x in zip(probs, xs):
        ro = oracle.relres(An, bn, oracle.lstsq_exact(An, bn))
        assert abs(oracle.relres(An, bn, x.cpu().numpy()) - ro) <= 1e-8 * ro
    check("msk_batch_lstsq 3 problems")
    print("checked build: all cases passed", flush=True)


if __name__ == "__main__":
    main()
