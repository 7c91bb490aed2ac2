"""Single-kernel-family cases for profiling and timing (ncu, CUDA events).

    python -m paper_2508_14209_gb300.cases sketch  --d 1048576 --n 64 --dtype f64
    python -m paper_2508_14209_gb300.cases gemm    --p 1024 --k 32768 --ncol 257 --prec bf16x3
    python -m paper_2508_14209_gb300.cases refined --d 1333142 --n 128 --log10-sigma -2.7 [--path single]
    python -m paper_2508_14209_gb300.cases ne      --d 8388608 --n 128 --log10-sigma -6
    python -m paper_2508_14209_gb300.cases sns     --d 8388608 --n 128 --log10-sigma -6 [--kind count|gauss|srht]
    python -m paper_2508_14209_gb300.cases rcq     --d 8388608 --n 128 --log10-sigma -6
    python -m paper_2508_14209_gb300.cases srht    --d 8388608 --n 128
    python -m paper_2508_14209_gb300.cases qr      --p 512 --ncol 129
    python -m paper_2508_14209_gb300.cases batchmix --nprob 32 [--tol 1e-7]

Each case draws its seeded synthetic input once on the GPU (the generators of
the `inputs` module), runs the library call `--reps` times and prints one JSON
line with the mean device time per call (CUDA events on the current stream).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv=None):
    import torch

    import inputs
    import paper_2508_14209_gb300 as msk

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["sketch", "gemm", "refined", "ne", "sns", "rcq", "srht", "host", "qr",
                                     "batchmix"])
    ap.add_argument("--nprob", type=int, default=32,
                    help="batchmix: requests in the batch (n cycling 16, 32, 64, 128; d log-uniform in "
                         "[2^14, 2^21]; FP32 A with sigma from 1 to 10^log10-sigma)")
    ap.add_argument("--d", type=int, default=1 << 20)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--p", type=int, default=1024)
    ap.add_argument("--k", type=int, default=32768)
    ap.add_argument("--ncol", type=int, default=257)
    ap.add_argument("--prec", default="bf16x3", choices=sorted(msk.GEMM_PRECS))
    ap.add_argument("--log10-sigma", type=float, default=-4.0)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--path", choices=["batch", "single", "plain"], default="batch",
                    help="refined: msk_batch_lstsq of one request (its inner loop runs inside a "
                         "graph's while node), ms_lstsq (the same kernels launched one by one), or "
                         "plain: FP64 sketch-and-solve of the same stored FP32 A (ms_lstsq, MSK_GEMM_F64, "
                         "no refinement), the served comparison's plain path")
    ap.add_argument("--kind", choices=["multi", "count", "gauss", "srht"], default="multi",
                    help="sns: the sketch (multisketch G C, CountSketch C alone, Gaussian G alone)")
    ap.add_argument("--chunk-rows", type=int, default=0, help="host: rows per staged block (0: ~256 MiB)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0x5EED0004)
    ap.add_argument("--tune", action="append", default=[], metavar="KNOB=VALUE",
                    help="set a tuning-registry knob before the run (repeatable)")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    msk.load()
    for kv in a.tune:
        name, value = kv.split("=", 1)
        msk.tune_set(name, int(value))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {"case": a.case, "tune": a.tune}
    if a.case == "sketch":
        dt = torch.float64 if a.dtype == "f64" else torch.float32
        A = inputs.normal_matrix(a.d, a.n, a.seed, dtype=dt, device=dev)
        k = 2 * a.n * a.n
        Y = torch.empty((k, a.n), dtype=dt, device=dev)
        call = lambda: msk.cs_sketch(A, k, a.seed, Y=Y)  # noqa: E731
        out.update(d=a.d, n=a.n, k=k, dtype=a.dtype, bytes_per_call=a.d * a.n * A.element_size())
    elif a.case == "host":
        # multisketch of a page-locked HOST A (FP64 Gaussian stage), streamed
        # in row blocks: host-to-device copies overlap the CountSketch
        dt = torch.float64 if a.dtype == "f64" else torch.float32
        Ad = inputs.normal_matrix(a.d, a.n, a.seed, dtype=dt, device=dev)
        buf = torch.empty((a.n, a.d), dtype=dt, pin_memory=True)
        buf.copy_(Ad.t())
        A = buf.t()
        del Ad
        k, p = 2 * a.n * a.n, 4 * a.n
        Zh = torch.empty((a.n, p), dtype=torch.float64, pin_memory=True).t()
        ws = msk.workspace(msk.msk_ms_host_workspace(a.d, a.n, False, k, p, msk.MSK_F64 if a.dtype == "f64"
                                                     else msk.MSK_F32, msk.GEMM_F64, a.chunk_rows), dev)
        call = lambda: msk.ms_sketch_host(A, k, p, a.seed, gemm_prec=msk.GEMM_F64, Z=Zh,  # noqa: E731
                                          chunk_rows=a.chunk_rows, ws=ws)
        out.update(d=a.d, n=a.n, k=k, p=p, dtype=a.dtype, chunk_rows=a.chunk_rows,
                   bytes_per_call=a.d * a.n * buf.element_size())
    elif a.case == "srht":
        # SRHT of A (d a power of two) to k = 2 n^2 rows: FP64 adds, d n log2(d)
        A = inputs.normal_matrix(a.d, a.n, a.seed, dtype=torch.float64, device=dev)
        k = 2 * a.n * a.n
        Y = torch.empty((k, a.n), dtype=torch.float64, device=dev)
        ws = msk.workspace(msk.msk_srht_workspace(a.d, a.n, False, k), dev)
        call = lambda: msk.srht_sketch(A, k, a.seed, Y=Y, ws=ws)  # noqa: E731
        m = a.d.bit_length() - 1
        out.update(d=a.d, n=a.n, k=k, adds_per_call=a.d * a.n * m)
    elif a.case == "batchmix":
        # one batch shaped like the served trace: msk_batch_lstsq, refined
        import numpy as np

        rng = np.random.default_rng(a.seed)
        prob = []
        for j in range(a.nprob):
            n = (16, 32, 64, 128)[j % 4]
            d = int(2 ** rng.uniform(14, 21))
            A, b, _ = inputs.ls_problem(d, n, a.log10_sigma, seed=a.seed + j, dtype=torch.float32, device=dev)
            prob.append((A, b, a.seed + j))
        ws = msk.workspace(msk.msk_batch_workspace(prob, True), dev)
        res = {}

        def call():
            r = msk.msk_batch_lstsq(prob, refine=True, tol=a.tol, max_iter=4, ws=ws)
            res["r"] = {"converged": sum(int(i["converged"]) for i in r[1]),
                        "inner_iters_mean": float(np.mean([i["iters"] for i in r[1]]))}
        out.update(nprob=a.nprob, tol=a.tol, rows=sum(p_[0].shape[0] for p_ in prob),
                   bytes_per_pass=sum(p_[0].shape[0] * p_[0].shape[1] * 4 for p_ in prob))
    elif a.case == "qr":
        # Householder QR of a p x ncol FP64 matrix (the sketched [SA Sb]),
        # restored from a saved copy before every call (copy included)
        Z0 = inputs.normal_matrix(a.p, a.ncol, a.seed, dtype=torch.float64, device=dev)
        W = msk.colmajor(a.p, a.ncol, torch.float64, dev)

        def call():
            W.copy_(Z0)
            msk.msk_householder_qr(W)
        out.update(p=a.p, ncol=a.ncol, flops_per_call=2 * a.p * a.ncol ** 2 - 2 * a.ncol ** 3 // 3)
    elif a.case == "gemm":
        prec = msk.GEMM_PRECS[a.prec]
        ydt = torch.float64 if prec == msk.GEMM_F64 else torch.float32
        Y = inputs.normal_matrix(a.k, a.ncol, a.seed, dtype=ydt, device=dev)
        Yr = torch.empty((a.k, a.ncol), dtype=ydt, device=dev)  # row-major k x ncol
        Yr.copy_(Y)
        Z = msk.colmajor(a.p, a.ncol, torch.float64, dev)
        ws = msk.workspace(msk.msk_gemm_workspace(a.p, a.k, a.ncol, prec), dev)
        call = lambda: msk.msk_gemm(a.seed, a.p, Yr, gemm_prec=prec, Z=Z, ws=ws)  # noqa: E731
        out.update(p=a.p, k=a.k, ncol=a.ncol, prec=a.prec, flops_per_call=2 * a.p * a.k * a.ncol)
    elif a.case in ("ne", "sns", "rcq"):
        # FP64 normal equations (Gram of [A b], Cholesky, two TRSV) or FP64
        # multisketch sketch-and-solve (k = 2n^2, p = 4n) on the same request
        A, b, _ = inputs.ls_problem(a.d, a.n, a.log10_sigma, seed=a.seed, dtype=torch.float64, device=dev)
        res = {}
        if a.case == "ne":
            ws = msk.workspace(msk.msk_ne_workspace(a.d, a.n), dev)

            def call():
                res["r"] = {"status": msk.ne_lstsq(A, b, ws=ws)[1]}
            out.update(flops_per_call=a.d * (a.n + 1) * (a.n + 2))  # upper triangle incl. diagonal
        elif a.case == "rcq":
            # rand_cholQR least squares (Algorithm 5): sketch, QR, Q0 = A R0^{-1},
            # Gram of [Q0 b], Cholesky, two triangular solves
            k, p = 2 * a.n * a.n, 4 * a.n
            ws = msk.workspace(msk.msk_rcq_workspace(a.d, a.n, k, p, msk.MSK_F64, msk.GEMM_F64), dev)

            def call():
                x, info, rc = msk.rcq_lstsq(A, b, k, p, a.seed, msk.GEMM_F64, ws=ws)
                res["r"] = dict(info, status=rc)
            # Q0: n(n+1)/2 FMAs per row; Gram of [Q0 b]: (n+1)(n+2)/2 per row
            out.update(flops_per_call=a.d * (a.n * (a.n + 1) + (a.n + 1) * (a.n + 2)))
        else:
            k, p = 2 * a.n * a.n, 4 * a.n
            kind = {"multi": msk.SKETCH_MULTI, "count": msk.SKETCH_COUNT, "gauss": msk.SKETCH_GAUSS,
                    "srht": msk.SKETCH_SRHT}[a.kind]
            ws = msk.workspace(msk.msk_sns_workspace(a.d, a.n, kind, k, p, msk.MSK_F64), dev)

            def call():
                x, info, rc = msk.sns_lstsq(A, b, kind, k, p, a.seed, ws=ws)
                res["r"] = dict(info, status=rc)
            out.update(kind=a.kind)
        out.update(d=a.d, n=a.n, log10_sigma=a.log10_sigma)
    else:
        A, b, _ = inputs.ls_problem(a.d, a.n, a.log10_sigma, seed=a.seed, dtype=torch.float32, device=dev)
        res = {}
        if a.path == "batch":
            prob = [(A, b, a.seed)]
            ws = msk.workspace(msk.msk_batch_workspace(prob, True), dev)

            def call():
                r = msk.msk_batch_lstsq(prob, refine=True, tol=a.tol, max_iter=4, ws=ws)
                res["r"] = r[1][0]
        elif a.path == "plain":
            k, p = 2 * a.n * a.n, 4 * a.n
            ws = msk.workspace(msk.msk_lstsq_workspace(a.d, a.n, k, p, msk.MSK_F32, msk.GEMM_F64, 0), dev)

            def call():
                res["r"] = msk.ms_lstsq(A, b, k, p, a.seed, msk.GEMM_F64, ws=ws)[1]
        else:
            k, p = 2 * a.n * a.n, 4 * a.n
            ws = msk.workspace(msk.msk_lstsq_workspace(a.d, a.n, k, p, msk.MSK_F32, msk.GEMM_BF16X3, 1), dev)

            def call():
                res["r"] = msk.ms_lstsq(A, b, k, p, a.seed, msk.GEMM_BF16X3, refine=True, tol=a.tol,
                                        max_iter=4, ws=ws)[1]

        out.update(d=a.d, n=a.n, tol=a.tol, path=a.path, bytes_per_pass=a.d * a.n * 4)
    call()
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(a.reps):
        call()
    ev[1].record()
    torch.cuda.synchronize()
    out["ms_per_call"] = round(ev[0].elapsed_time(ev[1]) / a.reps, 5)
    if a.case in ("refined", "ne", "sns", "rcq", "batchmix"):
        out["info"] = res["r"]
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
