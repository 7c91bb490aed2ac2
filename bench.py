"""Benchmark of the multisketch hot path on one GB300 (or N replicas).

Workload (default): a 4194304 x 64 FP64 matrix with N(0,1) entries, CountSketch
to k = 2n^2 = 8192 rows, then the p = 4n = 256 row Gaussian sketch in FP64
(the paper's multisketch, Section 6.2).  One step = the CountSketch (zero Y,
hashed scatter-add of A) and the FP64 Gaussian stage Z = G Y (G sliced on the
tensor cores).  The input (2 GiB) is larger than L2 (129 MB), so every step
reads A from HBM.

Prints ONE JSON line (rank 0).  value = CountSketch-input bytes per second over
the whole step (GB/s); roofline = the CountSketch kernel against the measured
HBM copy bandwidth; e2e = the same metric through the public ms_sketch_host
call with pinned host buffers (host->device copy of A and device->host copy of
Z inside the timed region); cpu_baseline = the CPU oracle on the machine's host,
the same program and sample as the reference arm's step.

The line also carries:
* "least_squares": the least-squares configurations, device-timed: FP64
  multisketch sketch-and-solve against the normal equations at 8388608 x 128
  (sigma to 1e-6 and to 1e-10), and the refined mixed-precision solve at
  16777216 x 256 (split-BF16, BF16 and FP16 Gaussian stages) against FP64
  sketch-and-solve; every relative residual recomputed in FP64 by torch;
* "serving": a pool of least-squares problems shaped like the served
  configuration (n uniform in {16, 32, 64, 128}, d log-uniform in
  [2^14, 2^21], sigma log-spaced from 1 to 10^-U(2,8), FP32 A), a trace of
  requests drawn from the pool with fresh seeds, at capacity (all at t = 0)
  and with Poisson arrivals, solved (a) by the request server with the
  mixed-precision path (FP32 CountSketch, split-BF16 tensor-core Gaussian
  stage, FP64 QR, refinement to the minimiser), (b) one at a time by plain
  FP64 sketch-and-solve, and (c) one at a time by the FP64 sketch refined to
  the same tolerance as (a); solves/s and p50/p99 latency (arrival to
  completion) for each, and the accuracy of a sample of (a)'s results against
  the least-squares minimiser.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (d, n, k, p, dtype, gemm_prec)
    "multisketch_f64_4194304x64": (1 << 22, 64, 8192, 256, "f64", "f64"),
    "multisketch_f32_4194304x64": (1 << 22, 64, 8192, 256, "f32", "f32"),
    "countsketch_f64_65536x32": (65536, 32, 2048, 0, "f64", None),
    # profiling size (512 MiB of A: larger than L2, small enough for ncu replays)
    "multisketch_f64_1048576x64": (1 << 20, 64, 8192, 256, "f64", "f64"),
    "multisketch_f32_1048576x64": (1 << 20, 64, 8192, 256, "f32", "f32"),
}
DEFAULT = "multisketch_f64_4194304x64"

# DRAM bytes (read + write) of one CountSketch kernel launch, from one ncu
# capture of the same kernel on a quarter-size case (1048576 rows: 541.10 MB
# read + 3.06 MB written FP64; 270.55 + 3.13 MB FP32), scaled by the rows
# processed (the kernel streams A once, so traffic grows in proportion).
CS_TRAFFIC = {
    "multisketch_f64_4194304x64": 4 * (541.098e6 + 3.041e6),
    "multisketch_f32_4194304x64": 4 * (270.554e6 + 3.080e6),
    "multisketch_f64_1048576x64": 541.098e6 + 3.041e6,
    "multisketch_f32_1048576x64": 270.554e6 + 3.080e6,
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), float(pk["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms_local, device=None):
    """The largest per-rank duration over all ranks (all-reduce MAX; the value
    itself without a multi-rank process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms_local)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_rank, world, ms_max):
    """Whole-job throughput: the bytes every rank processed over the slowest
    rank's time (weak scaling: each replica sketches its own matrix)."""
    return world * bytes_per_rank / (ms_max * 1e-3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_ours(args):
    import numpy as np
    import torch

    import inputs
    import paper_2508_14209_gb300 as msk

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    d, n, k, p, dts, prec = WORKLOADS[args.workload]
    dtype = torch.float64 if dts == "f64" else torch.float32
    esz = 8 if dts == "f64" else 4
    seed = 0x5EED0002 + rank
    A = inputs.normal_matrix(d, n, seed, dtype=dtype, device=dev)
    stream = torch.cuda.current_stream()
    gp = msk.GEMM_PRECS[prec] if prec else None
    dt_code = msk.MSK_F64 if dts == "f64" else msk.MSK_F32
    Y = torch.empty((k, n), dtype=dtype, device=dev)
    launches_per_step = 1
    if gp is not None:
        # the multisketch is one library call (ms_sketch); events around its
        # CountSketch come from the library's stage-event hook, recorded on
        # the stream the kernel runs on
        Z = msk.colmajor(p, n, torch.float64, dev)
        mws_dev = msk.workspace(msk.msk_ms_workspace(d, n, False, k, p, dt_code, gp), dev)
        # CountSketch, G sampling, column maxima, Y slicing, sliced GEMM,
        # exact reduction (SIMT path: 4)
        launches_per_step = 6 if (gp == msk.GEMM_F64 and k >= 1024) else 4

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        if gp is None:
            msk.cs_sketch(A, k, seed, Y=Y)
            if ev is not None:
                ev[1].record(stream)
                ev[2].record(stream)
        else:
            msk.ms_sketch(A, k, p, seed, gemm_prec=gp, Z=Z, ws=mws_dev,
                          cs_events=None if ev is None else (ev[1], ev[2]))
        if ev is not None:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    for e in evs:  # create the events before the timed region
        for x in e:
            x.record(stream)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t0.record(stream)
    for s in range(args.steps):
        step(evs[s])
    t1.record(stream)
    torch.cuda.synchronize()
    time.sleep(0.2)
    clk = clocks.stop()
    ms_total = max_over_ranks(t0.elapsed_time(t1), device=dev)
    ms_step = ms_total / args.steps
    cs_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    gemm_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in evs]))
    a_bytes = d * n * esz
    value = whole_job_gbs(a_bytes, ws, ms_step)
    hbm, _, peak_src = _peaks()
    cs_alg_bytes = a_bytes + k * n * esz  # read A once, write Y once
    achieved = cs_alg_bytes / (cs_ms * 1e-3) / 1e9

    # end to end: the public ms_sketch_host call, page-locked host A in, host
    # Z out (row blocks copied to the device while the previous block is
    # sketched)
    e2e = None
    if gp is not None and not args.no_e2e:
        Ah = torch.empty((n, d), dtype=dtype, pin_memory=True)
        Ah.copy_(A.t())
        Zh = torch.empty((n, p), dtype=torch.float64, pin_memory=True).t()
        mws = msk.workspace(msk.msk_ms_host_workspace(d, n, False, k, p, dt_code, gp), dev)

        def e2e_step():
            msk.ms_sketch_host(Ah.t(), k, p, seed, gemm_prec=gp, Z=Zh, ws=mws)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ke = max(3, args.steps // 4)
        for _ in range(ke):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1) / ke, device=dev)
        e2e = {"value": round(whole_job_gbs(a_bytes, ws, ms_e2e), 3), "unit": "GB/s",
               "ms_per_step": round(ms_e2e, 4), "h2d_bytes_per_step": a_bytes,
               "d2h_bytes_per_step": p * n * 8}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args.workload, A)
    del A
    torch.cuda.empty_cache()
    ls_configs = None
    if not args.no_ls:
        ls_configs = run_ls_configs(dev)
    serving = None
    if args.serve_requests > 0:
        serving = run_serving(args, dev, rank)

    if rank == 0:
        out = {
            "metric": "CountSketch GB/s (% HBM peak); LS solves/s + p99 latency vs plain path",
            "value": round(value, 3), "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dts, "data": "synthetic",
            "config": {"workload": args.workload, "d": d, "n": n, "k": k, "p": p,
                       "gemm": prec, "countsketch": "atomic (L2 reductions)",
                       "l2": "inputs larger than L2 (2 GiB A per step)",
                       "parallelism": f"replicas{ws}"},
            "stages_ms": {"countsketch": round(cs_ms, 5), "gaussian_gemm": round(gemm_ms, 5),
                          "note": "countsketch: memset + kernel, events from the library's stage hook; "
                                  "gaussian_gemm: the Gaussian stage after the CountSketch"},
            "roofline": {"bound": "hbm", "kernel": "cs_fixed_f64_kernel (+Y zeroing memset)" if dts == "f64" else "cs_fixed_f32_kernel (+Y zeroing memset)",
                         "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "peak_source": peak_src,
                         "traffic": CS_TRAFFIC.get(args.workload),
                         "traffic_note": "ncu dram bytes of one 1048576-row launch, scaled by rows"},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "cpu_baseline": cpu,
            "least_squares": ls_configs,
            "serving": serving,
        }
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _serve_pool(dev, seed):
    import numpy as np
    import torch

    import inputs

    rng = np.random.default_rng(seed)
    pool = []
    for n in (16, 32, 64, 128):
        for i in range(6):
            d = int(2 ** rng.uniform(14, 21))
            e = float(rng.uniform(2, 8))
            A, b, _ = inputs.ls_problem(d, n, -e, seed=seed + 97 * n + i, dtype=torch.float32, device=dev)
            pool.append((A, b, d, n))
    torch.cuda.synchronize()
    return pool


SERVED = {"mem_budget": 64 << 30, "workers": 3, "max_batch": 32, "max_iter": 4}


def _serve_mixed(msk, pool, pick, arrivals, dev, tol, keep=None):
    import numpy as np
    import torch

    srv = msk.Server(mem_budget=SERVED["mem_budget"], workers=SERVED["workers"], max_batch=SERVED["max_batch"],
                     refine=True, tol=tol, max_iter=SERVED["max_iter"])
    xs = [torch.empty(pool[j][3], dtype=torch.float64, device=dev) for j in pick]
    tickets = []
    t0 = time.perf_counter()
    for i, j in enumerate(pick):
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        A, b, d, n = pool[j]
        tickets.append(srv.submit(A, b, 0x5EED0005 + i, xs[i]))
    srv.wait_all()
    wall = time.perf_counter() - t0
    lat, iters, conv = [], [], 0
    for t in tickets:
        done, info, l, rc = srv.poll(t)
        lat.append(l)
        iters.append(info["iters"])
        conv += int(info["converged"] == 1 and rc == 0)
    stats = srv.stats()
    srv.close()
    if keep is not None:
        keep.extend(xs[:16])
    lat = np.array(lat)
    return {"solves_per_s": round(len(pick) / wall, 1), "p50_ms": round(1e3 * float(np.median(lat)), 3),
            "p99_ms": round(1e3 * float(np.quantile(lat, 0.99)), 3), "mean_inner_iters": round(float(np.mean(iters)), 2),
            "converged": conv, "batches": stats["batches"]}


def _serve_plain(msk, pool, pick, arrivals, dev, keep=None, refine_tol=None):
    """One request at a time: FP64 sketch-and-solve (the plain path), or with
    refine_tol the same FP64 sketch refined to that tolerance (the plain path
    at the served path's accuracy)."""
    import numpy as np
    import torch

    refine = refine_tol is not None
    ws = {}
    lat = []
    xs = []
    t0 = time.perf_counter()
    for i, j in enumerate(pick):
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        A, b, d, n = pool[j]
        k, p = 2 * n * n, 4 * n
        if (d, n) not in ws:
            ws[(d, n)] = msk.workspace(msk.msk_lstsq_workspace(d, n, k, p, msk.MSK_F32, msk.GEMM_F64, int(refine)),
                                       dev)
        x = torch.empty(n, dtype=torch.float64, device=dev)
        msk.ms_lstsq(A, b, k, p, 0x5EED0005 + i, msk.GEMM_F64, refine=refine, tol=refine_tol or 0.0,
                     max_iter=SERVED["max_iter"], x=x, ws=ws[(d, n)], want_info=refine)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0 - arrivals[i])
        if keep is not None and len(xs) < 16:
            xs.append(x)
    wall = time.perf_counter() - t0
    if keep is not None:
        keep.extend(xs)
    lat = np.array(lat)
    return {"solves_per_s": round(len(pick) / wall, 1), "p50_ms": round(1e3 * float(np.median(lat)), 3),
            "p99_ms": round(1e3 * float(np.quantile(lat, 0.99)), 3)}


def _relres_fp64(A, b, x):
    """||b - A x|| / ||b|| in FP64 by torch (cuBLAS), independent of the
    library's kernels: the accuracy figures of the bench are measured, not
    taken from the solver's own report.  A is widened to FP64 in row blocks."""
    import torch

    rr = torch.zeros((), dtype=torch.float64, device=b.device)
    for r0 in range(0, A.shape[0], 1 << 21):
        r1 = min(A.shape[0], r0 + (1 << 21))
        r = b[r0:r1] - A[r0:r1].double() @ x
        rr += r @ r
    return float(torch.sqrt(rr) / torch.linalg.vector_norm(b))


def _timed(call, reps, warm=True):
    """Median CUDA-event time (ms) of `call` over `reps` runs (after one
    untimed run when `warm`); returns (ms, last result)."""
    import numpy as np
    import torch

    out = call() if warm else None
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = call()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), out


def run_ls_configs(dev):
    """The least-squares configurations, timed on the device (CUDA events,
    median), each result's relative residual recomputed in FP64 by torch:
    * A 8388608 x 128 FP64 = G diag(sigma) V^T, sigma 1 -> 1e-6 and
      1 -> 1e-10, b = A e + 1e-6 noise: multisketch sketch-and-solve
      (k = 32768, p = 512) against the normal equations (Section 6.3);
    * A 16777216 x 256 FP32, sigma 1 -> 1e-8: the refined mixed-precision
      solve (FP32 CountSketch to k = 131072, Gaussian stage to p = 1024 in
      split-BF16, BF16 and FP16, FP64 QR and residuals), against FP64
      sketch-and-solve of the same stored A."""
    import torch

    import inputs
    import paper_2508_14209_gb300 as msk

    out = {}
    d, n = 1 << 23, 128
    k, p = 2 * n * n, 4 * n
    for lsig in (-6, -10):
        A, b, _ = inputs.ls_problem(d, n, lsig, seed=0x5EED0003, dtype=torch.float64, device=dev)
        wss = msk.workspace(msk.msk_lstsq_workspace(d, n, k, p, msk.MSK_F64, msk.GEMM_F64, 0), dev)
        wsn = msk.workspace(msk.msk_ne_workspace(d, n), dev)
        xs = torch.empty(n, dtype=torch.float64, device=dev)
        xn = torch.empty(n, dtype=torch.float64, device=dev)
        ms_s, (_, _, rcs) = _timed(lambda: msk.ms_lstsq(A, b, k, p, 0x5EED0003, msk.GEMM_F64, x=xs, ws=wss,
                                                        want_info=False), 5)
        ms_n, (_, rcn) = _timed(lambda: msk.ne_lstsq(A, b, x=xn, ws=wsn), 3)
        rs = _relres_fp64(A, b, xs)
        rn = _relres_fp64(A, b, xn) if rcn == 0 else None
        out[f"ls_f64_8388608x128_sigma1e{lsig}"] = {
            "multisketch_sns": {"ms_per_solve": round(ms_s, 3), "solves_per_s": round(1e3 / ms_s, 2),
                                "status": rcs, "relres": float(f"{rs:.6e}")},
            "normal_equations": {"ms_per_solve": round(ms_n, 3), "solves_per_s": round(1e3 / ms_n, 2),
                                 "status": rcn, "relres": None if rn is None else float(f"{rn:.6e}")},
            "sns_time_over_ne": round(ms_s / ms_n, 4),
            "bytes_read_per_solve": {"sns": d * (n + 1) * 8, "ne": d * (n + 1) * 8}}
        del A, b, wss, wsn
        torch.cuda.empty_cache()
    d, n = 1 << 24, 256
    k, p = 2 * n * n, 4 * n
    A, b, _ = inputs.ls_problem(d, n, -8, seed=0x5EED0004, dtype=torch.float32, device=dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    ws64 = msk.workspace(msk.msk_lstsq_workspace(d, n, k, p, msk.MSK_F32, msk.GEMM_F64, 0), dev)
    ms64, (_, i64, rc64) = _timed(lambda: msk.ms_lstsq(A, b, k, p, 0x5EED0004, msk.GEMM_F64, x=x, ws=ws64), 2)
    r64 = _relres_fp64(A, b, x)
    del ws64
    cfg4 = {"fp64_sns": {"ms_per_solve": round(ms64, 3), "status": rc64, "relres": float(f"{r64:.6e}")}}
    # the single-rounding arms may run out of steps (MSK_ENOCONV after
    # max_iter outer steps of up to 200 CG iterations): timed once, cold
    for name, reps in (("bf16x3", 3), ("bf16", 1), ("f16", 1)):
        gp = msk.GEMM_PRECS[name]
        ws = msk.workspace(msk.msk_lstsq_workspace(d, n, k, p, msk.MSK_F32, gp, 1), dev)
        ms, (_, info, rc) = _timed(lambda: msk.ms_lstsq(A, b, k, p, 0x5EED0004, gp, refine=True, tol=1e-10,
                                                        max_iter=10, x=x, ws=ws), reps, warm=name == "bf16x3")
        rg = _relres_fp64(A, b, x)
        cfg4[f"refined_{name}"] = {
            "ms_per_solve": round(ms, 3), "status": rc, "converged": info["converged"],
            "inner_iterations": info["iters"], "relres": float(f"{rg:.6e}"),
            "min_bytes_read_per_solve": (info["iters"] + 2) * d * n * 4,
            "relres_over_fp64_sns": round(rg / r64, 6),
            "relres_sketch_and_solve_start": float(f"{info['relres_sns']:.6e}")}
        del ws
    out["refined_f32_16777216x256_sigma1e-8"] = cfg4
    del A, b
    torch.cuda.empty_cache()
    return out


def _minimiser_relres(A, b):
    """Relative residual of the least-squares minimiser of the stored A, by a
    QR-based FP64 solve (torch.linalg.lstsq, driver gels) on the GPU."""
    import torch

    A64 = A.double()
    x = torch.linalg.lstsq(A64, b.reshape(-1, 1), driver="gels").solution.reshape(-1)
    return _relres_fp64(A64, b, x)


def run_serving(args, dev, rank):
    """Served least squares: mixed-precision server vs plain FP64 one at a time."""
    import tempfile

    import numpy as np

    import paper_2508_14209_gb300 as msk
    from paper_2508_14209_gb300 import autotune

    pool = _serve_pool(dev, 0x5EED0005 + rank)
    rng = np.random.default_rng(0x5EED0005 + rank)
    N = args.serve_requests
    pick = rng.integers(0, len(pool), N)
    out = {"requests": N, "pool_problems": len(pool), "tol": args.serve_tol,
           "server": {"workers": SERVED["workers"], "max_batch": SERVED["max_batch"],
                      "max_iter": SERVED["max_iter"], "mem_budget_bytes": SERVED["mem_budget"]},
           "workload": "served: n in {16,32,64,128}, d log-uniform [2^14, 2^21], FP32 A, k=2n^2, p=4n"}
    # the autotuner on a batch of the trace, its choice cached per device and
    # batch signature, and the cached choice applied before serving
    cache = os.environ.get("MSK_AUTOTUNE_CACHE", os.path.join(tempfile.gettempdir(), "msketch_autotune.json"))
    tb = [(pool[j][0], pool[j][1], 0x5EED0005 + i) for i, j in enumerate(pick[:SERVED["max_batch"]])]
    dkey = autotune.device_key(dev)
    sig = autotune.signature([tuple(A.shape) for A, _, _ in tb])
    t = time.perf_counter()
    if not autotune.apply_cached(cache, dkey, sig):
        autotune.tune(tb, cache=cache, refine=True, tol=args.serve_tol, max_iter=SERVED["max_iter"])
        autotune.apply_cached(cache, dkey, sig)
    out["autotune"] = {"signature": sig, "chosen": autotune.lookup(cache, dkey, sig),
                       "seconds": round(time.perf_counter() - t, 2)}
    # warm-up of both paths (module loads, graph machinery, workspace)
    _serve_mixed(msk, pool, pick[:16], np.zeros(16), dev, args.serve_tol)
    _serve_plain(msk, pool, pick[:16], np.zeros(16), dev)
    _serve_plain(msk, pool, pick[:16], np.zeros(16), dev, refine_tol=args.serve_tol)
    zero = np.zeros(N)
    x_mixed, x_plain = [], []
    out["capacity"] = {"mixed": _serve_mixed(msk, pool, pick, zero, dev, args.serve_tol, keep=x_mixed),
                       "plain_fp64": _serve_plain(msk, pool, pick, zero, dev, keep=x_plain),
                       "plain_fp64_refined": _serve_plain(msk, pool, pick, zero, dev, refine_tol=args.serve_tol)}
    rate = args.serve_rate
    arrivals = np.cumsum(rng.exponential(1.0 / rate, N))
    out["poisson"] = {"rate_per_s": rate,
                      "mixed": _serve_mixed(msk, pool, pick, arrivals, dev, args.serve_tol),
                      "plain_fp64": _serve_plain(msk, pool, pick, arrivals, dev),
                      "plain_fp64_refined": _serve_plain(msk, pool, pick, arrivals, dev, refine_tol=args.serve_tol)}
    # accuracy of the first 16 served results (capacity run), recomputed in
    # FP64 outside the library: two-sided against the least-squares minimiser
    # of the stored A, and one-sided against plain FP64 sketch-and-solve of
    # the same request
    two_sided, ratios, worse = [], [], 0
    for i, (xm, xp) in enumerate(zip(x_mixed, x_plain)):
        A, b, d, n = pool[pick[i]]
        rm = _relres_fp64(A, b, xm)
        rp = _relres_fp64(A, b, xp)
        ro = _minimiser_relres(A, b)
        two_sided.append(abs(rm - ro) / ro)
        ratios.append(rm / rp)
        worse += int(rm > (1 + 1e-8) * rp)
    out["accuracy_sample"] = {
        "requests": len(ratios), "from": "served results at capacity (first 16 of the trace)",
        "max_two_sided_rel_error_vs_minimiser": float(f"{max(two_sided):.3e}"),
        "within_1e-8_of_minimiser": int(sum(e <= 1e-8 for e in two_sided)),
        "mixed_above_fp64_sns_by_1e-8": worse,
        "max_relres_ratio_mixed_over_fp64_sns": round(max(ratios), 6),
        "min_relres_ratio_mixed_over_fp64_sns": round(min(ratios), 6),
        "how": "FP64 residuals by torch; minimiser by torch.linalg.lstsq (gels) of the stored A in FP64"}
    return out


def _oracle_step(workload, Ah):
    """One pass of the CPU oracle (as it stands) over the whole workload: the
    CountSketch of A and, for a multisketch, the Gaussian stage on all of G."""
    import oracle

    d, n, k, p, dts, prec = WORKLOADS[workload]
    if prec is None:
        oracle.countsketch(Ah, k, 0x5EED0002)
    else:
        oracle.multisketch(Ah, k, p, 0x5EED0002, gemm_prec=prec)


def _oracle_sample(workload):
    d, n, *_ = WORKLOADS[workload]
    return f"whole workload ({d}x{n}, all of G), one pass per step, single thread"


def cpu_baseline(workload, A_dev):
    """The CPU oracle (unchanged) on the same workload, timed on this host:
    the same program, sample and unit as the reference arm's step."""
    d, n, k, p, dts, prec = WORKLOADS[workload]
    Ah = A_dev.cpu().numpy()
    t = time.perf_counter()
    _oracle_step(workload, Ah)
    dt = time.perf_counter() - t
    esz = 8 if dts == "f64" else 4
    return {"value": round(d * n * esz / dt / 1e9, 5), "unit": "GB/s", "cores": 1,
            "kind": "oracle", "seconds": round(dt, 3), "sample": _oracle_sample(workload)}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, timed on the host cores on
    the whole workload each step (the same program and sample as
    cpu_baseline; about 2.5 s per step for the default workload)."""
    import torch

    import inputs

    ws, rank, _ = _dist()
    if rank != 0:
        return
    d, n, k, p, dts, prec = WORKLOADS[args.workload]
    dtype = torch.float64 if dts == "f64" else torch.float32
    esz = 8 if dts == "f64" else 4
    Ah = inputs.normal_matrix(d, n, 0x5EED0002, dtype=dtype).numpy()
    for _ in range(args.warmup):
        _oracle_step(args.workload, Ah)
    t = time.perf_counter()
    for _ in range(args.steps):
        _oracle_step(args.workload, Ah)
    dt = (time.perf_counter() - t) / args.steps
    val = d * n * esz / dt / 1e9
    print(json.dumps({
        "impl": "reference", "metric": "CountSketch GB/s (% HBM peak); LS solves/s + p99 latency vs plain path",
        "value": round(val, 5), "unit": "GB/s", "n_gpus": ws, "device": "host cores (no GPU used)",
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dts, "data": "synthetic",
        "config": {"workload": args.workload, "d": d, "n": n, "k": k, "p": p, "gemm": prec},
        "cpu_baseline": {"value": round(val, 5), "unit": "GB/s", "kind": "oracle", "cores": 1,
                         "sample": _oracle_sample(args.workload)},
        "e2e": {"value": round(val, 5), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ls", action="store_true", help="skip the least-squares configurations")
    ap.add_argument("--serve-requests", type=int, default=4000)
    ap.add_argument("--serve-rate", type=float, default=400.0)
    ap.add_argument("--serve-tol", type=float, default=1e-7)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        import paper_2508_14209_gb300.build as b

        b.build()
        run_ours(args)


if __name__ == "__main__":
    main()
