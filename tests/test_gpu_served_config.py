"""The request server in the configuration the served benchmark runs
(tolerance 1e-7, at most 4 outer refinement steps, 3 workers, batches of up
to 32), on requests shaped like the served workload: n from {16, 32, 64, 128},
d log-uniform, sigma log-spaced from 1 to 10^-U(2,8), FP32 A, k = 2n^2,
p = 4n, fresh seeds.  Every result is checked against the oracle:

* two-sided against the exact least-squares minimiser of the stored A:
  |relres - relres*| <= 1e-8 relres*;
* one-sided against FP64 sketch-and-solve of the same request (same S and G):
  relres <= (1 + 1e-8) relres_SnS64;
* the relative residual the server reports is the oracle's recomputation.
"""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu

SERVED = dict(tol=1e-7, max_iter=4, workers=3, max_batch=32)


@pytest.fixture(scope="module")
def msk():
    import paper_2508_14209_gb300 as m
    from paper_2508_14209_gb300 import build

    assert torch.cuda.is_available()
    build.build()
    m.load()
    return m


def _requests():
    # d log-uniform; the upper end is kept where the oracle's QR of the whole
    # [A b] takes seconds (2^17 rows at n <= 64, 2^15 at n = 128; up to 2^19
    # at n = 16)
    rng = np.random.default_rng(0x5EED0005)
    top = {16: 19, 32: 17, 64: 17, 128: 15}
    out = []
    for n in (16, 32, 64, 128):
        for i in range(4 if n < 128 else 3):
            d = int(2 ** rng.uniform(14, top[n]))
            e = float(rng.uniform(2, 8))
            out.append((d, n, -e, 1000 + 17 * n + i))
    return out


def test_served_configuration_reaches_minimiser(msk, orc):
    probs = []
    for j, (d, n, ls, sd) in enumerate(_requests()):
        A, b, _ = inputs.ls_problem(d, n, ls, seed=sd, dtype=torch.float32)
        Ad = msk.colmajor(d, n, torch.float32, "cuda")
        Ad.copy_(A)
        probs.append((Ad, b.cuda(), 0x5EED0005 + j, A.numpy(), b.numpy()))
    srv = msk.Server(mem_budget=8 << 30, workers=SERVED["workers"], max_batch=SERVED["max_batch"],
                     refine=True, tol=SERVED["tol"], max_iter=SERVED["max_iter"])
    try:
        xs = [torch.empty(A.shape[1], dtype=torch.float64, device="cuda") for A, *_ in probs]
        tickets = [srv.submit(A, b, s, x) for (A, b, s, _, _), x in zip(probs, xs)]
        srv.wait_all()
        results = [srv.poll(t) for t in tickets]
    finally:
        srv.close()
    worst = 0.0
    for (A, b, s, An, bn), x, (done, info, lat, rc) in zip(probs, xs, results):
        d, n = A.shape
        assert done and rc in (msk.MSK_OK, msk.MSK_ENOCONV), (d, n, rc)
        xg = x.cpu().numpy()
        rg = orc.relres(An, bn, xg)
        ro = orc.relres(An, bn, orc.lstsq_exact(An, bn))
        worst = max(worst, abs(rg - ro) / ro)
        assert abs(rg - ro) <= 1e-8 * ro, (d, n, rg, ro, info)
        _, r_sns64, _ = orc.sns_lstsq(An.astype(np.float64), bn, 2 * n * n, 4 * n, s, "f64")
        assert rg <= (1 + 1e-8) * r_sns64, (d, n, rg, r_sns64)
        assert abs(info["relres"] - rg) <= 1e-10 * rg
    print(f"served configuration: worst |relres - relres*| / relres* = {worst:.3e}")
