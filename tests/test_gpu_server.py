"""Request server: results are the same alone and in the mix (refined, within
1e-8 of the relative residual of a single-problem solve and of the oracle's
minimiser), admission by the memory budget, refusal of oversized requests,
latency bookkeeping."""
import time

import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msk():
    import paper_2508_14209_gb300 as m
    from paper_2508_14209_gb300 import build

    assert torch.cuda.is_available()
    build.build()
    m.load()
    return m


def test_server_mix_equals_alone(msk, orc):
    specs = [(6000, 16, -3), (20000, 32, -6), (15000, 64, -8), (40000, 128, -5), (8000, 16, -8),
             (12000, 32, -2), (9000, 64, -4), (30000, 16, -6)]
    probs = []
    for j, (d, n, ls) in enumerate(specs):
        A, b, _ = inputs.ls_problem(d, n, ls, seed=900 + j, dtype=torch.float32)
        Ad = msk.colmajor(d, n, torch.float32, "cuda")
        Ad.copy_(A)
        probs.append((Ad, b.cuda(), 77 + j, A.numpy(), b.numpy()))
    srv = msk.Server(mem_budget=2 << 30, workers=2, max_batch=4, refine=True, tol=1e-12, max_iter=10)
    try:
        xs, tickets = [], []
        for A, b, s, _, _ in probs:  # arrivals spread over time so batches overlap
            x = torch.empty(A.shape[1], dtype=torch.float64, device="cuda")
            xs.append(x)
            tickets.append(srv.submit(A, b, s, x))
            time.sleep(0.002)
        srv.wait_all()
        for (A, b, s, An, bn), x, t in zip(probs, xs, tickets):
            done, info, lat, rc = srv.poll(t)
            assert done and rc == 0 and lat > 0.0, srv.error()
            n = A.shape[1]
            rmix = orc.relres(An, bn, x.cpu().numpy())
            x1, i1, rc1 = msk.ms_lstsq(A, b, 2 * n * n, 4 * n, s, msk.GEMM_BF16X3, refine=True,
                                       tol=1e-12, max_iter=10)
            ralone = orc.relres(An, bn, x1.cpu().numpy())
            ro = orc.relres(An, bn, orc.lstsq_exact(An, bn))
            assert abs(rmix - ralone) <= 1e-8 * ralone
            assert abs(rmix - ro) <= 1e-8 * ro
        st = srv.stats()
        assert st["solved"] == len(probs) and st["batches"] >= 2
    finally:
        srv.close()


def test_server_admission_and_refusal(msk):
    A, b, _ = inputs.ls_problem(200000, 128, -4, seed=3, dtype=torch.float32, device="cuda")
    need = msk.msk_batch_workspace([(A, b, 1)], refine=True)
    # a budget whose worker share cannot hold this request: refused at submit
    srv = msk.Server(mem_budget=max(need // 2, 1 << 20), workers=1, max_batch=8)
    try:
        x = torch.empty(128, dtype=torch.float64, device="cuda")
        with pytest.raises(msk.MskError) as ei:
            srv.submit(A, b, 1, x)
        assert ei.value.code == msk.MSK_ENOMEM
    finally:
        srv.close()
    # a share that holds exactly one such request: each batch admits one
    srv = msk.Server(mem_budget=int(need * 1.5), workers=1, max_batch=8)
    try:
        xs = [torch.empty(128, dtype=torch.float64, device="cuda") for _ in range(3)]
        ts = [srv.submit(A, b, 10 + i, xs[i]) for i in range(3)]
        srv.wait_all()
        assert all(srv.poll(t)[0] for t in ts)
        assert srv.stats()["batches"] == 3
    finally:
        srv.close()


def test_server_request_larger_than_a_worker_share(msk, orc):
    """A request whose workspace exceeds one worker's share of the budget,
    but not the budget, is solved alone with the whole pool (no worker starts
    a batch meanwhile); the small requests around it are solved as usual."""
    big_A, big_b, _ = inputs.ls_problem(40000, 128, -5, seed=41, dtype=torch.float32, device="cuda")
    need = msk.msk_batch_item_bound((big_A, big_b, 1))
    small = [inputs.ls_problem(6000, 16, -3, seed=50 + i, dtype=torch.float32, device="cuda") for i in range(4)]
    # two workers, each with 3/4 of the big request's bound
    srv = msk.Server(mem_budget=int(need * 1.5), workers=2, max_batch=4, refine=True, tol=1e-12, max_iter=10)
    try:
        reqs = [(A, b) for A, b, _ in small[:2]] + [(big_A, big_b)] + [(A, b) for A, b, _ in small[2:]]
        xs = [torch.empty(A.shape[1], dtype=torch.float64, device="cuda") for A, _ in reqs]
        ts = [srv.submit(A, b, 60 + i, x) for i, ((A, b), x) in enumerate(zip(reqs, xs))]
        srv.wait_all()
        for (A, b), x, t in zip(reqs, xs, ts):
            done, info, lat, rc = srv.poll(t)
            assert done and rc == 0, srv.error()
            An, bn = A.cpu().numpy(), b.cpu().numpy()
            ro = orc.relres(An, bn, orc.lstsq_exact(An, bn))
            assert abs(orc.relres(An, bn, x.cpu().numpy()) - ro) <= 1e-8 * ro
    finally:
        srv.close()
