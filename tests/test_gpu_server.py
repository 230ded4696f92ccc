"""The solve service: requests of several matrices submitted together are answered with the
same accuracy as solving each alone (both within the residual bound, and
|A (x_mix - x_alone)| <= 2 tol |b|), cached hierarchies are reused, requests for one
matrix are batched, and a budget too small for a hierarchy rejects it."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1302_2547_gb300 import _lib as U
from paper_1302_2547_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    from paper_1302_2547_gb300 import build as B

    B.build()


def test_mix_equals_alone():
    tol = 1e-8
    mats = [I.grid2d(80, 70), I.grid3d(24, sigma=0.25, seed=3), I.rgg(20000, 8.0, seed=5)]
    params = U.uaamg_default_params(max_agg_size=0, kcycle_ratio=5.0)
    rng = np.random.default_rng(0)
    reqs = []  # (matrix index, b)
    for k in range(24):
        m = int(rng.integers(0, 3)) if k >= 3 else k
        reqs.append((m, rng.uniform(-1, 1, mats[m].n)))
    srv = U.Server(params, workers=3, max_batch=8)
    try:
        tickets = [srv.submit(mats[m].rowptr, mats[m].col, mats[m].val, b, tol) for m, b in reqs]
        answers = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["done"] == len(reqs) and stats["rejected"] == 0
    assert stats["setups"] <= len(mats) + 2  # cached hierarchies are reused
    # a request batched with the setup of its matrix is not a cache hit; requests arriving
    # for a matrix held in the cache are
    assert stats["cache_hits"] <= stats["done"] and stats["batches"] < len(reqs)
    assert max(a[5] for a in answers) >= 2  # some requests were solved together
    handles = [U.uaamg_setup(A.rowptr, A.col, A.val, params) for A in mats]
    try:
        for (m, b), (st, x, it, rr, lat, batch) in zip(reqs, answers):
            A = mats[m]
            Asp = sp.csr_matrix((A.val, A.col, A.rowptr))
            bn = np.linalg.norm(b)
            assert st == 0 and lat > 0
            assert np.linalg.norm(b - Asp @ x) <= tol * bn * 1.0001
            xa = np.zeros(A.n)
            st1, it1, _ = U.uaamg_solve(handles[m], b, xa, tol)
            assert st1 == 0
            assert np.linalg.norm(Asp @ (x - xa)) <= 2.0001 * tol * bn
            assert abs(it - it1) <= 3
    finally:
        for h in handles:
            U.uaamg_free(h)


def test_budget_rejects_what_cannot_fit():
    A = I.grid3d(40, sigma=0.25, seed=1)
    held0 = U.uaamg_memory_in_use()
    srv = U.Server(U.uaamg_default_params(max_agg_size=0), budget_bytes=1 << 20, workers=1)
    try:
        t = srv.submit(A.rowptr, A.col, A.val, np.ones(A.n))
        st, *_ = srv.wait(t)
        assert st == 6  # UAAMG_ERR_BUDGET
        assert srv.stats()["rejected"] == 1
        # the rejected request holds no device memory, before and after the server ends
        assert U.uaamg_memory_in_use() == held0
    finally:
        srv.close()
    assert U.uaamg_memory_in_use() == held0


def test_cancel_withdraws_queued_requests_only():
    """With one worker busy on the first request, requests queued behind it can be withdrawn:
    their wait reports UAAMG_ERR_CANCELLED and no worker solves them; the others (the one
    in flight included) are answered as usual."""
    tol = 1e-8
    big = I.grid3d(48, sigma=0.25, seed=9)
    small = [I.grid2d(40 + 3 * k, 37) for k in range(4)]
    srv = U.Server(U.uaamg_default_params(max_agg_size=0), workers=1, max_batch=4)
    try:
        t0 = srv.submit(big.rowptr, big.col, big.val, np.ones(big.n), tol)
        ts = [srv.submit(A.rowptr, A.col, A.val, np.ones(A.n), tol) for A in small]
        withdrawn = [srv.cancel(t) for t in ts[1::2]]
        assert all(withdrawn)
        res0 = srv.wait(t0)
        res = [srv.wait(t) for t in ts]
        stats = srv.stats()
    finally:
        srv.close()
    assert res0[0] == 0
    for k, r in enumerate(res):
        if k % 2 == 1:
            assert r[0] == U.UAAMG_ERR_CANCELLED
        else:
            A = small[k]
            Asp = sp.csr_matrix((A.val, A.col, A.rowptr))
            assert r[0] == 0
            assert np.linalg.norm(np.ones(A.n) - Asp @ r[1]) <= tol * np.sqrt(A.n) * 1.0001
    assert stats["done"] == 1 + len(small) // 2 + len(small) % 2


def test_requests_for_different_matrices_share_one_batch():
    """With the one worker busy, requests for three different matrices (two of them twice)
    queue up; the next batch takes all six at once, as three systems of one
    uaamg_solve_batch call, and every answer meets the bars of solving it alone."""
    tol = 1e-8
    blocker = I.grid3d(48, sigma=0.25, seed=9)
    mats = [I.grid2d(50, 41), I.rgg(6000, 8.0, seed=31), I.grid3d(14, sigma=0.25, seed=32)]
    params = U.uaamg_default_params(max_agg_size=0, kcycle_ratio=3.0)
    rng = np.random.default_rng(5)
    reqs = [(m, rng.uniform(-1, 1, mats[m].n)) for m in (0, 1, 2, 0, 1, 2)]
    srv = U.Server(params, workers=1, max_batch=16)
    try:
        t0 = srv.submit(blocker.rowptr, blocker.col, blocker.val, np.ones(blocker.n), tol)
        ts = [srv.submit(mats[m].rowptr, mats[m].col, mats[m].val, b, tol) for m, b in reqs]
        assert srv.wait(t0)[0] == 0
        answers = [srv.wait(t) for t in ts]
    finally:
        srv.close()
    assert all(a[5] == len(reqs) for a in answers), [a[5] for a in answers]
    handles = [U.uaamg_setup(A.rowptr, A.col, A.val, params) for A in mats]
    try:
        for (m, b), (st, x, it, rr, lat, batch) in zip(reqs, answers):
            A = mats[m]
            Asp = sp.csr_matrix((A.val, A.col, A.rowptr))
            bn = np.linalg.norm(b)
            assert st == 0
            assert np.linalg.norm(b - Asp @ x) <= tol * bn * 1.0001
            xa = np.zeros(A.n)
            st1, it1, _ = U.uaamg_solve(handles[m], b, xa, tol)
            assert st1 == 0
            assert np.linalg.norm(Asp @ (x - xa)) <= 2.0001 * tol * bn
            assert abs(it - it1) <= 3
    finally:
        for h in handles:
            U.uaamg_free(h)
