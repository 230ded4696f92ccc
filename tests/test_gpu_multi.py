"""GPU parity of uaamg_solve_many (several right-hand sides at once): every column must
satisfy the same bars as a single solve (relative residual <= tol on the host in FP64, and
|A (x_col - x_oracle)| <= 2 tol |b|), with iteration counts close to uaamg_solve's on the
same handle (FP64: within 1; mixed: within 3, the columns' FP32 rounding differs)."""
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


CASES = [
    ("poisson2d_64", lambda: I.poisson2d_64(), {}),
    ("grid3d_36_bench", lambda: I.grid3d(36, sigma=0.25, seed=3), "BENCH"),
    ("rgg_30k", lambda: I.rgg(30000, 8.0, seed=2), {"max_agg_size": 0, "kcycle_ratio": 3.0}),
    ("grid2d_100_tau", lambda: I.grid2d(100), {"kcycle_tau": 0.25}),
]


@pytest.mark.parametrize("precision", [U.UAAMG_FP64, U.UAAMG_MIXED])
@pytest.mark.parametrize("R", [1, 3, 16])
@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_solve_many_columns(oracle, name, make, kw, R, precision):
    A = make()
    if kw == "BENCH":
        from bench import BENCH_PARAMS as kw
    tol = 1e-8
    p = U.uaamg_default_params(precision=precision, **kw)
    h = U.uaamg_setup(A.rowptr, A.col, A.val, p)
    okeys = ("coarse_size", "max_levels", "max_agg_size", "pass_mode", "seed", "pre", "post",
             "kcycle_inner", "kcycle_tau", "max_iter", "agg_repeat", "kcycle_ratio",
             "min_coarsening", "jacobi_omega")
    H = oracle.Hierarchy(A.rowptr, A.col, A.val,
                         oracle.Params(**{k: getattr(p, k) for k in okeys}))
    try:
        rng = np.random.default_rng(R)
        B = rng.uniform(-1, 1, (A.n, R))
        X = np.zeros_like(B)
        st, its, rrs = U.uaamg_solve_many(h, B, X, tol)
        assert st == 0, (its, rrs)
        Asp = sp.csr_matrix((A.val, A.col, A.rowptr))
        for r in range(R):
            b = np.ascontiguousarray(B[:, r])
            bn = np.linalg.norm(b)
            x = X[:, r]
            assert np.linalg.norm(b - Asp @ x) <= tol * bn * 1.0001, r
            assert abs(rrs[r] - np.linalg.norm(b - Asp @ x) / bn) <= 1e-3 * tol + 1e-14
            xo, ito, _, sto, _ = H.solve(b, tol)
            assert sto == 0 and np.linalg.norm(Asp @ (x - xo)) <= 2.0001 * tol * bn
            xs = np.zeros(A.n)
            st1, it1, _ = U.uaamg_solve(h, b, xs, tol)
            assert st1 == 0
            slack = 1 if precision == U.UAAMG_FP64 else 3
            assert abs(int(its[r]) - it1) <= slack, (r, its[r], it1)
    finally:
        U.uaamg_free(h)


def test_solve_many_zero_and_device_columns():
    import torch

    A = I.grid3d(20, sigma=0.25, seed=1)
    h = U.uaamg_setup(A.rowptr, A.col, A.val, U.uaamg_default_params(max_agg_size=0))
    try:
        dev = torch.device("cuda:0")
        B = torch.rand(A.n, 32, dtype=torch.float64, device=dev) * 2 - 1
        B[:, 5] = 0.0
        X = torch.empty_like(B)
        st, its, rrs = U.uaamg_solve_many(h, B, X, 1e-9)
        torch.cuda.synchronize()
        assert st == 0 and its[5] == 0 and torch.all(X[:, 5] == 0)
        Asp = sp.csr_matrix((A.val, A.col, A.rowptr))
        Xh, Bh = X.cpu().numpy(), B.cpu().numpy()
        for r in range(32):
            if r == 5:
                continue
            assert np.linalg.norm(Bh[:, r] - Asp @ Xh[:, r]) <= 1e-9 * np.linalg.norm(Bh[:, r]) * 1.0001
        # a smaller batch on the same handle reuses the workspace
        st, its2, _ = U.uaamg_solve_many(h, Bh[:, :4].copy(), np.zeros((A.n, 4)), 1e-9)
        assert st == 0
    finally:
        U.uaamg_free(h)
