"""Kernel-class profiling of a solve leaves its arithmetic unchanged.

With a solve-time class profiled (the level-0 first sweep, or the level-0 FP64 SpMV of the
outer iteration), the first three outer iterations of each solve run launch by launch with
CUDA events around the profiled launch, and the remaining iterations run in the device-side
loop.  The same kernels run in the same order either way, so the solution and the iteration
count are bitwise those of the unprofiled solve, on a fresh handle and on a second solve
that reuses the handle's loop graph; exactly three launches per solve are timed (every
iteration's launch without graphs).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("kclass", ["smooth0", "spmv64"])
def test_profiled_solve_matches_unprofiled(kclass, graphs):
    import torch

    from paper_1302_2547_gb300 import _lib as U
    from paper_1302_2547_gb300 import inputs as I

    assert torch.cuda.is_available()
    cls = {"smooth0": U.UAAMG_KCLASS_SMOOTH0, "spmv64": U.UAAMG_KCLASS_SPMV64}[kclass]
    A = I.laplace3d_128(32)
    b = I.rhs_uniform(A.n, I.RHS_SEED + 7)
    p = U.uaamg_default_params(precision=U.UAAMG_MIXED, use_graphs=graphs, max_agg_size=4,
                               agg_repeat=2, kcycle_ratio=6.0, min_coarsening=1.5)
    runs = {}
    for prof in (0, cls):
        h = U.uaamg_setup(A.rowptr, A.col, A.val, p)
        try:
            if prof:
                U.uaamg_set_profiling(h, prof)
            sols = []
            for _ in range(2):  # the second solve reuses the handle's graphs
                x = np.zeros(A.n)
                st, it, rr = U.uaamg_solve(h, b, x, 1e-10)
                assert st == 0 and rr <= 1e-10
                sols.append((x, it, U.uaamg_residual_history(h)))
            runs[prof] = sols
            if prof:
                n, ms, per = U.uaamg_get_profile(h)
                its = [s[1] for s in sols]
                expect = sum(its) if not graphs else sum(min(3, k) for k in its)
                assert n == expect, (n, its)
                assert ms > 0.0 and per > 0.0
        finally:
            U.uaamg_free(h)
    for (x0, it0, h0), (x1, it1, h1) in zip(runs[0], runs[cls]):
        assert it0 == it1
        assert np.array_equal(x0, x1)
        assert len(h0) == len(h1)
        np.testing.assert_allclose(h1, h0, rtol=1e-12, atol=0.0)
