"""Bounded device waits run out without harming the device.

The cooperative aggregation kernel synchronises its blocks with grid barriers whose wait is
bounded by the handle's wait limit (uaamg_params.wait_limit_ns).  With a limit of 1 ns every
block that finds a barrier incomplete gives up at once, so setting up a graph large enough
for many blocks makes the barriers run out: the setup must report UAAMG_ERR_TIMEOUT (and
free what it built), and the next setup and solve on the same device, with the default
limit, must succeed.  No wait is left unbounded and nothing faults: the blocks that give up
return, and the host reads the error word.
"""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu


def test_barrier_wait_limit_runs_out_and_device_stays_usable():
    import torch

    from paper_1302_2547_gb300 import _lib as U
    from paper_1302_2547_gb300 import build as B
    from paper_1302_2547_gb300 import inputs as I

    assert torch.cuda.is_available()
    B.build()
    A = I.grid2d(512, 512)  # 262,144 vertices: the grid-wide aggregation kernel
    held0 = U.uaamg_memory_in_use()
    with pytest.raises(U.UaamgError) as e:
        U.uaamg_setup(A.rowptr, A.col, A.val, U.uaamg_default_params(wait_limit_ns=1))
    assert e.value.status == 8  # UAAMG_ERR_TIMEOUT
    assert U.uaamg_memory_in_use() == held0  # the failed setup released everything
    # the same device, the default limit: a clean setup and solve
    h = U.uaamg_setup(A.rowptr, A.col, A.val, U.uaamg_default_params())
    try:
        b = I.rhs_uniform(A.n, 7)
        x = np.zeros(A.n)
        st, it, rr = U.uaamg_solve(h, b, x, 1e-8)
        assert st == 0
        Asp = sp.csr_matrix((A.val, A.col, A.rowptr))
        assert np.linalg.norm(b - Asp @ x) <= 1e-8 * np.linalg.norm(b) * 1.0001
    finally:
        U.uaamg_free(h)

