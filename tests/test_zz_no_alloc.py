"""uaamg_aggregate_static: aggregation for callers that cannot allocate device memory.

Such callers (an external memory manager owns the device's memory, or the thread must not
call cudaMalloc/cudaFree while other work runs) pass only their input CSR and output
buffer; the library's scratch is a static device array of fixed size.  This test checks,
through the C ABI, that two calls in a row give exactly the level-0 aggregates that the
allocating entry point (uaamg_setup) computes for the same graph and parameters, and that
graphs above the array's limit are rejected before any device work.  Aggregates are
integers, so the bar is bit-exact equality, as in the other aggregation tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _reference(A, t, mode, seed):
    """Level-0 aggregates of uaamg_setup with one aggregation stage (agg_repeat = 1), the
    setup this entry point reproduces."""
    from paper_1302_2547_gb300 import _lib as U

    p = U.uaamg_default_params(max_agg_size=t, pass_mode=mode, seed=seed,
                               precision=U.UAAMG_FP64, agg_repeat=1)
    h = U.uaamg_setup(A.rowptr, A.col, A.val, p)
    try:
        return U.uaamg_get_aggregates(h, 0), U.uaamg_level_info(h, 1)[0]
    finally:
        U.uaamg_free(h)


def test_static_aggregation_matches_setup_twice():
    import torch

    from paper_1302_2547_gb300 import _lib as U
    from paper_1302_2547_gb300 import build as B
    from paper_1302_2547_gb300 import inputs as I

    assert torch.cuda.is_available()
    B.build()
    dev = torch.device("cuda:0")
    cases = [(I.grid3d(40, sigma=0.25, seed=3), 0, U.UAAMG_PASS_SINGLE_ROUND, 0x5EED),
             (I.grid2d(300, 250), 5, U.UAAMG_PASS_SINGLE_ROUND, 0x5EED),
             (I.rgg(60000, 8.0, seed=4), 0, U.UAAMG_PASS_MAXIMAL, 12345)]
    for A, t, mode, seed in cases:
        ref, nc_ref = _reference(A, t, mode, seed)
        rp, cc, vv = (torch.from_numpy(a).to(dev) for a in (A.rowptr, A.col, A.val))
        aggs = [torch.full((A.n,), -7, dtype=torch.int32, device=dev) for _ in range(2)]
        torch.cuda.synchronize()
        for call in range(2):
            # the second call must not take any device memory: neither the device's free
            # memory nor the library's own allocation count may change across it (the first
            # call may still load kernels)
            free0, held0 = torch.cuda.mem_get_info()[0], U.uaamg_memory_in_use()
            nc = U.uaamg_aggregate_static(rp, cc, vv, aggs[call], max_agg_size=t,
                                          pass_mode=mode, seed=seed)
            torch.cuda.synchronize()
            if call == 1:
                assert torch.cuda.mem_get_info()[0] == free0, A.name
                assert U.uaamg_memory_in_use() == held0, A.name
            assert nc == nc_ref, (A.name, call)
            assert np.array_equal(aggs[call].cpu().numpy(), ref), (A.name, call)


def test_static_aggregation_rejects_graphs_above_its_limit():
    import torch

    from paper_1302_2547_gb300 import _lib as U
    from paper_1302_2547_gb300 import inputs as I

    A = I.path_graph((1 << 18) + 1, dirichlet=True)
    dev = torch.device("cuda:0")
    rp, cc, vv = (torch.from_numpy(a).to(dev) for a in (A.rowptr, A.col, A.val))
    agg = torch.empty(A.n, dtype=torch.int32, device=dev)
    with pytest.raises(U.UaamgError) as e:
        U.uaamg_aggregate_static(rp, cc, vv, agg)
    assert e.value.status == 9  # UAAMG_ERR_UNSUPPORTED
