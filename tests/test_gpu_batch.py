"""uaamg_solve_batch: many systems of different sizes, kinds and depths solved together.

Bars (the solve bars of the single-system tests, per column):
  * every column reaches |b - A x| <= tol |b| (checked here in FP64) and lies within the
    oracle's solution in the sense |A (x - x_oracle)| <= 2 tol |b|;
  * a system's result in the mix is bit for bit its result when solved alone through the
    same entry point (its tiles and inner-product order depend on itself only), with the
    same iteration counts;
  * FP64 batches take within one iteration of uaamg_solve_many on the same handle.
The mix spans single-level systems (exact solve only), two-stage aggregation with one
flexible-CG step on weakly coarsened levels, unbounded aggregates, a zero right-hand side,
and 1 to 32 columns per system.
"""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu

GRID = dict(max_agg_size=4, agg_repeat=2, kcycle_ratio=5.0, min_coarsening=1.5)
RGG = dict(max_agg_size=0, agg_repeat=1, kcycle_ratio=3.0, min_coarsening=1.5)


def _systems(I):
    """(matrix, parameter overrides, columns) of the mix."""
    return [
        (I.grid2d(30, 30), GRID, 3),
        (I.rgg(5000, 8.0, seed=21), RGG, 1),
        (I.path_graph(50, dirichlet=True), {}, 2),  # one level: the exact solve only
        (I.grid2d(100, 91), GRID, 4),
        (I.grid3d(16, sigma=0.25, seed=22), GRID, 2),
        (I.rgg(20000, 8.0, seed=23), RGG, 5),
        (I.random_graph(700, 900, seed=24, integer_weights=False), {}, 1),
        (I.grid2d(57, 44), {}, 32),
    ]


def _rhs(A, R, seed, zero_col=None):
    B = np.random.default_rng(seed).uniform(-1.0, 1.0, (A.n, R))
    if zero_col is not None:
        B[:, zero_col] = 0.0
    return np.ascontiguousarray(B)


@pytest.fixture(scope="module")
def built():
    import torch

    assert torch.cuda.is_available()
    from paper_1302_2547_gb300 import build as B

    B.build()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_mix_equals_alone_and_meets_the_oracle(built, oracle, inputs, precision):
    from paper_1302_2547_gb300 import _lib as U

    I = inputs
    prec = U.UAAMG_MIXED if precision == "mixed" else U.UAAMG_FP64
    tol = 1e-8
    systems = _systems(I)
    params = [U.uaamg_default_params(precision=prec, **kw) for _, kw, _ in systems]
    hs = U.uaamg_setup_batch([(A.rowptr, A.col, A.val) for A, _, _ in systems], params,
                             threads=4)
    try:
        Bs = [_rhs(A, R, 100 + k, zero_col=1 if k == 0 else None)
              for k, (A, _, R) in enumerate(systems)]
        Xs = [np.zeros_like(B) for B in Bs]
        st, its, rrs = U.uaamg_solve_batch(hs, Bs, Xs, tol)
        assert st == 0
        for k, (A, kw, R) in enumerate(systems):
            Asp = sp.csr_matrix((A.val, A.col, A.rowptr))
            H = oracle.Hierarchy(A.rowptr, A.col, A.val, oracle.Params(**kw))
            for c in range(R):
                b, x = Bs[k][:, c], Xs[k][:, c]
                bn = np.linalg.norm(b)
                if bn == 0.0:
                    assert np.all(x == 0.0) and its[k][c] == 0
                    continue
                assert np.linalg.norm(b - Asp @ x) <= tol * bn * 1.0001, (k, c)
                assert rrs[k][c] <= tol * 1.0001
                if c < 2:  # the oracle on two columns per system
                    xo, ito, _, sto, _ = H.solve(b, tol)
                    assert sto == 0
                    assert np.linalg.norm(Asp @ (x - xo)) <= 2.0001 * tol * bn, (k, c)
        # each system alone: the same bits and iteration counts
        for k in range(len(systems)):
            Xa = [np.zeros_like(Bs[k])]
            st1, it1, rr1 = U.uaamg_solve_batch([hs[k]], [Bs[k]], Xa, tol)
            assert st1 == 0
            assert np.array_equal(Xa[0], Xs[k]), k
            assert np.array_equal(it1[0], its[k]), k
        if prec == U.UAAMG_FP64:  # the same algorithm as uaamg_solve_many, per column
            for k, (A, _, R) in enumerate(systems):
                if R < 2:
                    continue
                Xm = np.zeros_like(Bs[k])
                stm, itm, _ = U.uaamg_solve_many(hs[k], Bs[k], Xm, tol)
                assert stm == 0
                assert np.all(np.abs(itm.astype(int) - its[k].astype(int)) <= 1), (k, itm, its[k])
    finally:
        for h in hs:
            U.uaamg_free(h)


def test_batch_rejects_what_it_cannot_run(built, inputs):
    from paper_1302_2547_gb300 import _lib as U

    A = inputs.grid2d(20)
    h = U.uaamg_setup(A.rowptr, A.col, A.val, U.uaamg_default_params())
    h2 = U.uaamg_setup(A.rowptr, A.col, A.val, U.uaamg_default_params(pre=2))
    h3 = U.uaamg_setup(A.rowptr, A.col, A.val, U.uaamg_default_params(precision=U.UAAMG_FP64))
    try:
        B = np.ones((A.n, 1))
        X = np.zeros_like(B)
        for hl, code in (([h, h], 1), ([h2], 9), ([h, h3], 1)):
            with pytest.raises(U.UaamgError) as e:
                U.uaamg_solve_batch(hl, [B] * len(hl), [X] * len(hl))
            assert e.value.status == code
        with pytest.raises(U.UaamgError) as e:
            U.uaamg_solve_batch([h], [np.ones((A.n, 33))], [np.zeros((A.n, 33))])
        assert e.value.status == 9
    finally:
        for x in (h, h2, h3):
            U.uaamg_free(x)
