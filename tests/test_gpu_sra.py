"""GPU parity of subgraph reshaping (Section 3.2, Algorithm 3) through the C ABI.

Bars:
  * the aggregation after every round of every compared level: bit-exact with the oracle
    (integer work; both sides take each split's decision in FP64 with the same tie rule, so
    a split may differ only where two energies lie within the tie tolerance of each other,
    and the inputs below have none);
  * the coarse matrix built from the reshaped aggregates: bit-exact (Eq. 2.4, same order);
  * at the full 128^3 size, where the oracle cannot reshape every pair in seconds: every
    pair of the oracle's round-1 matching is split into balanced halves labelled by the
    pair's own numbers, all other vertices keep their aggregate, and sampled pairs are
    split exactly as the oracle splits them;
  * a solve with a reshaped hierarchy reaches the requested FP64 residual.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sra as SRA
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


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def oracle_levels(oracle, A, p, nlev):
    """Aggregations of levels 0..nlev-2 with reshaping, and the CSR of every level."""
    rp, cc, vv = A.rowptr, A.col, A.val
    aggs, mats = [], [(rp, cc, vv)]
    for l in range(nlev - 1):
        P = oracle.priorities(rp, cc, p.seed, l)
        root, _, _ = oracle.paa(rp, cc, P, p.max_agg_size, p.pass_mode)
        agg, nc = oracle.renumber(root)
        agg = SRA.reshape_level(rp, cc, vv, agg, nc, p.seed, l, p.sra_rounds)
        aggs.append(agg)
        rp, cc, vv = oracle.coarse(rp, cc, vv, agg, nc)
        mats.append((rp, cc, vv))
    return aggs, mats


CASES = [
    ("grid2d_40x36", lambda: I.grid2d(40, 36), {}),
    ("grid2d_40x36_t4_3rounds", lambda: I.grid2d(40, 36), {"max_agg_size": 4, "sra_rounds": 3}),
    ("grid3d_10x9x8_lognormal", lambda: I.grid3d(10, 9, 8, sigma=0.25, seed=4), {}),
    ("rgg_3000_unbounded", lambda: I.rgg(3000, 8.0, seed=7), {"max_agg_size": 0}),
    ("random_1500_real", lambda: I.random_graph(1500, 2500, seed=2, integer_weights=False), {}),
    ("grid2d_33x30_maximal", lambda: I.grid2d(33, 30), {"pass_mode": 0, "max_agg_size": 0}),
    ("path_97", lambda: I.path_graph(97, dirichlet=True), {}),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_reshaped_levels_match_the_oracle(oracle, name, make, kw):
    A = make()
    args = {"sra_rounds": 2, "coarse_size": 16}
    args.update(kw)
    p = U.uaamg_default_params(**args)
    h = U.uaamg_setup(A.rowptr, A.col, A.val, p)
    try:
        nlev = min(3, U.uaamg_num_levels(h))
        assert nlev >= 2
        aggs, mats = oracle_levels(oracle, A, p, nlev)
        for l in range(nlev - 1):
            got = U.uaamg_get_aggregates(h, l)
            assert np.array_equal(got, aggs[l]), (name, l, int(np.sum(got != aggs[l])))
            rp, cc, vv = U.uaamg_get_level_csr(h, l + 1)
            orp, occ, ovv = mats[l + 1]
            assert np.array_equal(rp, orp) and np.array_equal(cc, occ), (name, l + 1)
            assert np.array_equal(bits(vv), bits(ovv)), (name, l + 1)
    finally:
        U.uaamg_free(h)


def test_reshaping_changes_the_aggregates_and_keeps_their_number(oracle):
    A = I.grid2d(40, 36)
    p0 = U.uaamg_default_params(coarse_size=16)
    p1 = U.uaamg_default_params(coarse_size=16, sra_rounds=1)
    h0 = U.uaamg_setup(A.rowptr, A.col, A.val, p0)
    h1 = U.uaamg_setup(A.rowptr, A.col, A.val, p1)
    try:
        a0, a1 = U.uaamg_get_aggregates(h0, 0), U.uaamg_get_aggregates(h1, 0)
        assert U.uaamg_level_info(h0, 1)[0] == U.uaamg_level_info(h1, 1)[0]
        assert a0.max() == a1.max()
        assert np.sum(a0 != a1) > 0
        # the passes of Algorithm 2 are untouched by the post-process
        assert np.array_equal(U.uaamg_get_pass_of(h0, 0), U.uaamg_get_pass_of(h1, 0))
    finally:
        U.uaamg_free(h0)
        U.uaamg_free(h1)


@pytest.mark.parametrize("precision", [U.UAAMG_FP64, U.UAAMG_MIXED])
def test_solve_with_reshaped_hierarchy(precision):
    A = I.grid3d(24, 22, 20, sigma=0.25, seed=9)
    p = U.uaamg_default_params(sra_rounds=2, precision=precision)
    h = U.uaamg_setup(A.rowptr, A.col, A.val, p)
    try:
        b = I.rhs_uniform(A.n, 77)
        x = np.zeros(A.n)
        st, it, rr = U.uaamg_solve(h, b, x, 1e-10)
        Asp = sp.csr_matrix((A.val, A.col, A.rowptr))
        assert st == 0 and it <= 60
        assert np.linalg.norm(b - Asp @ x) <= 1e-10 * np.linalg.norm(b) * 1.0001
    finally:
        U.uaamg_free(h)


def test_profile_class_counts_the_pair_kernel():
    A = I.grid2d(64, 64)
    p = U.uaamg_default_params(sra_rounds=3, profile_class=U.UAAMG_KCLASS_SRA)
    h = U.uaamg_setup(A.rowptr, A.col, A.val, p)
    try:
        launches, ms, flops = U.uaamg_get_profile(h)
        assert launches == 3 and ms > 0.0 and flops > 0.0
    finally:
        U.uaamg_free(h)


def test_full_size_first_reshaping_round(oracle):
    """128^3 with lognormal weights, device-resident input, one reshaping round on level 0."""
    import torch

    from bench import BENCH_PARAMS

    A = I.laplace3d_128()
    dev = torch.device("cuda:0")
    rp, cc, vv = (torch.from_numpy(a).to(dev) for a in (A.rowptr, A.col, A.val))
    kw = dict(BENCH_PARAMS)
    kw["sra_rounds"] = 1
    kw["agg_repeat"] = 1
    p = U.uaamg_default_params(**kw)
    h = U.uaamg_setup(rp, cc, vv, p)
    try:
        got = U.uaamg_get_aggregates(h, 0)
    finally:
        U.uaamg_free(h)
    P = oracle.priorities(A.rowptr, A.col, p.seed, 0)
    root, _, _ = oracle.paa(A.rowptr, A.col, P, p.max_agg_size, p.pass_mode)
    agg, nc = oracle.renumber(root)
    assert got.max() == nc - 1
    pairs = SRA.matching(A.rowptr, A.col, A.val, agg, nc, SRA.round_salt(p.seed, 0, 0))
    assert len(pairs) > nc // 10
    pI = np.array([a for a, _ in pairs])
    pJ = np.array([b for _, b in pairs])
    in_pair = np.zeros(nc, bool)
    in_pair[pI] = True
    in_pair[pJ] = True
    # vertices outside the matched unions keep their aggregate
    out = ~in_pair[agg]
    assert np.array_equal(got[out], agg[out])
    # every union stays with its own two numbers; a changed union is split into balanced
    # halves (an unchanged one either had no admissible split or was already the best)
    partner = np.full(nc, -1)
    partner[pI] = pJ
    partner[pJ] = pI
    v = np.flatnonzero(~out)
    assert np.all((got[v] == agg[v]) | (got[v] == partner[agg[v]]))
    lo = np.minimum(agg[v], partner[agg[v]])
    cnt_lo = np.bincount(lo[got[v] == lo], minlength=nc)
    tot = np.bincount(lo, minlength=nc)
    changed = np.bincount(lo, weights=(got[v] != agg[v]), minlength=nc) > 0
    assert changed.sum() > len(pairs) // 4
    assert np.all(np.abs(2 * cnt_lo[changed] - tot[changed]) <= 1)
    # sampled pairs split exactly as the oracle splits them
    order = np.argsort(agg, kind="stable")
    ptr = np.concatenate([[0], np.cumsum(np.bincount(agg, minlength=nc))])
    rng = np.random.default_rng(11)
    for k in rng.choice(len(pairs), size=min(120, len(pairs)), replace=False):
        a, b = pairs[k]
        Uu = np.sort(np.concatenate([order[ptr[a]:ptr[a + 1]], order[ptr[b]:ptr[b + 1]]]))
        best, _ = SRA.reshape_pair(SRA.local_laplacian(A.rowptr, A.col, A.val, Uu))
        if best is None:
            expect = agg[Uu]
        else:
            first, other = (a, b) if best & 1 else (b, a)
            expect = np.array([first if best >> j & 1 else other for j in range(len(Uu))])
        assert np.array_equal(got[Uu], expect), (a, b)


def oracle_levels_twice(oracle, A, p, nlev):
    """As oracle_levels with aggregation applied twice per level (Section 3.3): stage 1
    (priority salt index 2l) is reshaped, stage 2 (salt 2l+1) aggregates its coarse matrix,
    and the level's aggregates are the unions."""
    rp, cc, vv = A.rowptr, A.col, A.val
    aggs, mats = [], [(rp, cc, vv)]
    for l in range(nlev - 1):
        P = oracle.priorities(rp, cc, p.seed, 2 * l)
        root, _, _ = oracle.paa(rp, cc, P, p.max_agg_size, p.pass_mode)
        a1, n1 = oracle.renumber(root)
        a1 = SRA.reshape_level(rp, cc, vv, a1, n1, p.seed, l, p.sra_rounds)
        r1, c1, v1 = oracle.coarse(rp, cc, vv, a1, n1)
        agg, nxt = a1, (r1, c1, v1)
        if n1 > p.coarse_size:
            P2 = oracle.priorities(r1, c1, p.seed, 2 * l + 1)
            root2, _, _ = oracle.paa(r1, c1, P2, p.max_agg_size, p.pass_mode)
            a2, n2 = oracle.renumber(root2)
            if n2 < n1:
                agg, nxt = a2[a1], oracle.coarse(r1, c1, v1, a2, n2)
        aggs.append(agg)
        rp, cc, vv = nxt
        mats.append(nxt)
    return aggs, mats


def test_reshaped_first_stage_of_double_aggregation(oracle):
    """Reshaping with two aggregation stages per level (the benchmark's setting): stage 1 is
    reshaped before stage 2 aggregates its coarse matrix; bit-exact with the oracle."""
    A = I.grid3d(12, 11, 10, sigma=0.25, seed=5)
    p = U.uaamg_default_params(sra_rounds=2, coarse_size=16, agg_repeat=2, max_agg_size=4)
    h = U.uaamg_setup(A.rowptr, A.col, A.val, p)
    try:
        nlev = min(3, U.uaamg_num_levels(h))
        assert nlev == 3
        aggs, mats = oracle_levels_twice(oracle, A, p, nlev)
        for l in range(nlev - 1):
            got = U.uaamg_get_aggregates(h, l)
            assert np.array_equal(got, aggs[l]), (l, int(np.sum(got != aggs[l])))
            rp, cc, vv = U.uaamg_get_level_csr(h, l + 1)
            orp, occ, ovv = mats[l + 1]
            assert np.array_equal(rp, orp) and np.array_equal(cc, occ), l + 1
            assert np.array_equal(bits(vv), bits(ovv)), l + 1
    finally:
        U.uaamg_free(h)
