"""Pins of the CPU oracle against what the paper prints and what the mathematics fixes.

None of these tests touches the GPU.  Each compares the oracle with something other than
itself: values printed in the paper's tables, a hand-worked example, closed forms, dense
linear algebra, brute-force graph searches and exact rational arithmetic.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from tests import bruteforce as BF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------
# The problem (Section 2): generator closed forms
# ---------------------------------------------------------------------------------------

def test_grid2d_dirichlet_closed_form(inputs):
    A = inputs.grid2d(7, 5, dirichlet=True).dense()
    assert np.array_equal(A, A.T)
    assert np.all(np.diag(A) == 4.0)
    off = A - np.diag(np.diag(A))
    assert set(np.unique(off)) <= {0.0, -1.0}
    # row sums = number of eliminated boundary neighbours
    rs = A.sum(axis=1).reshape(5, 7)
    assert rs[2, 3] == 0 and rs[0, 0] == 2 and rs[0, 3] == 1


def test_grid2d_neumann_zero_row_sums(inputs):
    A = inputs.grid2d(6, dirichlet=False).dense()
    assert np.allclose(A.sum(axis=1), 0.0, atol=0)
    assert np.linalg.matrix_rank(A) == A.shape[0] - 1


def test_grid3d_weights_and_dirichlet(inputs):
    Ac = inputs.grid3d(4, 3, 5, sigma=0.25, seed=7)
    A = Ac.dense()
    assert np.array_equal(A, A.T)
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)
    wD = A.sum(axis=1).reshape(5, 3, 4)
    assert abs(wD[2, 1, 1]) < 1e-12  # interior unknown: no boundary edge
    assert np.all(wD[0] > 0) and np.all(wD[:, :, 0] > 0)
    assert np.all(np.linalg.eigvalsh(A) > 0)
    # the full-size workload: n and nnz of the 128^3 grid
    n = 128
    assert n**3 == 2_097_152 and n**3 + 6 * (n - 1) * n * n == 14_581_760


def test_rgg_connected_symmetric(inputs):
    A = inputs.rgg(3000, 8.0, seed=5)
    D = A.dense()
    assert np.array_equal(D, D.T)
    adj = BF.adjacency(A.rowptr, A.col)
    assert len(BF.bfs_distances(adj, 0)) == A.n  # the kept component is connected
    rs = D.sum(axis=1)
    assert rs[0] == 1.0 and np.all(rs[1:] == 0.0)  # one pinned vertex
    assert 6.0 < (A.nnz - A.n) / A.n < 8.5  # mean degree near 8 (border effect lowers it)


# ---------------------------------------------------------------------------------------
# Priority vector, Eq. (3.2)
# ---------------------------------------------------------------------------------------

def _fmix32_inverse(h):
    M = 0xFFFFFFFF
    inv = lambda a: pow(a, -1, 1 << 32)

    def unxorshift(x, s):
        y = x
        for _ in range(32 // s + 1):
            y = x ^ (y >> s)
        return y & M

    h = unxorshift(h, 16)
    h = (h * inv(0xC2B2AE35)) & M
    h = unxorshift(h, 13)
    h = (h * inv(0x85EBCA6B)) & M
    h = unxorshift(h, 16)
    return h


def test_hash_is_a_bijection(oracle):
    rng = np.random.default_rng(1)
    for x in list(rng.integers(0, 2**32, 2000)) + [0, 1, 2**32 - 1]:
        assert _fmix32_inverse(oracle.fmix32(int(x))) == int(x)
    assert oracle.fmix32(0) == 0  # xor-shift / multiply steps fix zero


def test_hash_uniform(oracle):
    h = np.array([oracle.fmix32(i + 12345) for i in range(40000)], dtype=np.uint64)
    counts = np.bincount((h >> np.uint64(28)).astype(np.int64), minlength=16)
    chi2 = ((counts - 2500.0) ** 2 / 2500.0).sum()
    assert chi2 < 40  # 15 dof, p ~ 5e-4


@pytest.mark.parametrize("seed", [0, 0x5EED, 2**40 + 3])
def test_priority_order_matches_eq_3_2(oracle, inputs, seed):
    A = inputs.random_graph(60, 80, seed=3)
    P = oracle.priorities(A.rowptr, A.col, seed, level=2)
    d = BF.degree_dense(A.dense())
    salt = oracle.level_salt(seed, 2)
    v = []
    for i in range(A.n):
        h = oracle.fmix32((i + salt) & 0xFFFFFFFF)
        v.append(Fraction(int(d[i])) + (Fraction(i % 12) + Fraction(h, 2**32)) / 12)
    order_v = sorted(range(A.n), key=lambda i: v[i], reverse=True)
    order_P = sorted(range(A.n), key=lambda i: int(P[i]), reverse=True)
    assert order_v == order_P
    assert len(set(P.tolist())) == A.n


# ---------------------------------------------------------------------------------------
# Algorithm 2 and the coarse operator: hand-worked example
# ---------------------------------------------------------------------------------------

def _load_path_golden():
    cases, band = [], None
    for line in open(os.path.join(GOLDEN, "path5_worked.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("band"):
            band = [int(x) for x in line.split()[1:]]
            continue
        parts = [p.strip() for p in line.split("|")]
        _, mode, t = parts[0].split()
        rec = {"mode": 0 if mode == "maximal" else 1, "t": int(t)}
        for p in parts[1:]:
            k, *vals = p.split()
            rec[k] = [float(x) if k == "val" else int(x) for x in vals]
        cases.append(rec)
    return band, cases


def test_path5_worked_example(oracle, inputs):
    band, cases = _load_path_golden()
    A = inputs.path_graph(5)
    P = oracle.priorities(A.rowptr, A.col, 0x5EED)
    assert [int(p) >> 32 for p in P] == band
    for c in cases:
        ro, po, _ = oracle.paa(A.rowptr, A.col, P, t=c["t"], mode=c["mode"])
        agg, nc = oracle.renumber(ro)
        assert agg.tolist() == c["agg"], c
        assert po.tolist() == c["pass_of"], c
        rp, cc, vv = oracle.coarse(A.rowptr, A.col, A.val, agg, nc)
        assert rp.tolist() == c["rowptr"] and cc.tolist() == c["col"] and vv.tolist() == c["val"]


# ---------------------------------------------------------------------------------------
# Values printed in the paper: Tables 5.1, 5.2, 5.3, 5.6
# ---------------------------------------------------------------------------------------

def _tables():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_tables.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            head, *rest = [p.strip() for p in line.split("|")]
            rows.append((head.split(), [[float(x) for x in r.split()] for r in rest]))
    return rows


def _aggregate(oracle, A, t, mode=1):
    P = oracle.priorities(A.rowptr, A.col, 0x5EED)
    ro, _, _ = oracle.paa(A.rowptr, A.col, P, t=t, mode=mode)
    return oracle.renumber(ro)


def _energy_dirichlet(rowptr, col, val, agg, nc):
    """|Q|_A^2 = largest eigenvalue of A^{-1} Q A Q, Q the l2 projection on range(P)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    n = len(rowptr) - 1
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    P = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))
    cnt = np.asarray(P.sum(axis=0)).ravel()
    Q = lambda v: P @ ((P.T @ v) / cnt)
    lu = sla.splu(A.tocsc())
    op = sla.LinearOperator((n, n), matvec=lambda v: lu.solve(Q(A @ Q(v))), dtype=float)
    return float(np.real(sla.eigs(op, k=1, which="LR", tol=1e-7)[0][0]))


def _energy_neumann(rowptr, col, val, agg, nc):
    """Seminorm version on the complement of the constants."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    n = len(rowptr) - 1
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    P = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))
    cnt = np.asarray(P.sum(axis=0)).ravel()
    Q = lambda v: P @ ((P.T @ v) / cnt)
    proj = lambda v: v - v.mean()

    # For w orthogonal to the constants, A y = w is solved exactly by the matrix with one
    # vertex pinned: summing its rows forces the pinned component of y to zero.
    Ap = A.tolil()
    Ap[0, 0] += 1.0
    lu = sla.splu(Ap.tocsc())

    def pinv(w):
        return proj(lu.solve(proj(w)))

    op = sla.LinearOperator((n, n), matvec=lambda v: pinv(Q(A @ Q(proj(v)))), dtype=float)
    return float(np.real(sla.eigs(op, k=1, which="LR", tol=1e-6)[0][0]))


def test_table_5_1_and_5_2_coarsening_ratios(oracle, inputs):
    for head, vals in _tables():
        if head[0] not in ("table5.1", "table5.2"):
            continue
        A = inputs.grid2d(int(head[2]), dirichlet=(head[1] == "dirichlet"))
        for t, (ratio, _) in zip((2, 3, 4, 5), vals):
            _, nc = _aggregate(oracle, A, t)
            assert round(A.n / nc, 2) == ratio, (head, t, A.n / nc)


def test_table_5_1_energies_n128(oracle, inputs):
    A = inputs.grid2d(128, dirichlet=True)
    row = [v for h, v in _tables() if h[:3] == ["table5.1", "dirichlet", "128"]][0]
    for t, (_, energy) in zip((2, 3, 4, 5), row):
        agg, nc = _aggregate(oracle, A, t)
        assert round(_energy_dirichlet(A.rowptr, A.col, A.val, agg, nc), 2) == energy, t


@pytest.mark.slow
def test_table_5_2_energy_neumann_n128_t5(oracle, inputs):
    A = inputs.grid2d(128, dirichlet=False)
    row = [v for h, v in _tables() if h[:3] == ["table5.2", "neumann", "128"]][0]
    agg, nc = _aggregate(oracle, A, 5)
    assert round(_energy_neumann(A.rowptr, A.col, A.val, agg, nc), 2) == row[3][1]


def test_table_5_3_mod12_patterns(oracle, inputs):
    for head, vals in _tables():
        if head[0] != "table5.3":
            continue
        A = inputs.grid2d(int(head[1]), dirichlet=False)
        for t, ratio in zip((2, 3, 4, 5), vals[0]):
            _, nc = _aggregate(oracle, A, t)
            assert round(A.n / nc, 2) == ratio, (head, t)


def test_table_5_6_multilevel(oracle, inputs):
    A = inputs.grid2d(128, dirichlet=True)
    H = oracle.Hierarchy(A.rowptr, A.col, A.val,
                         oracle.Params(max_agg_size=5, pass_mode=oracle.SINGLE_ROUND, coarse_size=99))
    assert H.num_levels == 6 and H.n(5) < 100  # "the coarsest level we get is level 5"
    for head, vals in _tables():
        if head[0] != "table5.6":
            continue
        l = int(head[1])
        ratio, energy = vals[0]
        assert round(H.n(l) / H.n(l + 1), 2) == ratio
        rp, cc, vv = H.csr(l)
        assert round(_energy_dirichlet(rp, cc, vv, H.agg(l), H.n(l + 1)), 2) == energy


# ---------------------------------------------------------------------------------------
# Algorithm 2: invariants on random graphs, against brute force
# ---------------------------------------------------------------------------------------

GRAPHS = [("random", 40, 30, 1), ("random", 70, 140, 2), ("random", 25, 200, 3),
          ("grid", 9, 0, 0), ("path", 17, 0, 0), ("star", 12, 0, 0)]


def _graph(inputs, kind, n, m, seed):
    if kind == "random":
        return inputs.random_graph(n, m, seed=seed)
    if kind == "grid":
        return inputs.grid2d(n, n - 2, dirichlet=True)
    if kind == "path":
        return inputs.path_graph(n, dirichlet=True)
    return inputs.laplacian_from_edges(n, np.zeros(n - 1, int), np.arange(1, n), np.ones(n - 1),
                                       np.r_[1.0, np.zeros(n - 1)])


@pytest.mark.parametrize("g", GRAPHS)
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("t", [0, 2, 3, 5])
def test_paa_matches_bruteforce(oracle, inputs, g, mode, t):
    A = _graph(inputs, *g)
    adj = BF.adjacency(A.rowptr, A.col)
    P = oracle.priorities(A.rowptr, A.col, 0x5EED, level=1)
    ro, po, npass = oracle.paa(A.rowptr, A.col, P, t=t, mode=mode)
    ro_bf, po_bf = BF.paa_bruteforce(A.n, adj, [int(p) for p in P], t, mode)
    assert ro.tolist() == ro_bf.tolist()
    assert po.tolist() == po_bf.tolist()
    assert npass == po.max() + 1


@pytest.mark.parametrize("g", GRAPHS)
@pytest.mark.parametrize("mode", [0, 1])
def test_paa_invariants(oracle, inputs, g, mode):
    A = _graph(inputs, *g)
    adj = BF.adjacency(A.rowptr, A.col)
    t = 3
    P = oracle.priorities(A.rowptr, A.col, 99)
    ro, po, npass = oracle.paa(A.rowptr, A.col, P, t=t, mode=mode)
    roots = np.flatnonzero(ro == np.arange(A.n))
    # partition into stars of size <= t around each root
    for r in roots:
        members = np.flatnonzero(ro == r)
        assert len(members) <= t
        assert all(m == r or m in adj[r] for m in members)
        assert np.all(po[members] == po[r])
    for p in range(npass):
        rp = [r for r in roots if po[r] == p]
        assert rp, "every pass selects at least one root"
        for a in rp:  # distance >= 3 within a pass, Eq. (3.1)
            d = BF.bfs_distances(adj, a, limit=2)
            assert not any(b in d for b in rp if b != a)
        un = np.flatnonzero(po >= p)
        top = un[np.argmax(P[un])]
        assert ro[top] == top and po[top] == p  # the global maximum is always chosen
        if mode == 0:  # maximal: every other unprocessed vertex is near a chosen root
            for v in un:
                if v in rp:
                    continue
                d = BF.bfs_distances(adj, int(v), limit=2)
                assert any(r in d for r in rp)
    agg, nc = oracle.renumber(ro)
    assert nc == len(roots)
    assert np.all(np.diff(agg[roots]) == 1) and agg[roots[0]] == 0  # Section 5.1 ordering


# ---------------------------------------------------------------------------------------
# Coarse operator, Eq. (2.3)-(2.4)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("integer", [True, False])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_coarse_equals_dense_triple_product(oracle, inputs, integer, seed):
    A = inputs.random_graph(50, 90, seed=seed, integer_weights=integer)
    agg, nc = _aggregate(oracle, A, 4, mode=seed % 2)
    rp, cc, vv = oracle.coarse(A.rowptr, A.col, A.val, agg, nc)
    P = BF.prolongator(agg, nc)
    dense = P.T @ A.dense() @ P
    got = np.zeros((nc, nc))
    rows = np.repeat(np.arange(nc), np.diff(rp))
    got[rows, cc] = vv
    assert np.all(np.diff(cc)[np.diff(rows) == 0] > 0)  # sorted, unique columns
    if integer:
        assert np.array_equal(got, dense)
    else:
        assert np.allclose(got, dense, rtol=1e-13, atol=1e-13)
    # structural pattern: every aggregate pair touched by a stored entry
    touched = (P.T @ (A.dense() != 0).astype(float) @ P) > 0
    assert np.array_equal(touched, np.isin(np.arange(nc * nc).reshape(nc, nc),
                                           rows * nc + cc))


def test_coarse_row_sums(oracle, inputs):
    A = inputs.random_graph(80, 120, seed=9, integer_weights=True, pin=None)  # Neumann
    agg, nc = _aggregate(oracle, A, 0)
    rp, cc, vv = oracle.coarse(A.rowptr, A.col, A.val, agg, nc)
    rows = np.repeat(np.arange(nc), np.diff(rp))
    assert np.all(np.bincount(rows, weights=vv, minlength=nc) == 0.0)
    B = inputs.grid2d(12, dirichlet=True)  # Dirichlet: coarse row sum = sum of wD
    agg, nc = _aggregate(oracle, B, 5)
    rp, cc, vv = oracle.coarse(B.rowptr, B.col, B.val, agg, nc)
    rows = np.repeat(np.arange(nc), np.diff(rp))
    wD = B.dense().sum(axis=1)
    assert np.array_equal(np.bincount(rows, weights=vv, minlength=nc),
                          np.bincount(agg, weights=wD, minlength=nc))


# ---------------------------------------------------------------------------------------
# Smoother (Section 4.1) and the coarsest solve
# ---------------------------------------------------------------------------------------

def test_l1_jacobi_closed_form(oracle, inputs):
    A = inputs.grid2d(6, dirichlet=True)
    m = oracle.minv(A.rowptr, A.col, A.val).reshape(6, 6)
    assert m[2, 2] == 1 / 8 and m[0, 2] == 1 / 7 and m[0, 0] == 1 / 6


def test_cholesky(oracle):
    rng = np.random.default_rng(0)
    for m in (1, 5, 40):
        X = rng.standard_normal((m, m))
        S = X @ X.T + m * np.eye(m)
        L = oracle.cholesky(S)
        assert np.allclose(L @ L.T, S, rtol=1e-13, atol=1e-12)
        b = rng.standard_normal(m)
        assert np.allclose(oracle.cholesky_solve(L, b), np.linalg.solve(S, b), rtol=1e-10)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


# ---------------------------------------------------------------------------------------
# Solve phase: two-level operator, K-cycle, outer flexible CG
# ---------------------------------------------------------------------------------------

def test_two_level_operator_is_the_dense_formula(oracle, inputs):
    A = inputs.grid2d(10, dirichlet=True)
    H = oracle.Hierarchy(A.rowptr, A.col, A.val, oracle.Params(max_levels=2, coarse_size=64))
    assert H.num_levels == 2
    agg, nc = H.agg(0), H.n(1)
    rp, cc, vv = H.csr(1)
    Ac = np.zeros((nc, nc))
    Ac[np.repeat(np.arange(nc), np.diff(rp)), cc] = vv
    B = BF.two_grid_B(A.dense(), agg, nc, np.linalg.inv(Ac))
    rng = np.random.default_rng(4)
    for _ in range(3):
        r = rng.standard_normal(A.n)
        assert np.allclose(H.apply_B(0, r), B @ r, rtol=1e-11, atol=1e-12)
    x, y = rng.standard_normal(A.n), rng.standard_normal(A.n)
    assert abs(y @ H.apply_B(0, x) - x @ H.apply_B(0, y)) < 1e-10 * np.linalg.norm(x) * np.linalg.norm(y)


def test_kcycle_is_two_step_cg(oracle, inputs):
    """With three levels, K_1 = two CG steps on A_1 e = rho preconditioned by the (linear,
    symmetric) two-level B_1: the A_1-orthogonal projection of A_1^{-1} rho onto
    span{B_1 rho, B_1 A_1 B_1 rho}."""
    A = inputs.grid2d(14, dirichlet=True)
    H = oracle.Hierarchy(A.rowptr, A.col, A.val, oracle.Params(max_levels=3, coarse_size=8))
    assert H.num_levels == 3
    rp, cc, vv = H.csr(1)
    n1 = H.n(1)
    A1 = np.zeros((n1, n1))
    A1[np.repeat(np.arange(n1), np.diff(rp)), cc] = vv
    rp2, cc2, vv2 = H.csr(2)
    A2 = np.zeros((H.n(2), H.n(2)))
    A2[np.repeat(np.arange(H.n(2)), np.diff(rp2)), cc2] = vv2
    B1 = BF.two_grid_B(A1, H.agg(1), H.n(2), np.linalg.inv(A2))
    rho = np.random.default_rng(8).standard_normal(n1)
    V = np.stack([B1 @ rho, B1 @ A1 @ B1 @ rho], axis=1)
    c = np.linalg.solve(V.T @ A1 @ V, V.T @ rho)
    assert np.allclose(H.apply_K(1, rho), V @ c, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("case", ["grid", "random", "rgg"])
def test_solve_against_dense(oracle, inputs, case):
    A = {"grid": lambda: inputs.grid2d(20, dirichlet=True),
         "random": lambda: inputs.random_graph(300, 500, seed=4, integer_weights=False),
         "rgg": lambda: inputs.rgg(900, 8.0, seed=2)}[case]()
    b = inputs.rhs_uniform(A.n, 11)
    H = oracle.Hierarchy(A.rowptr, A.col, A.val, oracle.Params(coarse_size=16, max_agg_size=0))
    assert H.num_levels >= 3
    x, it, rr, st, hist = H.solve(b, 1e-10)
    D = A.dense()
    assert st == 0 and rr <= 1e-10
    assert np.linalg.norm(b - D @ x) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
    xs = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.cond(D) * np.linalg.norm(xs)
    assert len(hist) == it + 1 and hist[-1] <= 1e-10


def test_solve_edge_cases(oracle, inputs):
    A = inputs.grid2d(16, dirichlet=True)
    H = oracle.Hierarchy(A.rowptr, A.col, A.val)
    x, it, rr, st, _ = H.solve(np.zeros(A.n))
    assert it == 0 and st == 0 and np.all(x == 0)
    b = inputs.rhs_uniform(A.n, 1)
    xs = np.linalg.solve(A.dense(), b)
    x, it, rr, st, _ = H.solve(b, 1e-8, x0=xs)
    assert it == 0 and st == 0
    small = inputs.grid2d(6, dirichlet=True)  # n = 36 <= coarse_size: one level, exact
    Hs = oracle.Hierarchy(small.rowptr, small.col, small.val)
    assert Hs.num_levels == 1
    x, it, rr, st, _ = Hs.solve(inputs.rhs_uniform(36, 2), 1e-12)
    assert it == 1 and rr < 1e-13


def test_iterations_roughly_flat_in_n(oracle, inputs):
    """Table 5.9 reports the same iteration count at 1M and 4M unknowns; here the count to
    1e-8 may grow slowly with n but stays in a narrow band (plausibility, not parity)."""
    its = []
    for n in (32, 64, 128, 256):
        A = inputs.grid2d(n, dirichlet=True)
        H = oracle.Hierarchy(A.rowptr, A.col, A.val)
        _, it, rr, st, _ = H.solve(inputs.rhs_uniform(A.n, 3), 1e-8)
        assert st == 0
        its.append(it)
    assert max(its) <= 1.6 * min(its) and max(its) <= 30, its


# ---------------------------------------------------------------------------------------
# Aggregating twice per level (Section 3.3) and the K-cycle safeguards
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("integer", [True, False])
def test_double_aggregation_is_two_stages(oracle, inputs, integer):
    """The level's aggregates are unions of first-stage aggregates (agg = agg2[agg1]) and the
    next matrix is Eq. 2.4 applied twice; with integer weights it equals the one-shot dense
    product (P1 P2)^T A (P1 P2) exactly."""
    A = inputs.random_graph(400, 900, seed=5, integer_weights=integer)
    H = oracle.Hierarchy(A.rowptr, A.col, A.val,
                         oracle.Params(agg_repeat=2, max_agg_size=4, coarse_size=8))
    P1 = oracle.priorities(A.rowptr, A.col, 0x5EED, level=0)
    r1, _, _ = oracle.paa(A.rowptr, A.col, P1, t=4, mode=1)
    a1, n1 = oracle.renumber(r1)
    rp1, cc1, vv1 = oracle.coarse(A.rowptr, A.col, A.val, a1, n1)
    P2 = oracle.priorities(rp1, cc1, 0x5EED, level=1)
    r2, _, _ = oracle.paa(rp1, cc1, P2, t=4, mode=1)
    a2, n2 = oracle.renumber(r2)
    assert n2 < n1 and H.n(1) == n2
    assert np.array_equal(H.agg(0), a2[a1])
    rp2, cc2, vv2 = oracle.coarse(rp1, cc1, vv1, a2, n2)
    hrp, hcc, hvv = H.csr(1)
    assert np.array_equal(hrp, rp2) and np.array_equal(hcc, cc2) and np.array_equal(hvv, vv2)
    P = BF.prolongator(a2[a1], n2)
    dense = P.T @ A.dense() @ P
    got = np.zeros((n2, n2))
    got[np.repeat(np.arange(n2), np.diff(hrp)), hcc] = hvv
    if integer:
        assert np.array_equal(got, dense)
    else:
        assert np.allclose(got, dense, rtol=1e-12, atol=1e-12)


def test_one_step_levels_under_the_ratio_rule(oracle, inputs):
    """With kcycle_ratio above every coarsening ratio, K_1 is one flexible-CG step:
    e = ((c1, rho) / (c1, A c1)) c1 with c1 = B_1 rho (dense two-level B_1)."""
    A = inputs.grid2d(14, dirichlet=True)
    H = oracle.Hierarchy(A.rowptr, A.col, A.val,
                         oracle.Params(max_levels=3, coarse_size=8, kcycle_ratio=1e9))
    assert H.num_levels == 3
    rp, cc, vv = H.csr(1)
    n1 = H.n(1)
    A1 = np.zeros((n1, n1))
    A1[np.repeat(np.arange(n1), np.diff(rp)), cc] = vv
    rp2, cc2, vv2 = H.csr(2)
    A2 = np.zeros((H.n(2), H.n(2)))
    A2[np.repeat(np.arange(H.n(2)), np.diff(rp2)), cc2] = vv2
    B1 = BF.two_grid_B(A1, H.agg(1), H.n(2), np.linalg.inv(A2))
    rho = np.random.default_rng(3).standard_normal(n1)
    c1 = B1 @ rho
    assert np.allclose(H.apply_K(1, rho), (c1 @ rho) / (c1 @ A1 @ c1) * c1, rtol=1e-10,
                       atol=1e-13)


def test_stagnation_stop(oracle, inputs):
    A = inputs.grid2d(64, dirichlet=True)
    full = oracle.Hierarchy(A.rowptr, A.col, A.val)
    stop = oracle.Hierarchy(A.rowptr, A.col, A.val, oracle.Params(min_coarsening=1e9))
    # the first level with at most 1024 unknowns becomes the coarsest
    first_small = next(l for l in range(full.num_levels) if full.n(l) <= 1024)
    assert stop.num_levels == first_small + 1
    assert [stop.n(l) for l in range(stop.num_levels)] == \
           [full.n(l) for l in range(first_small + 1)]
    b = inputs.rhs_uniform(A.n, 1)
    x, it, rr, st, _ = stop.solve(b, 1e-10)
    assert st == 0 and np.linalg.norm(b - A.dense() @ x) <= 1e-10 * np.linalg.norm(b) * 1.0001


def test_damped_jacobi_closed_form_and_solve(oracle, inputs):
    """Damped Jacobi (Section 4.1): Minv_i = omega / a_ii, and the hierarchy still solves."""
    A = inputs.grid2d(40, dirichlet=True)
    H = oracle.Hierarchy(A.rowptr, A.col, A.val, oracle.Params(jacobi_omega=0.6))
    assert np.all(H.minv(0) == 0.6 / 4.0)
    rp, cc, vv = H.csr(1)
    d = vv[np.concatenate([np.flatnonzero(cc[rp[i]:rp[i + 1]] == i) + rp[i]
                           for i in range(H.n(1))])]
    assert np.array_equal(H.minv(1), 0.6 / d)
    b = inputs.rhs_uniform(A.n, 3)
    x, it, rr, st, _ = H.solve(b, 1e-8)
    assert st == 0 and np.linalg.norm(b - A.dense() @ x) <= 1e-8 * np.linalg.norm(b) * 1.0001


@pytest.mark.parametrize("side", [14, 17])
def test_kcycle_tau_threshold(oracle, inputs, side):
    """The K-cycle threshold (Section 4.3, Notay's tau): the second flexible-CG step is
    skipped exactly when |rho~| <= tau |rho|.  Just above the actual ratio K_1 is the one-step
    e = (alpha1 / rho1) c1; just below it is the two-step combination, both computed densely
    from the two-level B_1."""
    A = inputs.grid2d(side, dirichlet=True)
    base = oracle.Hierarchy(A.rowptr, A.col, A.val, oracle.Params(max_levels=3, coarse_size=8))
    assert base.num_levels == 3
    rp, cc, vv = base.csr(1)
    n1 = base.n(1)
    A1 = np.zeros((n1, n1))
    A1[np.repeat(np.arange(n1), np.diff(rp)), cc] = vv
    rp2, cc2, vv2 = base.csr(2)
    n2 = base.n(2)
    A2 = np.zeros((n2, n2))
    A2[np.repeat(np.arange(n2), np.diff(rp2)), cc2] = vv2
    B1 = BF.two_grid_B(A1, base.agg(1), n2, np.linalg.inv(A2))
    rho = np.random.default_rng(side).standard_normal(n1)
    c1 = B1 @ rho
    v1 = A1 @ c1
    rho1, alpha1 = c1 @ v1, c1 @ rho
    rt = rho - (alpha1 / rho1) * v1
    ratio = np.linalg.norm(rt) / np.linalg.norm(rho)
    c2 = B1 @ rt
    v2 = A1 @ c2
    gamma, beta, alpha2 = c2 @ v1, c2 @ v2, c2 @ rt
    rho2 = beta - gamma * gamma / rho1
    two = (alpha1 / rho1 - gamma * alpha2 / (rho1 * rho2)) * c1 + (alpha2 / rho2) * c2
    one = (alpha1 / rho1) * c1
    for tau, expect in ((ratio * 1.01, one), (ratio * 0.99, two)):
        H = oracle.Hierarchy(A.rowptr, A.col, A.val,
                             oracle.Params(max_levels=3, coarse_size=8, kcycle_tau=tau))
        assert np.allclose(H.apply_K(1, rho), expect, rtol=1e-9, atol=1e-12), tau
    assert not np.allclose(one, two, rtol=1e-3)


@pytest.mark.parametrize("pre,post", [(0, 1), (1, 0), (2, 2), (3, 1)])
@pytest.mark.parametrize("omega", [0.0, 0.7])
def test_two_level_error_propagation(oracle, inputs, pre, post, omega):
    """Any number of smoothing sweeps (Algorithm 1 solve phase, Section 4.1): the two-level
    B_0 satisfies I - B_0 A = S^post (I - P A_c^{-1} P^T A) S^pre with S = I - M^{-1} A
    (l1-Jacobi, or damped Jacobi omega D^{-1}), from the closed forms of M^{-1}."""
    A = inputs.grid2d(12, 9, dirichlet=True)
    Ad = A.dense()
    H = oracle.Hierarchy(A.rowptr, A.col, A.val,
                         oracle.Params(max_levels=2, pre=pre, post=post, jacobi_omega=omega))
    assert H.num_levels == 2
    n, nc = A.n, H.n(1)
    P = BF.prolongator(H.agg(0), nc)
    Mi = np.diag(omega / np.diag(Ad)) if omega > 0 else np.diag(BF.l1_minv_dense(Ad))
    S = np.eye(n) - Mi @ Ad
    CG = np.eye(n) - P @ np.linalg.solve(P.T @ Ad @ P, P.T @ Ad)
    E = np.linalg.matrix_power(S, post) @ CG @ np.linalg.matrix_power(S, pre)
    B = (np.eye(n) - E) @ np.linalg.inv(Ad)
    rng = np.random.default_rng(pre * 10 + post)
    for _ in range(3):
        r = rng.standard_normal(n)
        assert np.allclose(H.apply_B(0, r), B @ r, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("side", [24, 31])
def test_outer_iteration_is_pcg_for_a_linear_preconditioner(oracle, inputs, side):
    """With two levels B_0 is linear and symmetric positive definite, and the outer flexible
    CG with one stored direction (Sections 1 and 4.4) must coincide with textbook
    preconditioned CG (Hestenes-Stiefel recurrences) run with the dense B_0."""
    A = inputs.grid2d(side, dirichlet=True)
    Ad = A.dense()
    H = oracle.Hierarchy(A.rowptr, A.col, A.val, oracle.Params(max_levels=2))
    assert H.num_levels == 2
    nc = H.n(1)
    P = BF.prolongator(H.agg(0), nc)
    B = BF.two_grid_B(Ad, H.agg(0), nc, np.linalg.inv(P.T @ Ad @ P))
    b = inputs.rhs_uniform(A.n, side)
    x, it, rr, st, hist = H.solve(b, 1e-10)
    assert st == 0
    # textbook PCG from x0 = 0
    r = b.copy()
    z = B @ r
    p = z.copy()
    rz = r @ z
    ref = [1.0]
    for _ in range(it + 2):
        q = Ad @ p
        alpha = rz / (p @ q)
        r = r - alpha * q
        ref.append(np.linalg.norm(r) / np.linalg.norm(b))
        z = B @ r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    k = min(8, it)
    assert np.allclose(hist[: k + 1], ref[: k + 1], rtol=1e-6)
    # PCG first reaches the tolerance within one iteration of the oracle's count
    first = next(j for j, v in enumerate(ref) if v <= 1e-10)
    assert abs(first - it) <= 1


def test_oracle_params_mirror_the_c_struct(oracle):
    """The ctypes mirror of the oracle's parameter struct has the C struct's fields in order."""
    import re

    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "oracle", "uaamg_oracle.c")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct or_params \{(.*?)\} or_params;", src, re.S).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            parts = [p.strip() for p in decl.split(",")]
            names.append(re.findall(r"(\w+)\s*$", parts[0])[0])
            names += [re.findall(r"(\w+)\s*$", p)[0] for p in parts[1:]]
    assert names == [f for f, _ in oracle._Params._fields_]
