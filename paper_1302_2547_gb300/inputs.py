"""Seeded synthetic graph-Laplacian systems (the problem statement of Section 2).

This module holds no part of the multigrid method: it only builds test matrices and
right-hand sides, and both the CUDA path and the CPU oracle read its output.

A graph Laplacian is given by its bilinear form (Section 2):
    (A u, v) = sum_{(i,j) in E} w_ij (u_i - u_j)(v_i - v_j) + sum_{j in S} wD_j u_j v_j,
so a_ij = -w_ij for an edge and a_ii = sum_j w_ij + wD_i.  Matrices are returned as CSR
with int32 row pointers and column indices (columns sorted, diagonal stored) and float64
values.

Workload recipes (all seeded, numpy PCG64):
  * 2D 5-point grid, nx x ny interior, Dirichlet: boundary nodes are eliminated, so every
    edge to the boundary adds its weight to wD (unit weights: diagonal 4, off-diagonal -1).
  * 3D 7-point grid, nx x ny x nz interior, Dirichlet, every edge of the (n+2)^3 grid
    weighted exp(N(0, sigma^2)).
  * Random geometric graph: points uniform in the unit square, radius
    sqrt(mean_degree / (pi N)), unit weights, largest connected component relabelled in
    ascending original order, one vertex (the component's first) pinned with wD = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        A[rows, self.col] = self.val
        return A


def laplacian_from_edges(n: int, ei, ej, w, wD=None, name: str = "") -> CSR:
    """CSR of the weighted graph Laplacian of undirected edges (ei[k], ej[k], w[k]), ei != ej,
    each edge listed once, plus the Dirichlet weights wD (length n, zeros allowed)."""
    from scipy.sparse import csr_matrix

    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    if np.any(ei == ej):
        raise ValueError("self loops are not edges")
    # a_ii: the weights of the row's edges added in edge order (ei occurrences, then ej),
    # then wD
    diag = np.bincount(np.concatenate([ei, ej]), weights=np.concatenate([w, w]), minlength=n)
    if wD is not None:
        diag = diag + np.asarray(wD, dtype=np.float64)
    rows = np.concatenate([ei, ej, np.arange(n)])
    cols = np.concatenate([ej, ei, np.arange(n)])
    vals = np.concatenate([-w, -w, diag])
    if len(rows) >= 2**31:
        raise ValueError("nnz does not fit int32")
    M = csr_matrix((vals, (rows, cols)), shape=(n, n))
    if M.nnz != len(rows):
        raise ValueError("duplicate edge")
    M.sort_indices()
    return CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64),
               name)


def grid2d(nx: int, ny: int | None = None, dirichlet: bool = True, weights=None,
           name: str | None = None) -> CSR:
    """5-point Laplacian on an nx x ny grid of unknowns, index i = x + nx*y.  Dirichlet
    eliminates the surrounding boundary nodes (unit-weight edges to them go to wD);
    Neumann keeps only the interior edges.  `weights=(wx, wy)` overrides unit weights
    (wx shape (ny, nx-1), wy shape (ny-1, nx))."""
    ny = nx if ny is None else ny
    idx = np.arange(nx * ny).reshape(ny, nx)
    hi, hj = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    vi, vj = idx[:-1, :].ravel(), idx[1:, :].ravel()
    if weights is None:
        wh, wv = np.ones(hi.size), np.ones(vi.size)
    else:
        wh, wv = np.asarray(weights[0]).ravel(), np.asarray(weights[1]).ravel()
    wD = np.zeros(nx * ny)
    if dirichlet:
        deg = np.zeros((ny, nx))
        deg[:, 0] += 1
        deg[:, -1] += 1
        deg[0, :] += 1
        deg[-1, :] += 1
        wD = deg.ravel()
    return laplacian_from_edges(nx * ny, np.concatenate([hi, vi]), np.concatenate([hj, vj]),
                                np.concatenate([wh, wv]), wD,
                                name or f"grid2d_{nx}x{ny}_{'dir' if dirichlet else 'neu'}")


def grid3d(nx: int, ny: int | None = None, nz: int | None = None, sigma: float = 0.0,
           seed: int = 0, name: str | None = None) -> CSR:
    """7-point Laplacian on an nx x ny x nz interior grid with Dirichlet boundary, index
    i = x + nx*(y + ny*z).  Every edge of the (nx+2) x (ny+2) x (nz+2) grid that touches an
    unknown gets weight exp(N(0, sigma^2)) (sigma = 0: unit weights); the weights are drawn
    for x-, then y-, then z-edges in C order.  Edges to boundary nodes add to wD."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)

    def draw(shape):
        if sigma == 0.0:
            return np.ones(shape)
        return np.exp(sigma * rng.standard_normal(shape))

    wx = draw((nz, ny, nx + 1))  # edge between x-1 and x, x = 0..nx (0 and nx touch the boundary)
    wy = draw((nz, ny + 1, nx))
    wz = draw((nz + 1, ny, nx))
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    ei = [idx[:, :, :-1].ravel(), idx[:, :-1, :].ravel(), idx[:-1, :, :].ravel()]
    ej = [idx[:, :, 1:].ravel(), idx[:, 1:, :].ravel(), idx[1:, :, :].ravel()]
    w = [wx[:, :, 1:nx].ravel(), wy[:, 1:ny, :].ravel(), wz[1:nz, :, :].ravel()]
    wD = np.zeros((nz, ny, nx))
    wD[:, :, 0] += wx[:, :, 0]
    wD[:, :, -1] += wx[:, :, nx]
    wD[:, 0, :] += wy[:, 0, :]
    wD[:, -1, :] += wy[:, ny, :]
    wD[0, :, :] += wz[0, :, :]
    wD[-1, :, :] += wz[nz, :, :]
    return laplacian_from_edges(nx * ny * nz, np.concatenate(ei), np.concatenate(ej),
                                np.concatenate(w), wD.ravel(),
                                name or f"grid3d_{nx}x{ny}x{nz}_s{sigma}")


def rgg(npts: int, mean_degree: float = 8.0, seed: int = 0, name: str | None = None) -> CSR:
    """Random geometric graph Laplacian (recipe in the module docstring)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((npts, 2))
    r = math.sqrt(mean_degree / (math.pi * npts))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    ei, ej = pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
    g = coo_matrix((np.ones(len(ei), dtype=np.int8), (ei, ej)), shape=(npts, npts))
    ncomp, lab = connected_components(g, directed=False)
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)  # ascending original order
    newid = -np.ones(npts, dtype=np.int64)
    newid[keep] = np.arange(len(keep))
    m = (newid[ei] >= 0) & (newid[ej] >= 0)
    ei, ej = newid[ei[m]], newid[ej[m]]
    a, b = np.minimum(ei, ej), np.maximum(ei, ej)
    wD = np.zeros(len(keep))
    wD[0] = 1.0
    return laplacian_from_edges(len(keep), a, b, np.ones(len(a)), wD,
                                name or f"rgg_{npts}_d{mean_degree}")


def random_graph(n: int, extra_edges: int, seed: int = 0, integer_weights: bool = True,
                 pin: int | None = 0, name: str | None = None) -> CSR:
    """Small connected test graph: a random spanning tree plus `extra_edges` random edges,
    weights in {1..4} (integer) or exp(N(0,1)); vertex `pin` gets wD = 1 (None: Neumann)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    parents = [perm[rng.integers(0, k)] for k in range(1, n)]
    edges = {(min(a, b), max(a, b)) for a, b in zip(perm[1:], parents)}
    tries = 0
    while len(edges) < n - 1 + extra_edges and tries < 100 * (extra_edges + 1):
        a, b = rng.integers(0, n, 2)
        tries += 1
        if a != b:
            edges.add((min(a, b), max(a, b)))
    e = np.array(sorted(edges), dtype=np.int64).reshape(-1, 2)
    if integer_weights:
        w = rng.integers(1, 5, len(e)).astype(np.float64)
    else:
        w = np.exp(rng.standard_normal(len(e)))
    wD = np.zeros(n)
    if pin is not None:
        wD[pin] = 1.0
    return laplacian_from_edges(n, e[:, 0], e[:, 1], w, wD, name or f"random_{n}_{extra_edges}")


def path_graph(n: int, dirichlet: bool = False) -> CSR:
    """Path 0-1-...-(n-1), unit weights; Dirichlet adds wD = 1 at both ends."""
    wD = np.zeros(n)
    if dirichlet:
        wD[0] += 1
        wD[-1] += 1
    return laplacian_from_edges(n, np.arange(n - 1), np.arange(1, n), np.ones(n - 1), wD,
                                f"path_{n}")


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """Right-hand side with entries uniform in [-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


# --- the named workloads ----------------------------------------------------------------

MATRIX_SEED = 1000
RHS_SEED = 2000
MIS_SEED = 0x5EED


def poisson2d_64() -> CSR:
    """2D 5-point Poisson, 64 x 64 interior grid (n = 4096), Dirichlet, unit weights."""
    return grid2d(64, 64, dirichlet=True, name="poisson2d_64x64")


def laplace3d_128(n: int = 128) -> CSR:
    """3D 7-point Laplacian, 128^3 interior grid (n = 2,097,152), Dirichlet, edge weights
    exp(N(0, 0.25^2))."""
    return grid3d(n, n, n, sigma=0.25, seed=MATRIX_SEED + 1, name=f"laplace3d_{n}^3_lognormal0.25")


def rgg_4m(npts: int = 4_000_000) -> CSR:
    """Random geometric graph, 4M points in the unit square, mean degree 8, LCC, one pin."""
    return rgg(npts, 8.0, seed=MATRIX_SEED + 2, name=f"rgg_{npts}_deg8")


def _batch_member(args):
    """System k of batch_mix (a separate function so that a process pool can build it)."""
    k, n, seed = args
    if k % 2 == 0:
        side = max(2, int(round(math.sqrt(n))))
        return grid2d(side, side, name=f"batch{k}_grid2d_{side}")
    return rgg(int(n), 8.0, seed=seed + k, name=f"batch{k}_rgg_{int(n)}")


def batch_mix_sizes(nsys: int = 512, nmin: int = 1024, nmax: int = 262144,
                    seed: int = MATRIX_SEED + 4) -> np.ndarray:
    """Requested sizes of batch_mix: log-uniform in [nmin, nmax]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(nmin), math.log(nmax), nsys)).astype(np.int64)


def batch_mix(nsys: int = 512, nmin: int = 1024, nmax: int = 262144,
              seed: int = MATRIX_SEED + 4, processes: int = 0) -> list:
    """The batched workload: nsys independent systems with sizes log-uniform in
    [nmin, nmax]; even-numbered systems are 2D 5-point Dirichlet grids of side
    round(sqrt(n)) (unit weights), odd-numbered ones random geometric graphs of mean degree 8
    (largest component, one pinned vertex).  processes > 1 builds them in that many spawned
    processes (the systems do not depend on it)."""
    sizes = batch_mix_sizes(nsys, nmin, nmax, seed)
    jobs = [(k, int(n), seed) for k, n in enumerate(sizes)]
    if processes > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_batch_member, jobs, chunksize=4)
    return [_batch_member(j) for j in jobs]


def _serving_base(args):
    kind, n, seed = args
    if kind == 0:
        side = max(8, int(round(math.sqrt(n))))
        return grid2d(side, side, name=f"serve_grid2d_{side}")
    if kind == 1:
        side = max(4, int(round(n ** (1.0 / 3.0))))
        return grid3d(side, sigma=0.25, seed=seed, name=f"serve_grid3d_{side}")
    return rgg(int(n), 8.0, seed=seed, name=f"serve_rgg_{int(n)}")


def serving_bases(per_kind: int = 8, nmin: float = 1e4, nmax: float = 8e6,
                  seed: int = MATRIX_SEED + 5, processes: int = 0) -> list:
    """Base graphs of the serving stream: for each kind (2D grid, 3D grid with lognormal
    weights, random geometric graph of mean degree 8), `per_kind` sizes spaced evenly in
    log between nmin and nmax.  Returns [(kind, size, CSR)], sizes ascending per kind."""
    sizes = np.exp(np.linspace(math.log(nmin), math.log(nmax), per_kind))
    jobs = [(k, float(n), seed + 10 * k + i) for k in range(3) for i, n in enumerate(sizes)]
    if processes > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(processes) as pool:
            mats = pool.map(_serving_base, jobs, chunksize=1)
    else:
        mats = [_serving_base(j) for j in jobs]
    return [(j[0], j[1], m) for j, m in zip(jobs, mats)]
