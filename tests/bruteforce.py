"""Brute-force checkers used to pin the oracle and to check the CUDA path's invariants.

Each routine is a different computation from the one the oracle performs (BFS distance
tables instead of 2-hop marking, parallel rounds instead of a greedy scan, dense matrix
products instead of aggregate sums), so a mistake on one side shows as a mismatch.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def adjacency(rowptr, col):
    n = len(rowptr) - 1
    return [[int(c) for c in col[rowptr[i]:rowptr[i + 1]] if c != i] for i in range(n)]


def bfs_distances(adj, src, limit=None):
    dist = {src: 0}
    dq = deque([src])
    while dq:
        u = dq.popleft()
        if limit is not None and dist[u] >= limit:
            continue
        for w in adj[u]:
            if w not in dist:
                dist[w] = dist[u] + 1
                dq.append(w)
    return dist


def within2(adj):
    """within2[i] = set of j != i with graph distance <= 2."""
    out = []
    for i in range(len(adj)):
        d = bfs_distances(adj, i, limit=2)
        out.append({j for j, v in d.items() if 0 < v <= 2})
    return out


def degree_dense(A_dense):
    return (np.abs(A_dense - np.diag(np.diag(A_dense))) > 0).sum(axis=1)


def mis_rounds(P, near2, cand):
    """Fixed-priority parallel rounds with snapshot semantics: every candidate that beats
    all remaining candidates within distance 2 is selected at once; selected vertices and
    the candidates within distance 2 of them leave.  Returns the selected set."""
    cand = set(cand)
    chosen = set()
    while cand:
        snap = set(cand)
        new = {i for i in snap if all(P[i] > P[j] for j in near2[i] if j in snap)}
        assert new, "a round must select the global maximum"
        chosen |= new
        gone = set(new)
        for i in new:
            gone |= (near2[i] & snap)
        cand = snap - gone
    return chosen


def paa_bruteforce(n, adj, P, t, mode):
    """Algorithm 2 from distance tables: passes of (A) a distance-2 independent set of the
    unprocessed vertices (parallel rounds for the maximal mode, one round of strict local
    maxima otherwise) and (B) star aggregates.  Returns (root_of, pass_of)."""
    near2 = within2(adj)
    root_of = -np.ones(n, dtype=np.int64)
    pass_of = -np.ones(n, dtype=np.int64)
    p = 0
    while (root_of < 0).any():
        un = [i for i in range(n) if root_of[i] < 0]
        if mode == 0:
            roots = mis_rounds(P, near2, un)
        else:
            uns = set(un)
            roots = {i for i in un if all(P[i] > P[j] for j in near2[i] if j in uns)}
        for c in sorted(roots):
            root_of[c] = c
            pass_of[c] = p
            taken = 1
            for u in sorted(adj[c]):
                if root_of[u] >= 0:
                    continue
                if t > 0 and taken >= t:
                    break
                root_of[u] = c
                pass_of[u] = p
                taken += 1
        p += 1
    return root_of, pass_of


def prolongator(agg, nc):
    n = len(agg)
    P = np.zeros((n, nc))
    P[np.arange(n), agg] = 1.0
    return P


def l1_minv_dense(A):
    d = np.diag(A)
    off = np.abs(A).sum(axis=1) - np.abs(d)
    return 1.0 / (d + off)


def two_grid_B(A, agg, nc, Ac_inv):
    """Dense matrix of the two-level preconditioner: one l1-Jacobi pre-sweep from zero, an
    exact coarse correction, one post-sweep."""
    n = A.shape[0]
    Mi = np.diag(l1_minv_dense(A))
    P = prolongator(agg, nc)
    I = np.eye(n)
    S = I - Mi @ A
    X2 = Mi + P @ Ac_inv @ P.T @ (I - A @ Mi)
    return S @ X2 + Mi
