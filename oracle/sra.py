"""Plain FP64 statement of subgraph reshaping (Section 3.2, Algorithm 3, Eq. 3.8).

TEST INFRASTRUCTURE ONLY: imported by the tests.  The product package never imports this
module, and it shares no code with the CUDA sources.

What it computes, step by step as the paper states it:

* Pair problem (Section 3.2).  For two neighbouring aggregates V1, V2 with union U (sorted
  ascending fine indices u_0 < ... < u_{n-1}), A_hat is the graph Laplacian of the subgraph
  induced by U: A_hat[k, l] = a(u_k, u_l) for k != l and A_hat[k, k] = -sum_{l != k}
  A_hat[k, l] (row sum in ascending l).  Two local vertices are neighbours when that
  entry is non-zero.  The local smoother R_hat is l1-Jacobi on A_hat (Section 4.1), and
  S_hat = I - R_hat A_hat.
* Coarse space of a split (S, S^c): psi = 1_S / |S| - 1_{S^c} / |S^c|.  Q is the
  A_hat-orthogonal projection onto span{psi}, and T = Q S_hat.
* Energy of a split: the trace of the rank-one W = S_hat^T A_hat Q S_hat A_hat^+ (pseudo
  inverse), computed by the rank-one trace rule of Eq. 3.8.
* Algorithm 3: among the splits with |S| = floor(n/2) whose two halves both induce connected
  subgraphs, take the one of largest energy.

Readings where the paper is silent, ambiguous or garbled:

* Eq. 3.8 as printed (column times column over the diagonal entry) is exact only for a
  symmetric rank-one W.  The W above is not symmetric, so the oracle uses row k times column
  k over W_kk, which equals the printed rule whenever W is symmetric.  The paper takes the
  first k with W_kk != 0.  In floating point the oracle takes the first k with |W_kk| at
  least 1e-8 times the largest |W_jj|.
* The paper states that the trace equals |T|_A.  It is |T|_A squared.  The argmax is the
  same.
* Each unordered split is a candidate once.  For an even n, S is the half that holds local
  vertex 0.  A candidate also needs a positive cut 1_S^T A_hat 1_S.  Symmetric splits have
  mathematically equal energies that FP64 rounds apart.  So energies within a relative
  TIE_REL count as equal: scanning the masks sum_{k in S} 2^k in ascending order, a
  candidate replaces the best one only when its energy exceeds it by more than that.  The
  half holding local vertex 0 keeps the smaller of the two aggregate numbers.  A pair
  without a candidate stays unchanged.
* The paper traverses the pairs of neighbouring aggregates without fixing an order.  Here a
  level is reshaped in rounds, and each round reshapes the pairs of a matching at once:
  - Aggregates I != J are neighbours when a stored fine entry a_st != 0 joins them.
  - A pair is eligible when |I| + |J| <= UNION_MAX.
  - In round r of level l, the pair {I, J} with I < J has the weight
    omega = fmix32(fmix32(I ^ s) + J), where s = fmix32(seed32 + 0x9E3779B9 * (64 l + r + 1))
    and seed32 = low 32 bits of (seed ^ (seed >> 32)).
  - Every aggregate proposes to the eligible neighbour of largest omega; equal weights go
    to the smaller J.  Mutual proposals are the round's pairs.
  - All pairs of a round are reshaped from the aggregation at the start of that round.
"""
from __future__ import annotations

import numpy as np

UNION_MAX = 16
TIE_REL = 1e-9
_M32 = 0xFFFFFFFF


# ---------------------------------------------------------------------------------------
# Hash used by the matching: the MurmurHash3 32-bit finalizer (Appleby, 2011)
# ---------------------------------------------------------------------------------------
def fmix32(h):
    """Vectorised MurmurHash3 finalizer on uint32 values (numpy wraps the products)."""
    h = np.asarray(h, dtype=np.uint32).copy()
    h ^= h >> np.uint32(16)
    h *= np.uint32(0x85EBCA6B)
    h ^= h >> np.uint32(13)
    h *= np.uint32(0xC2B2AE35)
    h ^= h >> np.uint32(16)
    return h


def round_salt(seed: int, level: int, rnd: int) -> int:
    seed32 = (seed ^ (seed >> 32)) & _M32
    return int(fmix32(np.uint32((seed32 + 0x9E3779B9 * (64 * level + rnd + 1)) & _M32)))


def pair_weight(I, J, salt: int):
    """omega(I, J) for I < J (arrays allowed)."""
    with np.errstate(over="ignore"):
        a = fmix32(np.asarray(I, dtype=np.uint32) ^ np.uint32(salt))
        return fmix32(a + np.asarray(J, dtype=np.uint32))


# ---------------------------------------------------------------------------------------
# The pair problem, Section 3.2
# ---------------------------------------------------------------------------------------
def local_laplacian(rowptr, col, val, U):
    """A_hat of the subgraph induced by the sorted vertex list U."""
    n = len(U)
    pos = {int(u): k for k, u in enumerate(U)}
    A = np.zeros((n, n))
    for k, s in enumerate(U):
        for q in range(rowptr[s], rowptr[s + 1]):
            t = int(col[q])
            if t != s and t in pos:
                A[k, pos[t]] = val[q]
    for k in range(n):
        d = 0.0
        for l in range(n):
            if l != k:
                d += A[k, l]
        A[k, k] = -d
    return A


def l1_jacobi(A_hat):
    """R_hat = diag(1 / (a_kk + sum_{l != k} |a_kl|)), Section 4.1 (0 where that sum is 0)."""
    n = A_hat.shape[0]
    r = np.zeros(n)
    for k in range(n):
        m = A_hat[k, k] + sum(abs(A_hat[k, l]) for l in range(n) if l != k)
        r[k] = 1.0 / m if m != 0.0 else 0.0
    return np.diag(r)


def psi_of(n, S):
    S = set(int(k) for k in S)
    return np.array([1.0 / len(S) if k in S else -1.0 / (n - len(S)) for k in range(n)])


def a_projection(A_hat, w):
    """Q: the A_hat-orthogonal projection onto span{w}, Q v = w (w^T A_hat v) / (w^T A_hat w)."""
    return np.outer(w, A_hat @ w) / float(w @ A_hat @ w)


def rank_one_trace(W):
    """Eq. 3.8 for a rank-one W: (row k . column k) / W_kk for the first usable k."""
    d = np.abs(np.diag(W))
    big = d.max()
    if big == 0.0:
        return 0.0
    for k in range(W.shape[0]):
        if d[k] >= 1e-8 * big:
            return float(W[k, :] @ W[:, k]) / float(W[k, k])
    return 0.0


def t_energy(A_hat, R_hat, w, A_pinv=None):
    """|T(span w)|_A^2 as the trace of W = S^T A Q S A^+ (Section 3.2, Eq. 3.8)."""
    n = A_hat.shape[0]
    S_hat = np.eye(n) - R_hat @ A_hat
    Q = a_projection(A_hat, w)
    if A_pinv is None:
        A_pinv = np.linalg.pinv(A_hat)
    W = S_hat.T @ A_hat @ Q @ S_hat @ A_pinv
    return rank_one_trace(W)


def connected(adj, mask: int) -> bool:
    """True iff the local vertices of `mask` induce a connected subgraph (depth-first walk)."""
    members = [k for k in range(len(adj)) if mask >> k & 1]
    if not members:
        return False
    seen = {members[0]}
    stack = [members[0]]
    while stack:
        k = stack.pop()
        for l in adj[k]:
            if mask >> l & 1 and l not in seen:
                seen.add(l)
                stack.append(l)
    return len(seen) == len(members)


def candidates(A_hat):
    """Algorithm 3 step (2): masks of the admissible splits, in ascending mask order."""
    n = A_hat.shape[0]
    m = n // 2
    adj = [[l for l in range(n) if l != k and A_hat[k, l] != 0.0] for k in range(n)]
    full = (1 << n) - 1
    out = []
    for mask in range(1, full):
        if bin(mask).count("1") != m:
            continue
        if n % 2 == 0 and not (mask & 1):
            continue
        if not (connected(adj, mask) and connected(adj, full ^ mask)):
            continue
        ind = np.array([(mask >> k) & 1 for k in range(n)], dtype=np.float64)
        if float(ind @ A_hat @ ind) <= 0.0:
            continue
        out.append(mask)
    return out


def reshape_pair(A_hat):
    """Algorithm 3 on a pair's local Laplacian.

    Returns (best_mask, energies) where energies maps every candidate mask to its energy,
    or (None, {}) when there is no admissible split.
    """
    n = A_hat.shape[0]
    R_hat = l1_jacobi(A_hat)
    A_pinv = np.linalg.pinv(A_hat)
    energies = {}
    for mask in candidates(A_hat):
        S = [k for k in range(n) if mask >> k & 1]
        energies[mask] = t_energy(A_hat, R_hat, psi_of(n, S), A_pinv)
    if not energies:
        return None, {}
    best = None
    for mask in sorted(energies):
        if best is None or energies[mask] > energies[best] + TIE_REL * abs(energies[best]):
            best = mask
    return best, energies


# ---------------------------------------------------------------------------------------
# One level: rounds of matched pairs
# ---------------------------------------------------------------------------------------
def members_of(agg, nc):
    order = np.argsort(agg, kind="stable")
    ptr = np.zeros(nc + 1, dtype=np.int64)
    np.add.at(ptr, np.asarray(agg, dtype=np.int64) + 1, 1)
    return np.cumsum(ptr), order


def matching(rowptr, col, val, agg, nc, salt):
    """The round's pairs as a list of (I, J), I < J, ascending I."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val)
    agg = np.asarray(agg, dtype=np.int64)
    n = len(rowptr) - 1
    size = np.bincount(agg, minlength=nc)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    I = agg[rows]
    J = agg[col]
    keep = (I != J) & (val != 0.0) & (size[I] + size[J] <= UNION_MAX)
    I, J = I[keep], J[keep]
    lo, hi = np.minimum(I, J), np.maximum(I, J)
    w = pair_weight(lo, hi, salt).astype(np.uint64)
    key = (w << np.uint64(32)) | (np.uint64(_M32) - J.astype(np.uint64))
    prop = np.zeros(nc, dtype=np.uint64)
    np.maximum.at(prop, I, key)
    partner = np.where(prop == 0, -1, (np.uint64(_M32) - (prop & np.uint64(_M32))).astype(np.int64))
    pairs = []
    for a in range(nc):
        b = partner[a]
        if b > a and partner[b] == a:
            pairs.append((a, int(b)))
    return pairs


def reshape_round(rowptr, col, val, agg, nc, seed, level, rnd, record=None):
    """One round: returns the new aggregation (a copy).  `record`, if a list, receives one
    (I, J, U, best_mask, energies) per matched pair."""
    agg = np.asarray(agg, dtype=np.int32).copy()
    salt = round_salt(seed, level, rnd)
    ptr, order = members_of(agg, nc)
    for I, J in matching(rowptr, col, val, agg, nc, salt):
        U = np.sort(np.concatenate([order[ptr[I]:ptr[I + 1]], order[ptr[J]:ptr[J + 1]]]))
        A_hat = local_laplacian(rowptr, col, val, U)
        best, energies = reshape_pair(A_hat)
        if record is not None:
            record.append((I, J, U, best, energies))
        if best is None:
            continue
        first = I if best & 1 else J  # the half holding local vertex 0 keeps min(I, J) = I
        other = J if first == I else I
        for k, u in enumerate(U):
            agg[u] = first if best >> k & 1 else other
    return agg


def reshape_level(rowptr, col, val, agg, nc, seed, level, rounds):
    for r in range(rounds):
        agg = reshape_round(rowptr, col, val, agg, nc, seed, level, r)
    return agg
