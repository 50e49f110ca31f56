"""Basis order by overlap signatures (Sec. III-B; appendix "Overlap-Signature
Construction and Basis-Function Clustering", Eq. cosine_distance), FP64.

TEST INFRASTRUCTURE: only tests, the smoke check and the benchmark's CPU
baseline use this module; the library never calls it.

Steps in the paper's order:
  1. overlap signature of each unit: its row of the overlap matrix S;
  2. pairwise cosine distance d(i, j) = 1 - s_i . s_j / (|s_i| |s_j|);
  3. agglomerative clustering with average linkage: start from singletons,
     repeatedly merge the two clusters with the smallest average inter-cluster
     distance until one cluster remains;
  4. at each merge, orient the two sub-trees so that their mutually closest
     leaves are adjacent; the root's leaf order is the permutation.

Readings:
  * units are shells, not single functions (a Cartesian shell's functions share
    centre and exponents, and the kernels evaluate a shell's functions together);
    the signature of shell s is the row of shell-block Frobenius norms
    T_s,t = ||S[s, t]||_F;
  * "mutually closest leaves": of the four end-leaf pairs of the two leaf
    sequences, the pair with the smallest leaf distance d becomes adjacent;
    the lower-numbered cluster goes first, ties in the order (last, first),
    (last, last), (first, first), (first, last);
  * the pair merged is the one with the smallest (distance, lower id, higher
    id); the merged cluster keeps the lower id; the average-linkage update is
    D(a u b, k) = (n_a D(a, k) + n_b D(b, k)) / (n_a + n_b);
  * sums run sequentially in index order (np.cumsum), products are not fused,
    so the library's host implementation returns the same permutation.

Pins (tests/test_oracle_reorder.py): merge heights equal scipy's average
linkage on the same distances; points on a line come out monotonic; shells of
two non-overlapping molecules form two contiguous segments; the result is a
permutation.
"""
from __future__ import annotations

import numpy as np


def _seqsum(x, axis=-1):
    """Sum in index order (no pairwise summation)."""
    return np.take(np.cumsum(x, axis=axis), -1, axis=axis)


def shell_signatures(S: np.ndarray, nfn) -> np.ndarray:
    """T[s, t] = sqrt(sum over the (s, t) block of S of S^2), row-major order."""
    nfn = np.asarray(nfn, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(nfn)])
    n = nfn.size
    T = np.zeros((n, n))
    for s in range(n):
        for t in range(n):
            blk = S[off[s]:off[s + 1], off[t]:off[t + 1]]
            T[s, t] = np.sqrt(_seqsum((blk * blk).ravel()))
    return T


def cosine_distances(T: np.ndarray) -> np.ndarray:
    """d(s, t) = 1 - T_s . T_t / (|T_s| |T_t|) (Eq. cosine_distance)."""
    norm = np.sqrt(_seqsum(T * T, axis=1))
    n = T.shape[0]
    d = np.zeros((n, n))
    for s in range(n):
        dot = _seqsum(T[s][None, :] * T, axis=1)
        d[s] = 1.0 - dot / (norm[s] * norm)
    return d


def cluster_order(d0: np.ndarray, heights: list | None = None) -> np.ndarray:
    """Average-linkage agglomerative clustering of the units with leaf
    distances d0, orienting sub-trees at each merge; returns the leaf order.
    `heights`, if given, receives the merge distances in merge order."""
    n = d0.shape[0]
    D = d0.copy()
    active = np.ones(n, dtype=bool)
    size = np.ones(n)
    leaves = [[s] for s in range(n)]
    upper = np.triu(np.ones((n, n), dtype=bool), k=1)
    for _ in range(n - 1):
        M = np.where(upper & active[:, None] & active[None, :], D, np.inf)
        p, q = np.unravel_index(int(np.argmin(M)), M.shape)   # first minimum in row-major order
        p, q = int(p), int(q)
        if heights is not None:
            heights.append(float(D[p, q]))
        A, B = leaves[p], leaves[q]
        c = [d0[A[-1], B[0]], d0[A[-1], B[-1]], d0[A[0], B[0]], d0[A[0], B[-1]]]
        k = 0
        for j in range(1, 4):
            if c[j] < c[k]:
                k = j
        if k >= 2:
            A = A[::-1]
        if k in (1, 3):
            B = B[::-1]
        leaves[p] = A + B
        leaves[q] = []
        active[q] = False
        others = np.where(active)[0]
        others = others[others != p]
        v = (size[p] * D[p, others] + size[q] * D[q, others]) / (size[p] + size[q])
        D[p, others] = v
        D[others, p] = v
        size[p] = size[p] + size[q]
    root = int(np.where(active)[0][0])
    return np.asarray(leaves[root], dtype=np.int64)


def order_shells(S: np.ndarray, nfn, heights: list | None = None) -> np.ndarray:
    """The shell permutation: position k holds old shell perm[k]."""
    return cluster_order(cosine_distances(shell_signatures(S, nfn)), heights)
