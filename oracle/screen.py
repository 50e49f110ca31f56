"""Block-level filtering and executable-pair selection (paper Sec. III-B-1,
Eq. block_matmul; Sec. III-B-3, Eqs. block_summary_A..retained_blocks_B;
Sec. III-C-1, Eqs. block_pair_filter, executed_block_pairs; App. D, Alg. 1).

Blocks: basis block p = functions [32 p, min(32 p + 32, N_basis)) of the
basis order; grid block g = points [128 g, 128 g + 128).

Readings (the paper defines the rule for a generic product C = A B):
  * summary of a Phi block: b_gp = max |phi_mu(r_i)| over i in g, mu in p;
    for the GGA also over the three gradient components (the matrix the
    paper calls Psi).  Retained set S_g = {p : b_gp >= t_b}.
  * D block summary d_pq = max |D_mu nu| (Eq. block_summary_A with A = D).
  * density product R = Phi_g D: executed pairs
      E1_g = {(p, q) in S_g x S_g : d_pq >= t_b and b_gp d_pq b_gq >= t_d},
    i.e. the pair rule a b >= t_d with the row-dot factor b_gp of the
    following rho = sum Phi . R also applied, which makes E1_g symmetric.
  * potential product Phi^T X: executed pairs
      E2_g = {(p, q) in S_g x S_g : x_gq >= t_b and b_gp x_gq >= t_d},
    x_gq = max |X_i nu| over i in g, nu in q.
  * the symmetric potential V = Phi^T X + X^T Phi: block (p, q) of grid
    block g's contribution is computed, both terms, when (p, q) or (q, p)
    is in E2_g (the paper writes only the symmetric LDA product
    Phi^T W Phi, whose block pair {p, q} is one block of one product; the
    rule is applied to the unordered pair, so no block gets one of its two
    terms without the other).

Pins (tests): Alg. 1 against numpy.nonzero; the pair sets against a
brute-force triple loop over elements.
"""
from __future__ import annotations

import numpy as np

D_BASIS = 32


def nbasis_blocks(nbf: int, d: int = D_BASIS) -> int:
    return (nbf + d - 1) // d


def block_max_cols(M: np.ndarray, d: int = D_BASIS) -> np.ndarray:
    """max |M[:, cols of block p]| for each column block p (rows = one grid block)."""
    nb = nbasis_blocks(M.shape[-1], d)
    out = np.zeros(nb)
    A = np.abs(M)
    for p in range(nb):
        out[p] = A[..., p * d:(p + 1) * d].max()
    return out


def d_block_max(D: np.ndarray, d: int = D_BASIS) -> np.ndarray:
    nb = nbasis_blocks(D.shape[0], d)
    out = np.zeros((nb, nb))
    A = np.abs(D)
    for p in range(nb):
        for q in range(nb):
            out[p, q] = A[p * d:(p + 1) * d, q * d:(q + 1) * d].max()
    return out


def retained(b: np.ndarray, t_b: float) -> np.ndarray:
    """S = {p : summary >= t_b} (Eq. block_filter_A), ascending."""
    return np.nonzero(b >= t_b)[0]


def executed_rho(S: np.ndarray, b: np.ndarray, dmax: np.ndarray, t_b: float, t_d: float) -> np.ndarray:
    """Boolean matrix over S x S of E1_g."""
    bp = b[S]
    dd = dmax[np.ix_(S, S)]
    return (dd >= t_b) & (bp[:, None] * dd * bp[None, :] >= t_d)


def executed_v(S: np.ndarray, b: np.ndarray, x: np.ndarray, t_b: float, t_d: float) -> np.ndarray:
    """Boolean matrix over S x S of E2_g (row p: Phi block, column q: X block)."""
    bp = b[S]
    xq = x[S]
    return (xq[None, :] >= t_b) & (bp[:, None] * xq[None, :] >= t_d)


def parallel_addressing(mask: np.ndarray):
    """App. D, Alg. 1: exclusive prefix sum P over the 0/1 mask (length n+1);
    S = P[n]; every position t with P[t] != P[t+1] writes t to I[P[t+1]-1]."""
    m = np.asarray(mask, dtype=np.int64)
    n = m.size
    P = np.zeros(n + 1, dtype=np.int64)
    for t in range(n):            # prefix sum written out
        P[t + 1] = P[t] + m[t]
    S = int(P[n])
    I = np.zeros(S, dtype=np.int64)
    for t in range(n):
        v = P[t + 1]
        if P[t] != v:
            I[v - 1] = t
    return S, I
