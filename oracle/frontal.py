"""Oracle: exact (dense) LDR factorization by fronts and its application.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``assemble_front`` builds A^(sigma): A(front, front) for a leaf (Eq. 3.2),
  the children's Schur complements plus the sparse cross blocks A~ for an
  inner node (Eq. 3.4).
* ``factor_dense`` eliminates every node bottom-up in post-order (Sec. 3.1):
  LU of A_ii with partial pivoting (LAPACK getrf: first index of the largest
  |Re| + |Im|), then L = -A_bi A_ii^{-1} (Eq. 3.3a), R = -A_ii^{-1} A_ib
  (Eq. 3.3b) and S = A_bb - A_bi A_ii^{-1} A_ib (Eq. 3.5).  The root only
  factors A_ii.  With no compression this is a sparse direct solver
  (start of Sec. 3.2), so P = A.
* ``apply_inverse`` is Algorithm 3.1: b(B) += L b(I) bottom-up, b(I) <-
  A_ii^{-1} b(I) at every node, b(I) += R b(B) top-down.

Vectors are in the original numbering at the interface; internally the tree's
permutation (new -> old) is used.  Everything is float64 / complex128.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .tree import Tree


def assemble_front(tree: Tree, s: int, A, S_children: dict) -> np.ndarray:
    """Dense front A^(s) in the order [I^s; B^s] (Eq. 3.2 / Eq. 3.4)."""
    m = int(tree.node_info[s, 5] + tree.node_info[s, 7])
    F = np.zeros((m, m), dtype=A.dtype)
    for k in tree.children(s):
        pos = tree.emap_of(k)
        F[np.ix_(pos, pos)] += S_children[k]
    lo, hi = tree.e_off[s], tree.e_off[s + 1]
    np.add.at(F, (tree.e_row[lo:hi], tree.e_col[lo:hi]), A.data[tree.e_idx[lo:hi]])
    return F


@dataclass
class DenseFactor:
    tree: Tree
    dtype: np.dtype
    lu: list = field(default_factory=list)     # (lu, piv) of A_ii per node
    L: list = field(default_factory=list)      # L^sigma, m_b x m_i (Eq. 3.3a)
    R: list = field(default_factory=list)      # R^sigma, m_i x m_b (Eq. 3.3b)
    S: list = field(default_factory=list)      # S^sigma, m_b x m_b (Eq. 3.5), kept for tests
    Aii: list = field(default_factory=list)    # A_ii^sigma, kept for tests


def factor_node(F: np.ndarray, m_i: int):
    """Eliminate the first m_i unknowns of the front F: (lu, L, R, S)."""
    Aii = F[:m_i, :m_i]
    Aib = F[:m_i, m_i:]
    Abi = F[m_i:, :m_i]
    Abb = F[m_i:, m_i:]
    lu = sla.lu_factor(Aii, check_finite=False) if m_i else (np.zeros((0, 0), F.dtype), np.zeros(0, np.int32))
    if m_i and F.shape[0] > m_i:
        R = -sla.lu_solve(lu, Aib, check_finite=False)                       # Eq. 3.3b
        L = -sla.lu_solve(lu, Abi.T, trans=1, check_finite=False).T          # Eq. 3.3a
        S = Abb + Abi @ R                                                    # Eq. 3.5
    else:
        mb = F.shape[0] - m_i
        R = np.zeros((m_i, mb), F.dtype)
        L = np.zeros((mb, m_i), F.dtype)
        S = Abb.copy()
    return lu, L, R, S


def factor_dense(tree: Tree, A) -> DenseFactor:
    """Exact factorization A = L D R by fronts, bottom-up in post-order."""
    fac = DenseFactor(tree=tree, dtype=A.dtype)
    S_keep = {}
    for s in range(tree.nnodes):                       # post-order = bottom-up
        F = assemble_front(tree, s, A, S_keep)
        m_i = int(tree.node_info[s, 5])
        lu, L, R, S = factor_node(F, m_i)
        for k in tree.children(s):
            S_keep.pop(k, None)
        S_keep[s] = S
        fac.lu.append(lu)
        fac.L.append(L)
        fac.R.append(R)
        fac.S.append(S)
        fac.Aii.append(F[:m_i, :m_i].copy())
    return fac


def apply_inverse(fac, b: np.ndarray, solve_ii=None) -> np.ndarray:
    """Algorithm 3.1 in the original numbering.  ``b`` may be (n,) or (n, k).

    ``solve_ii(s, y)`` applies (A_ii^s)^{-1}; by default the stored LU is used.
    """
    tree = fac.tree
    y = np.array(b, dtype=np.result_type(b.dtype, fac.dtype), copy=True)[tree.perm]
    for s in range(tree.nnodes):                                   # bottom-up
        if tree.node_info[s, 7]:
            I, B = tree.I(s), tree.B(s)
            y[B] += fac.L[s] @ y[I]
    for s in range(tree.nnodes):                                   # all nodes decoupled
        I = tree.I(s)
        if I.size:
            y[I] = solve_ii(s, y[I]) if solve_ii else sla.lu_solve(fac.lu[s], y[I], check_finite=False)
    for s in range(tree.nnodes - 1, -1, -1):                       # top-down
        if tree.node_info[s, 7]:
            I, B = tree.I(s), tree.B(s)
            y[I] += fac.R[s] @ y[B]
    x = np.empty_like(y)
    x[tree.perm] = y
    return x
