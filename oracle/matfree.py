"""Oracle: the matrix-free upper tier of Alg. 3.4 (Sec. 3.2 - 3.5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Strictly above the switching level L_HSS no front is formed as a dense
matrix.  A node sigma with children mu, nu (both compressed, Sec. 3.2) holds
its front implicitly:

* the children's Schur complements as HSS matrices whose cluster trees split
  first at [I^sigma n B^kappa ; B^sigma n B^kappa] (Fig. 4), so that
  S_ii^kappa and S_bb^kappa are the two sub-HSS matrices under the root and
  S_ib^kappa, S_bi^kappa are the root's low-rank coupling U_1 B_12 U_2^T;
* the sparse cross blocks A~ of A between the two children (Eq. 3.4).  Every
  entry of A that the front of sigma receives couples a DOF of box mu with
  one of box nu (an entry enters at the lowest common ancestor of its two
  DOFs' leaves), so A~ has no entries inside a child's own blocks.

The interior block A_ii = [[S_ii^mu, A~^(mu,nu)], [A~^(nu,mu), S_ii^nu]]
(Eq. 3.6) is inverted by the block elimination of Alg. 3.3: ULV factorization
of S_ii^mu, the Schur complement S~ = S_ii^nu - A~^(nu,mu) (S_ii^mu)^{-1}
A~^(mu,nu) compressed by Alg. A.1 from its products and entries (cluster tree
of S_ii^nu), and its ULV factorization.  R = -A_ii^{-1} A_ib (Eq. 3.7) is
found in low-rank form by randomized range finding on products with R
(Sec. 3.4), and S = A_bb + A_bi R (Eq. 3.5) is compressed by Alg. A.1 from
products x -> S x and entries S(i, j) (Sec. 3.5), with the parent-conforming
cluster tree of Fig. 4.

Readings (where the paper is silent or inconsistent):

* Alg. 3.3 subtracts A^(mu,nu) X_1 from X_2; by Alg. 3.2 (X_2 <- X_2 -
  B_21 X_1) the block is the one with rows in nu and columns in mu,
  A~^(nu,mu), which is what is used.  Its last step uses A~^(mu,nu) = B_12
  as Alg. 3.2 does.
* A is symmetric (real or complex), so the rows R(J, :) needed by the row ID
  are -(A_ii^{-1} E_J)^T A_ib = -(A_bi A_ii^{-1} E_J)^T: one block solve with
  the unit columns E_J and a product with A_bi.  L = R^T as on the other
  compressed levels.
* Philox streams: S of node s uses stream 2 s, R stream 2 s + 1 (as in the
  dense-then-compress tier), S~ stream 3 nnodes + s.
* Nodes on levels >= L_HSS, and leaves on any level, are formed and
  eliminated densely (the lower branch of Alg. 3.4); a node on level L_HSS
  also compresses its dense S (the switching-level branch of Alg. 3.4).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .frontal import assemble_front, factor_node
from .hss import HSS, Cluster, LowRank, cluster_tree, hss_compress, hss_matvec, lowrank_rows, ulv_factor, ulv_solve

# ----------------------------------------------------------------------------
# access to an HSS matrix without reconstructing it
# ----------------------------------------------------------------------------


def expanded_bases(H: HSS) -> dict:
    """Node -> the full row basis of its cluster (|I_i| x k_i): the leaf's U,
    or blockdiag(children's full bases) times the node's transfer matrix
    (the nested bases of Eq. 2.4)."""
    T = H.tree
    out = {}
    for i in sorted(range(len(T)), key=lambda i: -T[i].level):
        if i == 0:
            continue
        c = T[i]
        if not c.children:
            out[i] = H.U[i]
        else:
            a, b = c.children
            ka = H.U[a].shape[1]
            out[i] = np.vstack([out[a] @ H.U[i][:ka], out[b] @ H.U[i][ka:]])
    return out


def _leaves_and_parents(H: HSS):
    T = H.tree
    leaf = np.empty(H.n, dtype=np.int64)
    for i, c in enumerate(T):
        if not c.children:
            leaf[c.lo:c.hi] = i
    return leaf, [c.parent for c in T]


def hss_entries(H: HSS, I, J, Ubig: dict | None = None) -> np.ndarray:
    """The block A_HSS(I, J) for index arrays I, J, entry by entry from the
    generators (Eq. 2.2 - 2.5): D of the common leaf, otherwise
    U_a(i, :) B_ab U_b(j, :)^T with a, b the children of the two leaves'
    lowest common ancestor that contain i and j."""
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    T = H.tree
    out = np.zeros((I.size, J.size), dtype=H.dtype)
    if I.size == 0 or J.size == 0:
        return out
    if len(T) == 1:
        return np.asarray(H.D[0])[np.ix_(I, J)].astype(H.dtype)
    if Ubig is None:
        Ubig = expanded_bases(H)
    leaf, par = _leaves_and_parents(H)

    def chain(x):
        c = [x]
        while par[c[-1]] >= 0:
            c.append(par[c[-1]])
        return c

    li, lj = leaf[I], leaf[J]
    for a in np.unique(li):
        ra = np.nonzero(li == a)[0]
        ca = chain(a)
        for b in np.unique(lj):
            cb = np.nonzero(lj == b)[0]
            if a == b:
                lo = T[a].lo
                out[np.ix_(ra, cb)] = np.asarray(H.D[a])[np.ix_(I[ra] - lo, J[cb] - lo)]
                continue
            chb = chain(b)
            p = next(x for x in ca if x in chb)
            na = ca[ca.index(p) - 1]
            nb = chb[chb.index(p) - 1]
            Bp = H.B12[p] if na == T[p].children[0] else H.B21[p]
            out[np.ix_(ra, cb)] = (Ubig[na][I[ra] - T[na].lo] @ Bp) @ Ubig[nb][J[cb] - T[nb].lo].T
    return out


def hss_sub(H: HSS, i: int) -> HSS:
    """The HSS matrix of the diagonal block of cluster i: its subtree,
    re-indexed from 0, with the same generators (the root's basis dropped)."""
    T = H.tree
    base, lev0 = T[i].lo, T[i].level
    new = {i: 0}
    nodes = [Cluster(0, T[i].size, 0)]
    q = [i]
    while q:
        old = q.pop(0)
        for ch in T[old].children:
            new[ch] = len(nodes)
            nodes.append(Cluster(T[ch].lo - base, T[ch].hi - base, T[ch].level - lev0, parent=new[old]))
            nodes[new[old]].children.append(new[ch])
            q.append(ch)
    S = HSS(n=T[i].size, tree=nodes, dtype=H.dtype)
    for old, nw in new.items():
        if old in H.D:
            S.D[nw] = H.D[old]
        if old in H.B12:
            S.B12[nw], S.B21[nw] = H.B12[old], H.B21[old]
        if nw != 0 and old in H.U:
            S.U[nw] = H.U[old]
        if old in H.skel:
            S.skel[nw] = np.asarray(H.skel[old]) - base
    return S


def diag_block(H: HSS, lo: int, hi: int):
    """HSS form of the diagonal block [lo, hi) when it is a cluster of H (or
    H is one dense leaf); None for an empty range."""
    if hi <= lo:
        return None
    if len(H.tree) == 1:
        return HSS(n=hi - lo, tree=[Cluster(0, hi - lo, 0)], D={0: np.asarray(H.D[0])[lo:hi, lo:hi]}, dtype=H.dtype)
    if (lo, hi) == (0, H.n):
        return H
    for i, c in enumerate(H.tree):
        if (c.lo, c.hi) == (lo, hi):
            return hss_sub(H, i)
    raise ValueError(f"[{lo}, {hi}) is not a cluster of the HSS matrix")


@dataclass
class Coupling:
    """The off-diagonal blocks A(I_1, I_2) = U_1 B_12 U_2^T and A(I_2, I_1) =
    U_2 B_21 U_1^T of the root split [0, top) | [top, n) of an HSS matrix,
    or the dense blocks when the matrix is one leaf."""
    top: int
    n: int
    U1: np.ndarray = None
    U2: np.ndarray = None
    B12: np.ndarray = None
    B21: np.ndarray = None
    D12: np.ndarray = None
    D21: np.ndarray = None

    def mm12(self, X):         # A(I_1, I_2) X
        return self.D12 @ X if self.D12 is not None else self.U1 @ (self.B12 @ (self.U2.T @ X))

    def mm21(self, X):         # A(I_2, I_1) X
        return self.D21 @ X if self.D21 is not None else self.U2 @ (self.B21 @ (self.U1.T @ X))


def root_coupling(H: HSS, top: int) -> Coupling:
    T = H.tree
    cp = Coupling(top=top, n=H.n)
    if top <= 0 or top >= H.n:
        return cp
    if len(T) == 1:
        D = np.asarray(H.D[0])
        cp.D12, cp.D21 = D[:top, top:], D[top:, :top]
        return cp
    a, b = T[0].children
    assert (T[a].lo, T[a].hi, T[b].lo, T[b].hi) == (0, top, top, H.n), "root is not split at the given position"
    Ub = expanded_bases(H)
    cp.U1, cp.U2, cp.B12, cp.B21 = Ub[a], Ub[b], H.B12[0], H.B21[0]
    return cp


# ----------------------------------------------------------------------------
# the implicit front of a node above the switching level
# ----------------------------------------------------------------------------

@dataclass
class ChildPart:
    """Child kappa's compressed Schur complement as it enters the parent's
    front: the first ni rows (I^sigma n B^kappa) sit at the parent's
    interior positions pi (contiguous), the rest at parent B positions pb."""
    H: HSS
    ni: int
    pi: np.ndarray
    pb: np.ndarray
    Sii: object = None            # HSS of S_ii^kappa (or None when ni = 0)
    Sbb: object = None            # HSS of S_bb^kappa (or None)
    cp: Coupling = None
    Ubig: dict = None


class BlockInverse:
    """A_ii^{-1} by Alg. 3.3 for A_ii = [[S_ii^mu, A12], [A21, S_ii^nu]] with
    sparse A12 = A~^(mu,nu), A21 = A~^(nu,mu)."""

    def __init__(self, n1, n2, S1, S2, A12, A21, eps, beta, k0, r, seed, stream, rank_cap):
        self.n1, self.n2 = n1, n2
        self.A12, self.A21 = A12, A21
        self.U1 = ulv_factor(S1) if n1 else None
        self.St = None
        if n2:
            if n1:
                op = SchurOp(S2, self.U1, A12, A21)
                self.St = hss_compress(op, cluster_tree(n2, None, beta), eps, k0, r, seed, stream=stream,
                                       rank_cap=rank_cap)
            else:
                self.St = S2
            self.U2 = ulv_factor(self.St)
        self.kmax = self.St.kmax() if self.St is not None else 0

    def solve(self, X):
        X = np.array(X, copy=True)
        X1, X2 = X[:self.n1], X[self.n1:]
        if self.n1:
            X1 = ulv_solve(self.U1, X1)                       # X_1 <- (S_ii^mu)^{-1} X_1
        if self.n2:
            if self.n1:
                X2 = X2 - self.A21 @ X1                       # X_2 <- X_2 - A~^(nu,mu) X_1
            X2 = ulv_solve(self.U2, X2)                       # X_2 <- S~^{-1} X_2
            if self.n1:
                X1 = X1 - ulv_solve(self.U1, self.A12 @ X2)   # X_1 <- X_1 - (S_ii^mu)^{-1} A~^(mu,nu) X_2
        return np.concatenate([X1, X2], axis=0)

    def storage(self) -> int:
        s = self.A12.nnz + self.A21.nnz if self.n1 and self.n2 else 0
        return s + _ulv_size(self.U1) + (_ulv_size(self.U2) if self.n2 else 0)


def _ulv_size(U) -> int:
    if U is None:
        return 0
    tot = U.Dinv.size if U.Dinv is not None else 0
    for d in (U.Mup, U.W, U.Mm, U.E):
        tot += sum(v.size for v in d.values())
    return tot


class SchurOp:
    """S~ = S_ii^nu - A21 (S_ii^mu)^{-1} A12 through products and entries."""

    def __init__(self, S2: HSS, U1, A12, A21):
        self.S2, self.U1, self.A12, self.A21 = S2, U1, A12, A21
        self.shape = (S2.n, S2.n)
        self.dtype = np.result_type(S2.dtype, A12.dtype, np.float64)
        self.Ubig = expanded_bases(S2) if len(S2.tree) > 1 else None

    def matmat(self, X):
        return hss_matvec(self.S2, X) - self.A21 @ ulv_solve(self.U1, self.A12 @ X)

    def entries(self, I, J):
        W = ulv_solve(self.U1, self.A12[:, J].toarray())
        return hss_entries(self.S2, I, J, self.Ubig) - self.A21[I] @ W


class ImplicitFront:
    """The front of node s (Eq. 3.4) from its children's HSS Schur
    complements and the sparse entries of A it receives; products with its
    blocks A_ib, A_bi, A_bb and entries of A_bb."""

    def __init__(self, tree, s, A, hss: dict):
        self.m_i, self.m_b = int(tree.node_info[s, 5]), int(tree.node_info[s, 7])
        m = self.m_i + self.m_b
        lo, hi = tree.e_off[s], tree.e_off[s + 1]
        self.Sp = sp.csr_matrix((A.data[tree.e_idx[lo:hi]], (tree.e_row[lo:hi], tree.e_col[lo:hi])),
                                shape=(m, m), dtype=A.dtype)
        self.dtype = np.result_type(A.dtype, np.float64)
        self.parts = []
        for k in tree.children(s):
            if tree.node_info[k, 7] == 0:
                continue
            e = tree.emap_of(k).astype(np.int64)
            ni = int(np.sum(e < self.m_i))
            H = hss[k]
            assert np.all(e[:ni] < self.m_i) and np.all(e[ni:] >= self.m_i)
            part = ChildPart(H=H, ni=ni, pi=e[:ni], pb=e[ni:] - self.m_i)
            part.Sii = diag_block(H, 0, ni)
            part.Sbb = diag_block(H, ni, H.n)
            part.cp = root_coupling(H, ni)
            part.Ubig = expanded_bases(H) if len(H.tree) > 1 else None
            self.parts.append(part)
        # the interior positions of the children follow each other: [I n B^mu ; I n B^nu]
        off = 0
        for part in self.parts:
            assert np.array_equal(part.pi, np.arange(off, off + part.ni))
            off += part.ni
        assert off == self.m_i
        Spii = self.Sp[:self.m_i, :self.m_i].tocsr()
        n1 = self.parts[0].ni if self.parts else 0
        # no entry of A lies inside one child's interior block (only cross couplings, Eq. 3.4)
        assert Spii[:n1, :n1].nnz == 0 and Spii[n1:, n1:].nnz == 0
        self.n1 = n1
        self.A12 = Spii[:n1, n1:].tocsr()
        self.A21 = Spii[n1:, :n1].tocsr()
        self.Sib = self.Sp[:self.m_i, self.m_i:].tocsr()
        self.Sbi = self.Sp[self.m_i:, :self.m_i].tocsr()
        self.Sbb = self.Sp[self.m_i:, self.m_i:].tocsr()
        # parent B position -> (child part, child-local index)
        self.bpart = np.full(self.m_b, -1, dtype=np.int64)
        self.bloc = np.zeros(self.m_b, dtype=np.int64)
        for q, part in enumerate(self.parts):
            self.bpart[part.pb] = q
            self.bloc[part.pb] = part.ni + np.arange(part.pb.size)

    def _out(self, rows, X):
        return np.zeros((rows,) + X.shape[1:], dtype=np.result_type(self.dtype, X.dtype))

    def aib(self, X):            # A_ib X,  X: m_b x k
        Y = self._out(self.m_i, X) + self.Sib @ X
        for part in self.parts:
            if part.ni and part.pb.size:
                Y[part.pi] += part.cp.mm12(X[part.pb])
        return Y

    def abi(self, X):            # A_bi X,  X: m_i x k
        Y = self._out(self.m_b, X) + self.Sbi @ X
        for part in self.parts:
            if part.ni and part.pb.size:
                Y[part.pb] += part.cp.mm21(X[part.pi])
        return Y

    def abb(self, X):            # A_bb X,  X: m_b x k
        Y = self._out(self.m_b, X) + self.Sbb @ X
        for part in self.parts:
            if part.pb.size:
                Y[part.pb] += hss_matvec(part.Sbb, X[part.pb])
        return Y

    def abb_entries(self, I, J):
        I = np.asarray(I, dtype=np.int64)
        J = np.asarray(J, dtype=np.int64)
        out = self.Sbb[I][:, J].toarray().astype(self.dtype)
        for q, part in enumerate(self.parts):
            ri = np.nonzero(self.bpart[I] == q)[0]
            cj = np.nonzero(self.bpart[J] == q)[0]
            if ri.size and cj.size:
                out[np.ix_(ri, cj)] += hss_entries(part.H, self.bloc[I[ri]], self.bloc[J[cj]], part.Ubig)
        return out


class ROp:
    """R = -A_ii^{-1} A_ib (Eq. 3.7) through products and rows."""

    def __init__(self, front: ImplicitFront, binv: BlockInverse):
        self.f, self.binv = front, binv
        self.shape = (front.m_i, front.m_b)

    def matmat(self, X):
        return -self.binv.solve(self.f.aib(X))

    def rows(self, J):
        E = np.zeros((self.f.m_i, len(J)), dtype=self.f.dtype)
        E[np.asarray(J), np.arange(len(J))] = 1.0
        return -self.f.abi(self.binv.solve(E)).T          # A symmetric: R(J, :) = -(A_bi A_ii^{-1} E_J)^T


class SOp:
    """S = A_bb + A_bi R (Eq. 3.5) with R in low-rank form, through products
    and entries (Sec. 3.5)."""

    def __init__(self, front: ImplicitFront, R: LowRank | None):
        self.f, self.R = front, R
        self.shape = (front.m_b, front.m_b)
        self.dtype = front.dtype
        self.Z = front.abi(R.X) if R is not None else None        # A_bi X_R, m_b x k_R

    def matmat(self, X):
        Y = self.f.abb(X)
        if self.R is not None:
            Y = Y + self.f.abi(self.R.matmat(X))
        return Y

    def entries(self, I, J):
        out = self.f.abb_entries(I, J)
        if self.R is not None:
            out = out + self.Z[np.asarray(I)] @ self.R.RJ[:, np.asarray(J)]
        return out


# ----------------------------------------------------------------------------
# factorization and application
# ----------------------------------------------------------------------------

@dataclass
class MatfreeFactor:
    tree: object
    dtype: object
    L_hss: int
    lu: dict = field(default_factory=dict)      # dense nodes: LU of A_ii
    R: dict = field(default_factory=dict)       # dense ndarray or LowRank
    L: dict = field(default_factory=dict)       # dense ndarray, or None (L = R^T)
    binv: dict = field(default_factory=dict)    # nodes above the switching level: Alg. 3.3
    hss: dict = field(default_factory=dict)     # node -> HSS of S
    kmax: int = 0

    def storage_by_level(self) -> dict:
        """Stored entries per tree level (dense LU, R, L, Alg. 3.3 data; the
        compressed S of a level are counted on that level)."""
        out = {}
        lev = self.tree.node_info[:, 0]
        for s in range(self.tree.nnodes):
            n = 0
            if s in self.lu:
                n += self.lu[s][0].size
            if s in self.binv:
                n += self.binv[s].storage()
            R = self.R.get(s)
            if R is not None:
                n += R.size() if isinstance(R, LowRank) else R.size
            if self.L.get(s) is not None:
                n += self.L[s].size
            if s in self.hss:
                n += self.hss[s].storage()
            out[int(lev[s])] = out.get(int(lev[s]), 0) + n
        return out


def factor_matfree(tree, A, hss_levels: int = 4, eps: float = 1e-6, beta: int = 64, k0: int = 32, r: int = 16,
                   seed: int = 0, rank_cap: int = 512) -> MatfreeFactor:
    """Alg. 3.4: dense fronts on levels >= L_HSS = depth - hss_levels (a node
    on L_HSS compresses its dense S), implicit fronts (Alg. 3.3, low-rank R,
    S by Alg. A.1 from products and entries) on the levels above."""
    Lh = tree.depth - hss_levels
    fac = MatfreeFactor(tree=tree, dtype=A.dtype, L_hss=Lh)
    S_dense = {}
    nn = tree.nnodes
    for s in range(nn):
        lev = int(tree.node_info[s, 0])
        m_i, m_b = int(tree.node_info[s, 5]), int(tree.node_info[s, 7])
        kids = tree.children(s)
        top = None
        if m_b:
            p = int(tree.node_info[s, 1])
            top = int(np.sum(tree.emap_of(s) < tree.node_info[p, 5])) if p >= 0 else None
        if lev >= Lh or not kids:
            F = assemble_front(tree, s, A, S_dense)
            lu, L, R, S = factor_node(F, m_i)
            fac.lu[s] = lu
            if lev <= Lh and m_b:
                H = hss_compress(S, cluster_tree(m_b, top, beta), eps, k0, r, seed, stream=2 * s, rank_cap=rank_cap)
                fac.hss[s] = H
                fac.kmax = max(fac.kmax, H.kmax())
            else:
                S_dense[s] = S
            if lev < Lh and m_b and m_i:
                R = lowrank_rows(R, eps, k0, r, seed, stream=2 * s + 1, rank_cap=rank_cap)
                fac.kmax = max(fac.kmax, R.X.shape[1])
                L = None
            fac.R[s], fac.L[s] = R, L
        else:
            front = ImplicitFront(tree, s, A, fac.hss)
            n1 = front.n1
            p1 = front.parts[0] if front.parts else None
            p2 = front.parts[1] if len(front.parts) > 1 else None
            binv = BlockInverse(n1, m_i - n1, p1.Sii if p1 else None, p2.Sii if p2 else None,
                                front.A12, front.A21, eps, beta, k0, r, seed, 3 * nn + s, rank_cap)
            fac.binv[s] = binv
            fac.kmax = max(fac.kmax, binv.kmax)
            R = None
            if m_b and m_i:
                R = lowrank_rows(ROp(front, binv), eps, k0, r, seed, stream=2 * s + 1, rank_cap=rank_cap)
                fac.kmax = max(fac.kmax, R.X.shape[1])
            fac.R[s], fac.L[s] = R, None
            if m_b:
                H = hss_compress(SOp(front, R), cluster_tree(m_b, top, beta), eps, k0, r, seed, stream=2 * s,
                                 rank_cap=rank_cap)
                fac.hss[s] = H
                fac.kmax = max(fac.kmax, H.kmax())
        for k in kids:
            S_dense.pop(k, None)
    return fac


def apply_matfree(fac: MatfreeFactor, b: np.ndarray) -> np.ndarray:
    """Algorithm 3.1 with the factors of factor_matfree: L = R^T for the
    low-rank R, A_ii^{-1} by Alg. 3.3 above the switching level."""
    tree = fac.tree
    y = np.array(b, dtype=np.result_type(b.dtype, fac.dtype), copy=True)[tree.perm]
    for s in range(tree.nnodes):
        R = fac.R.get(s)
        if tree.node_info[s, 7] and R is not None and tree.node_info[s, 5]:
            I, B = tree.I(s), tree.B(s)
            y[B] += R.rmatmat(y[I]) if fac.L[s] is None else fac.L[s] @ y[I]
    for s in range(tree.nnodes):
        I = tree.I(s)
        if I.size:
            y[I] = fac.binv[s].solve(y[I]) if s in fac.binv else sla.lu_solve(fac.lu[s], y[I], check_finite=False)
    for s in range(tree.nnodes - 1, -1, -1):
        R = fac.R.get(s)
        if tree.node_info[s, 7] and R is not None and tree.node_info[s, 5]:
            I, B = tree.I(s), tree.B(s)
            y[I] += R.matmat(y[B]) if isinstance(R, LowRank) else R @ y[B]
    x = np.empty_like(y)
    x[tree.perm] = y
    return x
