"""Oracle: HSS matrices, randomized adaptive compression (Alg. A.1) and the
compressed factorization of Alg. 3.4 in its dense-then-compress variant
(every Schur complement eliminated densely, then compressed).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Cluster trees (Def. 2.1): contiguous index ranges; the top split is given
  (the parent-conforming split of Fig. 4), below it ranges are halved
  (floor(size / 2) first) until they hold at most beta indices (Eq. 2.1).
* HSS representation (Eq. 2.2 - 2.6) for symmetric (A = A^T, also complex
  symmetric) matrices: nested row bases U_i (leaf: |I_i| x k_i; inner node:
  (k_c1 + k_c2) x k_i), column bases V = U (symmetry), coupling blocks
  B_i = [[0, B12], [B21, 0]] at inner nodes, dense D_i at leaves.
* Alg. A.1: samples S = A Omega with n x (k + r) Gaussian Omega; levels
  processed bottom-up; a row interpolative decomposition (Eq. A.1) of every
  local sample block S_loc ~ U_i S_loc(J_i, :) chooses the skeleton rows; the
  estimator of Eq. 2.7 on r fresh samples decides whether to stop or to
  increase k by r and reuse all samples.  Where the paper is silent (an
  estimate that never reaches eps) the rank stops growing once a round of r
  more samples fails to halve an estimated error that is already within
  STAGNATION_FLOOR (10^3 unit roundoffs) of the block's norm: there the
  estimate sits at the floor set by the arithmetic; above it a slowly
  decaying spectrum keeps sampling.  At most MAX_SAMPLES samples per block:
  no round starts that would exceed it.
* Gaussian samples come from Philox4x32-10 (Salmon et al., SC'11) with the
  Box-Muller transform, keyed by (seed, stream), so any implementation of
  the same definition draws the same matrices.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

STAGNATION_FLOOR = 1e3 * np.finfo(np.float64).eps / 2    # relative, float64 arithmetic
MAX_SAMPLES = 256


def _matmat(A, X):
    """A X for a dense array, or an operator's own product (matrix-free form)."""
    return A @ X if isinstance(A, np.ndarray) else A.matmat(X)


def _entries(A, I, J):
    """The block A(I, J) of a dense array, or entries read from an operator."""
    return A[np.ix_(I, J)] if isinstance(A, np.ndarray) else A.entries(I, J)


def _stop(err, ref, eps, prev_err, nsamp, nmax, r):
    """The adaptive loop's stopping test (shared by both compressions)."""
    return (err <= eps * ref or nsamp >= nmax or nsamp + r > MAX_SAMPLES
            or (err > 0.5 * prev_err and err <= STAGNATION_FLOOR * ref))

# ----------------------------------------------------------------------------
# Philox4x32-10 and Gaussian matrices
# ----------------------------------------------------------------------------

_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32 with 10 rounds on counters ctr [N, 4] (uint32) and key (k0, k1)."""
    c = ctr.astype(np.uint32).copy()
    k0 = np.uint32(key[0])
    k1 = np.uint32(key[1])
    M = np.uint64(0xFFFFFFFF)
    for rnd in range(10):
        p0 = c[:, 0].astype(np.uint64) * _PHILOX_M0
        p1 = c[:, 2].astype(np.uint64) * _PHILOX_M1
        hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & M).astype(np.uint32)
        hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & M).astype(np.uint32)
        c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
        if rnd < 9:
            k0 = np.uint32((int(k0) + int(_PHILOX_W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(_PHILOX_W1)) & 0xFFFFFFFF)
    return c


def gaussian(rows: int, cols: int, seed: int, stream: int) -> np.ndarray:
    """rows x cols standard normal matrix, column-major element e = i + j*rows.

    Counter (e // 4, stream_lo, stream_hi, 0), key (seed_lo, seed_hi); the four
    32-bit outputs become uniforms u = (x + 0.5) / 2^32 and two Box-Muller pairs
    (u0, u1) -> sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), likewise (u2, u3).
    """
    seed, stream = int(seed), int(stream)
    n = rows * cols
    nb = (n + 3) // 4
    ctr = np.zeros((nb, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(nb, dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] = np.uint32(stream & 0xFFFFFFFF)
    ctr[:, 2] = np.uint32((stream >> 32) & 0xFFFFFFFF)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    x = philox4x32_10(ctr, key).astype(np.float64)
    u = (x + 0.5) / 4294967296.0
    r0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.stack([r0 * np.cos(2 * np.pi * u[:, 1]), r0 * np.sin(2 * np.pi * u[:, 1]),
                  r1 * np.cos(2 * np.pi * u[:, 3]), r1 * np.sin(2 * np.pi * u[:, 3])], axis=1).ravel()[:n]
    return z.reshape(cols, rows).T.copy()


# ----------------------------------------------------------------------------
# cluster trees
# ----------------------------------------------------------------------------

@dataclass
class Cluster:
    lo: int
    hi: int
    level: int
    parent: int = -1
    children: list = field(default_factory=list)

    @property
    def size(self) -> int:
        return self.hi - self.lo


def cluster_tree(n: int, top_split: int | None, beta: int) -> list:
    """Nodes in breadth-first order (root first).  The root [0, n) is split at
    ``top_split`` when 0 < top_split < n (Fig. 4), every other range at
    floor(size / 2), until a range holds at most beta indices."""
    nodes = [Cluster(0, n, 0)]
    q = [0]
    while q:
        i = q.pop(0)
        c = nodes[i]
        if c.size <= beta:
            continue
        if i == 0 and top_split is not None and 0 < top_split < n:
            mid = top_split
        else:
            mid = c.lo + c.size // 2
        for lo, hi in ((c.lo, mid), (mid, c.hi)):
            nodes.append(Cluster(lo, hi, c.level + 1, parent=i))
            c.children.append(len(nodes) - 1)
            q.append(len(nodes) - 1)
    return nodes


# ----------------------------------------------------------------------------
# interpolative decomposition (Eq. A.1)
# ----------------------------------------------------------------------------

def row_id(Sloc: np.ndarray, eps: float, max_rank: int):
    """Row ID S_loc ~ X S_loc(J, :) from a column-pivoted Householder QR
    (Businger-Golub, LAPACK geqp3) of S_loc^T.  Rank = number of leading
    |R_jj| > eps |R_11|, at most max_rank.  X(J, :) = I exactly."""
    m = Sloc.shape[0]
    if m == 0:
        return np.zeros(0, dtype=np.int64), np.zeros((0, 0), dtype=Sloc.dtype)
    Q, R, piv = sla.qr(Sloc.T, mode="economic", pivoting=True)
    d = np.abs(np.diag(R))
    if d.size == 0 or d[0] == 0:
        k = 0
    else:
        k = int(np.sum(d > eps * d[0]))
    k = max(0, min(k, max_rank, m))
    J = piv[:k]
    X = np.zeros((m, k), dtype=np.result_type(Sloc.dtype, np.float64))
    X[J, :] = np.eye(k)
    if k < m and k > 0:
        T = sla.solve_triangular(R[:k, :k], R[:k, k:], lower=False)      # R11^{-1} R12
        X[piv[k:], :] = T.T
    return np.asarray(J, dtype=np.int64), X


# ----------------------------------------------------------------------------
# HSS matrices
# ----------------------------------------------------------------------------

@dataclass
class HSS:
    n: int
    tree: list
    U: dict = field(default_factory=dict)       # node -> basis
    D: dict = field(default_factory=dict)       # leaf -> dense block
    B12: dict = field(default_factory=dict)     # inner node -> A(skel c1, skel c2)
    B21: dict = field(default_factory=dict)     # inner node -> A(skel c2, skel c1)
    skel: dict = field(default_factory=dict)    # node -> global skeleton indices
    dtype: object = np.float64
    rounds: int = 0
    samples: int = 0

    def ranks(self):
        return {i: self.U[i].shape[1] for i in self.U}

    def kmax(self) -> int:
        return max([u.shape[1] for u in self.U.values()] + [0])

    def storage(self) -> int:
        """Number of stored entries (D, U, B)."""
        return (sum(d.size for d in self.D.values()) + sum(u.size for u in self.U.values())
                + sum(b.size for b in self.B12.values()) + sum(b.size for b in self.B21.values()))


def hss_matvec(H: HSS, x: np.ndarray) -> np.ndarray:
    """y = A_HSS x via the telescoping form (Eq. 2.5 / 2.6): up-sweep of U^T,
    coupling by B, down-sweep of U, plus the leaf blocks D."""
    T = H.tree
    x2 = x.reshape(H.n, -1)
    xh = {}
    order = sorted(range(len(T)), key=lambda i: -T[i].level)      # deepest first
    for i in order:
        c = T[i]
        if i == 0:
            continue
        if not c.children:
            xh[i] = H.U[i].T @ x2[c.lo:c.hi]
        else:
            xh[i] = H.U[i].T @ np.vstack([xh[c.children[0]], xh[c.children[1]]])
    y = np.zeros((H.n, x2.shape[1]), dtype=np.result_type(H.dtype, x2.dtype))
    yh = {}
    for i in sorted(range(len(T)), key=lambda i: T[i].level):      # root first
        c = T[i]
        if not c.children:
            y[c.lo:c.hi] = H.D[i] @ x2[c.lo:c.hi]
            if i != 0:
                y[c.lo:c.hi] += H.U[i] @ yh[i]
            continue
        c1, c2 = c.children
        a = H.B12[i] @ xh[c2]
        b = H.B21[i] @ xh[c1]
        if i != 0:
            t = H.U[i] @ yh[i]
            k1 = H.U[c1].shape[1]
            a = a + t[:k1]
            b = b + t[k1:]
        yh[c1], yh[c2] = a, b
    return y.reshape(x.shape) if x.ndim == 1 else y


def hss_dense(H: HSS) -> np.ndarray:
    return hss_matvec(H, np.eye(H.n, dtype=H.dtype))


def hss_compress(A: np.ndarray, tree: list, eps: float, k0: int = 32, r: int = 16, seed: int = 0,
                 stream: int = 0, rank_cap: int = 512, oversample_min: int = 10) -> HSS:
    """Algorithm A.1 for a symmetric (or complex symmetric) matrix A.

    A is a dense array, or an operator with ``shape``, ``dtype``,
    ``matmat(X)`` and ``entries(I, J)``: the two accesses Alg. A.1 makes
    (products with Gaussian blocks, individual entries), as Sec. 3.5 uses it
    without forming the matrix.  The
    estimator (Eq. 2.7, relative reading): ||S~ - A_HSS Omega~||_F <= eps ||S~||_F
    with r fresh samples; on failure k <- k + r and Omega, S are extended.
    """
    n = A.shape[0]
    dtype = np.result_type(A.dtype, np.float64)
    k = k0
    Om = gaussian(n, k + r, seed, stream * 64 + 0)
    S = _matmat(A, Om)
    rnd = 0
    prev_err = np.inf
    while True:
        H = HSS(n=n, tree=tree, dtype=dtype)
        Hd = {}                                    # node -> (Omega_i, S_i)
        nsamp = Om.shape[1]
        maxr = min(rank_cap, max(1, nsamp - oversample_min))
        levels = max(c.level for c in tree)
        if len(tree) == 1:
            H.D[0] = A.copy() if isinstance(A, np.ndarray) else A.entries(np.arange(n), np.arange(n))
        for l in range(levels, 0, -1):
            for i, c in enumerate(tree):
                if c.level != l:
                    continue
                if not c.children:
                    Iloc = np.arange(c.lo, c.hi)
                    Oloc = Om[c.lo:c.hi]
                    Dii = _entries(A, Iloc, Iloc)
                    Sloc = S[c.lo:c.hi] - Dii @ Oloc
                    H.D[i] = Dii
                else:
                    c1, c2 = c.children
                    I1, I2 = H.skel[c1], H.skel[c2]
                    O1, S1 = Hd[c1]
                    O2, S2 = Hd[c2]
                    A12 = _entries(A, I1, I2)
                    A21 = _entries(A, I2, I1)
                    Iloc = np.concatenate([I1, I2])
                    Oloc = np.vstack([O1, O2])
                    Sloc = np.vstack([S1 - A12 @ O2, S2 - A21 @ O1])
                    H.B12[i], H.B21[i] = A12, A21
                J, X = row_id(Sloc, eps, maxr)
                H.U[i] = X
                Hd[i] = (X.T @ Oloc, Sloc[J])
                H.skel[i] = Iloc[J]
        if tree[0].children:
            c1, c2 = tree[0].children
            H.B12[0] = _entries(A, H.skel[c1], H.skel[c2])
            H.B21[0] = _entries(A, H.skel[c2], H.skel[c1])
        H.rounds = rnd + 1
        H.samples = nsamp
        Ot = gaussian(n, r, seed, stream * 64 + 1 + rnd)
        St = _matmat(A, Ot)
        err = np.linalg.norm(St - hss_matvec(H, Ot))
        ref = np.linalg.norm(St)
        # stop at eps, when the samples exhaust the matrix or reach MAX_SAMPLES, or when
        # r more samples did not halve an estimate already at the arithmetic's floor
        if len(tree) == 1 or _stop(err, ref, eps, prev_err, nsamp, min(n, rank_cap + oversample_min), r):
            return H
        prev_err = err
        Om = np.hstack([Om, Ot])
        S = np.hstack([S, St])
        k += r
        rnd += 1


# ----------------------------------------------------------------------------
# ULV factorization of an HSS matrix and its solve
# ----------------------------------------------------------------------------

@dataclass
class ULV:
    """ULV factorization of a (complex) symmetric HSS matrix (V = U; the
    coupling A(I_i, I_j) = U_i B_ij U_j^T uses transposes).

    Bottom-up, every node holds a current block D (m x m) with row basis U
    and column basis V (m x k).  A unitary Q with Q^H U = [R; 0] leaves the
    last ne = m - k equations without coupling to the rest of the matrix; a
    unitary W from the LQ factorization of those rows, (Q^H D)_b W = [L 0],
    turns them into ne triangular equations for the first ne transformed
    unknowns, which are eliminated.  The remaining k equations form the
    reduced block D^ = (Q^H D W)_t,2 with row basis U^ = R and column basis
    V^ (V^T W = [P1, V^^T]); siblings merge into the parent's block
    [[D^_a, U^_a B12 V^_b^T], [U^_b B21 V^_a^T, D^_b]] with bases
    blockdiag(U^_a, U^_b) E and blockdiag(V^_a, V^_b) E (E the nested
    transfer matrix); the root block is inverted densely.

    Solve data per node (everything the two sweeps need is a matrix-vector
    product): Mup = [L^-1 Q^H_b; Q^H_t - C L^-1 Q^H_b; P1 L^-1 Q^H_b] maps
    the node's right-hand side to (y1, r^, G): the eliminated unknowns, the
    reduced right-hand side and the eliminated unknowns' coupling to the
    outside (G accumulates E^T [G_a; G_b] from the children); Mm corrects a
    merged right-hand side for the children's G; W maps [y1; x^2] back to
    the node's unknowns on the way down."""
    tree: list
    n: int
    ne: dict = field(default_factory=dict)
    kt: dict = field(default_factory=dict)      # remaining unknowns after elimination
    k: dict = field(default_factory=dict)       # basis width (coupling rank)
    Mup: dict = field(default_factory=dict)
    W: dict = field(default_factory=dict)
    Mm: dict = field(default_factory=dict)      # inner nodes (incl. the root)
    E: dict = field(default_factory=dict)       # inner non-root nodes
    Dinv: object = None                          # root


def _blockdiag(a, b):
    out = np.zeros((a.shape[0] + b.shape[0], a.shape[1] + b.shape[1]), dtype=np.result_type(a.dtype, b.dtype))
    out[:a.shape[0], :a.shape[1]] = a
    out[a.shape[0]:, a.shape[1]:] = b
    return out


def ulv_factor(H: HSS) -> ULV:
    T = H.tree
    F = ULV(tree=T, n=H.n)
    red = {}
    for i in sorted(range(len(T)), key=lambda i: -T[i].level):          # deepest first
        c = T[i]
        if not c.children:
            D = np.asarray(H.D[i], dtype=H.dtype)
            U = V = (H.U[i] if i != 0 else None)
        else:
            a, b = c.children
            Da, Ua, Va = red[a]
            Db, Ub, Vb = red[b]
            A12 = Ua @ H.B12[i]
            A21 = Ub @ H.B21[i]
            D = np.block([[Da, A12 @ Vb.T], [A21 @ Va.T, Db]])
            ka, kb = H.B12[i].shape
            Mm = np.zeros((Da.shape[0] + Db.shape[0], ka + kb), dtype=D.dtype)
            Mm[:Da.shape[0], ka:] = A12
            Mm[Da.shape[0]:, :ka] = A21
            F.Mm[i] = Mm
            if i != 0:
                F.E[i] = H.U[i]
                U = _blockdiag(Ua, Ub) @ H.U[i]
                V = _blockdiag(Va, Vb) @ H.U[i]
        if i == 0:
            F.Dinv = np.linalg.inv(D)
            break
        m, k = D.shape[0], U.shape[1]
        ne = max(0, m - k)
        F.ne[i], F.k[i] = ne, k
        if ne == 0:
            F.kt[i] = m
            F.Mup[i] = np.vstack([np.eye(m, dtype=D.dtype), np.zeros((k, m), dtype=D.dtype)])
            F.W[i] = np.eye(m, dtype=D.dtype)
            red[i] = (D, U, V)
            continue
        Q, R = sla.qr(U, mode="full")                  # Q^H U = [R; 0]
        QH = Q.conj().T
        Dt = QH @ D
        Wq, Rl = sla.qr(Dt[k:, :].conj().T, mode="full")   # (Q^H D)_b = Rl^H Wq^H
        L = Rl[:ne, :ne].conj().T                      # (Q^H D)_b W = [L 0]
        DtW = Dt @ Wq
        C = DtW[:k, :ne]
        VtW = V.T @ Wq
        P1 = VtW[:, :ne]
        Linv = sla.solve_triangular(L, np.eye(ne, dtype=L.dtype), lower=True)
        Y = Linv @ QH[k:]
        F.Mup[i] = np.vstack([Y, QH[:k] - C @ Y, P1 @ Y])
        F.W[i] = Wq
        F.kt[i] = k
        red[i] = (DtW[:k, ne:], R[:k, :], VtW[:, ne:].T)
    return F


def ulv_solve(F: ULV, b: np.ndarray) -> np.ndarray:
    """x = A_HSS^{-1} b with the factors of ulv_factor (b: (n,) or (n, nrhs))."""
    T = F.tree
    b2 = b.reshape(F.n, -1)
    dt = np.result_type(b2.dtype, F.Dinv.dtype)
    if len(T) == 1:
        x = F.Dinv @ b2
        return x.reshape(b.shape) if b.ndim == 1 else x
    y1, rh, G = {}, {}, {}
    order = sorted(range(len(T)), key=lambda i: -T[i].level)
    for i in order:
        c = T[i]
        if c.children:
            a, bb = c.children
            r = np.vstack([rh[a], rh[bb]]) - F.Mm[i] @ np.vstack([G[a], G[bb]])
        else:
            r = b2[c.lo:c.hi].astype(dt)
        if i == 0:
            xt = F.Dinv @ r
            break
        out = F.Mup[i] @ r
        ne, kt, k = F.ne[i], F.kt[i], F.k[i]
        y1[i] = out[:ne]
        rh[i] = out[ne:ne + kt]
        G[i] = out[ne + kt:ne + kt + k]
        if c.children:
            G[i] = G[i] + F.E[i].T @ np.vstack([G[a], G[bb]])
    x = np.zeros((F.n, b2.shape[1]), dtype=dt)
    x2 = {}
    a, bb = T[0].children
    x2[a], x2[bb] = xt[:F.kt[a]], xt[F.kt[a]:]
    for i in sorted(range(len(T)), key=lambda i: T[i].level):
        if i == 0:
            continue
        c = T[i]
        xt_i = F.W[i] @ np.vstack([y1[i], x2[i]])
        if c.children:
            a, bb = c.children
            x2[a], x2[bb] = xt_i[:F.kt[a]], xt_i[F.kt[a]:]
        else:
            x[c.lo:c.hi] = xt_i
    return x.reshape(b.shape) if b.ndim == 1 else x


# ----------------------------------------------------------------------------
# low-rank factors (Sec. 3.4)
# ----------------------------------------------------------------------------

@dataclass
class LowRank:
    X: np.ndarray          # m x k interpolation matrix
    J: np.ndarray          # k skeleton rows
    RJ: np.ndarray         # R(J, :), k x nb

    def matmat(self, v):
        return self.X @ (self.RJ @ v)

    def rmatmat(self, v):
        return self.RJ.T @ (self.X.T @ v)

    def size(self):
        return self.X.size + self.RJ.size


def lowrank_rows(R: np.ndarray, eps: float, k0: int = 32, r: int = 16, seed: int = 0, stream: int = 0,
                 rank_cap: int = 512, oversample_min: int = 10) -> LowRank:
    """R ~ X R(J, :) by randomized range finding (Sec. 3.4): samples Y = R Omega,
    a row ID of Y, and the relative estimator on r fresh samples.  R is a
    dense array, or an operator with ``shape``, ``matmat(X)`` and
    ``rows(J)`` (the rows R(J, :))."""
    m, nb = R.shape
    k = k0
    Om = gaussian(nb, k + r, seed, stream * 64 + 32)
    Y = _matmat(R, Om)
    rnd = 0
    prev_err = np.inf
    while True:
        maxr = min(rank_cap, max(1, Y.shape[1] - oversample_min), m)
        J, X = row_id(Y, eps, maxr)
        lr = LowRank(X=X, J=J, RJ=R[J] if isinstance(R, np.ndarray) else R.rows(J))
        Ot = gaussian(nb, r, seed, stream * 64 + 33 + rnd)
        Yt = _matmat(R, Ot)
        err = np.linalg.norm(Yt - lr.matmat(Ot))
        if _stop(err, np.linalg.norm(Yt), eps, prev_err, Y.shape[1], min(m, nb, rank_cap + oversample_min), r):
            return lr
        prev_err = err
        Om = np.hstack([Om, Ot])
        Y = np.hstack([Y, Yt])
        k += r
        rnd += 1


# ----------------------------------------------------------------------------
# compressed factorization (Alg. 3.4, dense-then-compress tier) and its apply
# ----------------------------------------------------------------------------

@dataclass
class CompressedFactor:
    tree: object
    dtype: object
    L_hss: int                                  # switching level (levels <= L_hss compressed)
    lu: list = field(default_factory=list)
    R: list = field(default_factory=list)       # dense ndarray or LowRank
    L: list = field(default_factory=list)       # dense ndarray, or None (L = R^T by symmetry)
    S: list = field(default_factory=list)       # the Schur complement handed to the parent
    S_exact: list = field(default_factory=list)  # before compression (for tests)
    hss: dict = field(default_factory=dict)     # node -> HSS of S
    ulv: dict = field(default_factory=dict)     # node -> ULV of HSS(A_ii) (strictly above the switching level)
    kmax: int = 0


def ulv_order(tree, s: int) -> np.ndarray:
    """Order of I^s for its HSS form: by the coordinate along the node's cut,
    ties by position in I^s.  I^s = [F(mu); F(nu)] lists each child's side of
    the cut in that coordinate already (Sec. 3.3 numbering); merging the two
    puts the DOFs facing each other across the cut in the same cluster, so
    the off-diagonal blocks of every level couple separated stretches of the
    separator only (low rank), where the split [F(mu); F(nu)] would leave the
    band of couplings across the cut, a full-rank block, at the top."""
    m_i = int(tree.node_info[s, 5])
    axis = int(tree.node_info[s, 12])
    dofs = tree.perm[tree.I(s)]
    along = tree.coords[dofs, 1 - axis] if axis in (0, 1) else np.zeros(m_i, dtype=np.int64)
    return np.lexsort((np.arange(m_i), along)).astype(np.int64)


def factor_compressed(tree, A, hss_levels: int = 4, eps: float = 1e-6, beta: int = 64, k0: int = 32,
                      r: int = 16, seed: int = 0, rank_cap: int = 512, ulv: bool = False,
                      subtree: int | None = None) -> CompressedFactor:
    """Alg. 3.4 with every front formed densely (the matrix-free upper tier of
    Sec. 3.5 is not used): nodes on levels <= L_HSS = depth - hss_levels
    compress their Schur complement by Alg. A.1 with the parent-conforming
    cluster tree of Fig. 4, and the parent assembles the compressed S; nodes
    strictly above the switching level also store R (Eq. 3.3b) in low-rank
    form (Sec. 3.4) and use L = R^T (A symmetric).  R, L and S come from the
    dense elimination of the assembled front.  With ulv=True the assembled
    A_ii of the nodes strictly above the switching level is compressed too
    (Alg. A.1, top split [F(mu); F(nu)], Philox stream 2 nnodes + s) and its
    ULV factorization replaces the dense LU in the diagonal step of the
    apply; otherwise A_ii is factored densely everywhere.  With subtree = s0
    only the nodes of the subtree rooted at s0 are factored (a front depends
    on its own subtree only, and post-order numbers a subtree as the
    contiguous range ending at s0); the entries of the other nodes are None."""
    from .frontal import assemble_front, factor_node
    depth = tree.depth
    Lh = depth - hss_levels
    fac = CompressedFactor(tree=tree, dtype=A.dtype, L_hss=Lh)
    S_keep = {}
    first = 0
    if subtree is not None:
        first = subtree
        while True:                                  # lowest post-order number in the subtree
            ch = tree.children(first)
            if not ch:
                break
            first = min(ch)
        for lst in (fac.lu, fac.R, fac.L, fac.S, fac.S_exact):
            lst.extend([None] * first)
    last = tree.nnodes if subtree is None else subtree + 1
    for s in range(first, last):
        F = assemble_front(tree, s, A, S_keep)
        m_i, m_b = int(tree.node_info[s, 5]), int(tree.node_info[s, 7])
        lu, L, R, S = factor_node(F, m_i)
        lev = int(tree.node_info[s, 0])
        fac.S_exact.append(S)
        if lev <= Lh and m_b > 0:
            p = int(tree.node_info[s, 1])
            top = int(np.sum(tree.emap_of(s) < tree.node_info[p, 5]))       # |F(s)| = |I^parent n B^s|
            H = hss_compress(S, cluster_tree(m_b, top, beta), eps, k0, r, seed, stream=2 * s, rank_cap=rank_cap)
            fac.hss[s] = H
            fac.kmax = max(fac.kmax, H.kmax())
            S = hss_dense(H)
        if ulv and lev < Lh and m_i > 0:
            order = ulv_order(tree, s)
            Hii = hss_compress(F[:m_i, :m_i][np.ix_(order, order)], cluster_tree(m_i, None, beta), eps, k0, r, seed,
                               stream=2 * tree.nnodes + s, rank_cap=rank_cap)
            fac.ulv[s] = (order, ulv_factor(Hii))
            fac.kmax = max(fac.kmax, Hii.kmax())
        if lev < Lh and m_b > 0 and m_i > 0:
            R = lowrank_rows(R, eps, k0, r, seed, stream=2 * s + 1, rank_cap=rank_cap)
            fac.kmax = max(fac.kmax, R.X.shape[1])
            L = None
        for k in tree.children(s):
            S_keep.pop(k, None)
        S_keep[s] = S
        fac.lu.append(lu)
        fac.R.append(R)
        fac.L.append(L)
        fac.S.append(S)
    for lst in (fac.lu, fac.R, fac.L, fac.S, fac.S_exact):
        lst.extend([None] * (tree.nnodes - last))
    return fac


def apply_compressed(fac: CompressedFactor, b: np.ndarray) -> np.ndarray:
    """Algorithm 3.1 with low-rank R, L where stored so (Sec. 3.5, last
    paragraph) and ULV solves for the diagonal blocks held in HSS form."""
    tree = fac.tree
    y = np.array(b, dtype=np.result_type(b.dtype, fac.dtype), copy=True)[tree.perm]
    for s in range(tree.nnodes):
        if tree.node_info[s, 7]:
            I, B = tree.I(s), tree.B(s)
            R = fac.R[s]
            y[B] += (R.rmatmat(y[I]) if fac.L[s] is None else fac.L[s] @ y[I])
    for s in range(tree.nnodes):
        I = tree.I(s)
        if I.size:
            if s in fac.ulv:
                order, U = fac.ulv[s]
                v = np.empty_like(y[I])
                v[order] = ulv_solve(U, y[I][order])
                y[I] = v
            else:
                y[I] = sla.lu_solve(fac.lu[s], y[I], check_finite=False)
    for s in range(tree.nnodes - 1, -1, -1):
        if tree.node_info[s, 7]:
            I, B = tree.I(s), tree.B(s)
            R = fac.R[s]
            y[I] += (R.matmat(y[B]) if isinstance(R, LowRank) else R @ y[B])
    x = np.empty_like(y)
    x[tree.perm] = y
    return x
