"""Pins of the oracle's nested dissection against Def. 3.1 and Sec. 3.1-3.3."""
import numpy as np
import pytest
import scipy.sparse as sp

from ndhss_inputs import helmholtz_impedance, poisson_dirichlet
from oracle.tree import build_tree


def _problems():
    return [poisson_dirichlet(64), poisson_dirichlet(23, seed=1),
            helmholtz_impedance(16, 2, 10.0), helmholtz_impedance(13, 1, 5.0)]


@pytest.fixture(scope="module", params=range(4))
def prob_tree(request):
    P = _problems()[request.param]
    return P, build_tree(P.coords, P.A.indptr, P.A.indices, 64)


def _elim_node(T):
    return np.repeat(np.arange(T.nnodes), T.f("m_i"))[T.iperm]


def _ancestors(T, s):
    out = []
    p = T.node_info[s, 1]
    while p >= 0:
        out.append(p)
        p = T.node_info[p, 1]
    return out


def test_def31_partition(prob_tree):
    """Index sets are disjoint and cover all DOFs (Def. 3.1, first two items)."""
    P, T = prob_tree
    assert np.array_equal(np.sort(T.perm), np.arange(P.n))
    assert np.array_equal(T.perm[T.iperm], np.arange(P.n))
    assert T.f("m_i").sum() == P.n


def test_def31_coupling_by_brute_force(prob_tree):
    """A(i, j) != 0 with i in I^mu, j in I^nu, mu > nu  =>  nu is a descendant of mu."""
    P, T = prob_tree
    e = _elim_node(T)
    C = P.A.tocoo()
    anc = {s: set(_ancestors(T, s)) for s in range(T.nnodes)}
    for i, j in zip(C.row, C.col):
        mu, nu = e[i], e[j]
        if mu > nu:
            assert mu in anc[nu]
        elif nu > mu:
            assert nu in anc[mu]


def test_postorder_and_levels(prob_tree):
    P, T = prob_tree
    par = T.f("parent")
    assert par[-1] == -1 and np.sum(par == -1) == 1
    assert np.all(par[:-1] > np.arange(T.nnodes - 1))            # children before parents
    lev = T.f("level")
    assert np.all(lev[:-1] == lev[par[:-1]] + 1)


def test_boundary_is_coupled_ancestor_superset(prob_tree):
    """B^s contains every ancestor DOF coupled to I^s (Sec. 3.1) and only ancestor DOFs."""
    P, T = prob_tree
    e = _elim_node(T)
    S = (P.A != 0).astype(np.int8) + (P.A.T != 0).astype(np.int8)
    S = S.tocsr()
    for s in range(T.nnodes):
        I = T.perm[T.I(s)]
        B = set(T.perm[T.B(s)].tolist())
        anc = set(_ancestors(T, s))
        for b in B:
            assert e[b] in anc
        coupled = set(S[I].indices.tolist()) if I.size else set()
        for j in coupled:
            if e[j] in anc:
                assert j in B


def test_well_separated_siblings(prob_tree):
    """B^mu and B^nu of siblings are disjoint (Sec. 3.1, Fig. 3)."""
    P, T = prob_tree
    for s in range(T.nnodes):
        ch = T.children(s)
        if len(ch) == 2:
            assert not set(T.B(ch[0]).tolist()) & set(T.B(ch[1]).tolist())


def test_subtrees_of_a_level_touch_disjoint_unknowns(prob_tree):
    """B^s lies in box s (R4), so the nodes of one subtree read and write only
    their own interior unknowns and the subtree root's B: the subtrees of a
    level own disjoint unknowns, and a subtree's work needs nothing from its
    siblings (the up and down sweeps of Alg. 3.1 can run a whole subtree
    without waiting on another)."""
    P, T = prob_tree
    lev = T.f("level")

    def nodes(s):
        out = [s]
        for k in T.children(s):
            out += nodes(k)
        return out

    for L0 in range(1, T.depth + 1):
        owner = np.full(P.n, -1)
        for r in np.nonzero(lev == L0)[0]:
            sub = nodes(int(r))
            own = np.concatenate([T.I(s) for s in sub])
            touched = np.unique(np.concatenate([own] + [T.B(s) for s in sub]))
            assert np.all(owner[touched] == -1)
            owner[touched] = r
            assert set(touched.tolist()) - set(own.tolist()) <= set(T.B(int(r)).tolist())


def test_every_entry_enters_one_front(prob_tree):
    """Each A(i, j) is scattered once, inside its front, at the LCA of its leaves."""
    P, T = prob_tree
    assert T.e_off[-1] == P.A.nnz
    assert np.array_equal(np.sort(T.e_idx), np.arange(P.A.nnz))
    m = T.f("m_i") + T.f("m_b")
    for s in range(T.nnodes):
        lo, hi = T.e_off[s], T.e_off[s + 1]
        assert np.all(T.e_row[lo:hi] < m[s]) and np.all(T.e_col[lo:hi] < m[s])
        pairs = set(zip(T.e_row[lo:hi].tolist(), T.e_col[lo:hi].tolist()))
        assert len(pairs) == hi - lo


def test_extend_add_map_is_injective_and_parent_conforming(prob_tree):
    """S^kappa rows land on distinct front rows, F(kappa) in I^sigma first (Fig. 4)."""
    P, T = prob_tree
    for s in range(T.nnodes):
        ch = T.children(s)
        if not ch:
            continue
        rows = np.concatenate([T.emap_of(k) for k in ch])
        assert np.unique(rows).size == rows.size
        m_i = T.node_info[s, 5]
        for k in ch:
            em = T.emap_of(k)
            nI = np.sum(em < m_i)
            assert np.all(em[:nI] < m_i) and np.all(em[nI:] >= m_i)
            # the global DOF at each mapped position is the same DOF
            glob = np.concatenate([T.I(s), T.B(s)])
            assert np.array_equal(glob[em], T.B(k))


def test_c1_tree_shape():
    P = poisson_dirichlet(64)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    assert T.nnodes == 127 and T.depth == 6
    assert T.node_info[-1, 5] == 126 and T.f("m_b").max() == 78


def _bisect(lo, hi, beta):
    if hi - lo <= beta:
        return [(lo, hi)]
    mid = lo + (hi - lo) // 2
    return [(lo, hi)] + _bisect(lo, mid, beta) + _bisect(mid, hi, beta)


def test_cross_block_hss_rank_at_most_one():
    """CG: A~_ii^(mu,nu) has HSS rank <= 1 in the aligned cluster trees (Sec. 3.3)."""
    P = poisson_dirichlet(64)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 16)
    A = P.A.tocsr()
    checked = 0
    for s in range(T.nnodes):
        ch = T.children(s)
        if len(ch) != 2:
            continue
        I = T.perm[T.I(s)]
        f0 = int(np.sum(T.emap_of(ch[0]) < T.node_info[s, 5]))
        X = A[I[:f0]][:, I[f0:]].toarray()          # A~_ii^(mu,nu)
        if min(X.shape) < 2:
            continue
        rc = _bisect(0, X.shape[0], 4)
        cc = _bisect(0, X.shape[1], 4)
        # same tree structure: compare block rows/cols of clusters at equal depth positions
        for (r0, r1) in rc:
            blk = X[r0:r1].copy()
            # remove the "diagonal" column cluster with the same relative extent
            c0 = round(r0 * X.shape[1] / X.shape[0])
            c1 = round(r1 * X.shape[1] / X.shape[0])
            blk[:, c0:c1] = 0
            assert np.linalg.matrix_rank(blk) <= 1
            checked += 1
    assert checked > 50
