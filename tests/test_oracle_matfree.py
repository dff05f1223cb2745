"""Pins of the oracle's matrix-free upper tier (Sec. 3.2 - 3.5, Alg. 3.3,
Alg. 3.4's upper branch): every implicit operator against the dense front
of Eq. 3.4 built by the separate dense code, Alg. 3.3 against a dense
solve, R and S against the dense elimination (Eq. 3.5, 3.7), the whole
preconditioner against a sparse direct solve, the matrix-free property
itself (no front above the switching level is assembled), and the rank
claim of Sec. 3.3 for P1 continuous elements under this numbering."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle.matfree as mf
from ndhss_inputs import helmholtz_impedance, poisson_dirichlet
from oracle.frontal import assemble_front
from oracle.gmres import gmres
from oracle.hss import cluster_tree, hss_compress, hss_dense
from oracle.tree import build_tree


def _sym(n, rank, cplx, seed):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, n)
    K = np.exp(-np.abs(x[:, None] - x[None, :]) * 3.0)          # smooth kernel: low-rank off-diagonal blocks
    if cplx:
        K = K * np.exp(1j * 2.0 * (x[:, None] + x[None, :]))     # complex symmetric
    G = rng.standard_normal((n, rank))
    return K + 0.1 * G @ G.T + np.diag(rng.uniform(1, 2, n))


@pytest.mark.parametrize("cplx", [False, True])
def test_hss_entries_sub_blocks_and_coupling_match_reconstruction(cplx):
    n, top = 230, 97
    A = _sym(n, 3, cplx, 0)
    H = hss_compress(A, cluster_tree(n, top, 24), 1e-9, seed=1, stream=2)
    Hd = hss_dense(H)                                           # telescoping products (Eq. 2.5)
    rng = np.random.default_rng(3)
    I, J = rng.integers(0, n, 60), rng.integers(0, n, 45)
    E = mf.hss_entries(H, I, J)
    assert np.abs(E - Hd[np.ix_(I, J)]).max() <= 1e-13 * np.abs(Hd).max()
    for lo, hi in ((0, top), (top, n)):
        Hs = mf.diag_block(H, lo, hi)
        assert np.abs(hss_dense(Hs) - Hd[lo:hi, lo:hi]).max() <= 1e-13 * np.abs(Hd).max()
    cp = mf.root_coupling(H, top)
    X = rng.standard_normal((n - top, 3))
    Y = rng.standard_normal((top, 3))
    assert np.allclose(cp.mm12(X), Hd[:top, top:] @ X, rtol=0, atol=1e-12 * np.abs(Hd).max() * n)
    assert np.allclose(cp.mm21(Y), Hd[top:, :top] @ Y, rtol=0, atol=1e-12 * np.abs(Hd).max() * n)
    # a one-leaf HSS matrix: the dense block itself
    A20 = A[:20, :20].copy()
    H1 = hss_compress(A20, cluster_tree(20, 7, 24), 1e-9)
    assert np.array_equal(mf.hss_entries(H1, [3, 19], [0, 5]), A20[np.ix_([3, 19], [0, 5])])
    assert np.array_equal(mf.root_coupling(H1, 7).mm12(np.eye(13)), A20[:7, 7:])


def test_operator_form_of_alg_a1_is_the_dense_form():
    """hss_compress reads a matrix only through products and entries: an
    operator that answers them from the same array gives the same HSS."""
    A = _sym(150, 2, True, 4)

    class Op:
        shape, dtype = A.shape, A.dtype

        def matmat(self, X):
            return A @ X

        def entries(self, I, J):
            return A[np.ix_(I, J)]

    T = cluster_tree(150, 60, 20)
    H1, H2 = hss_compress(A, T, 1e-8, seed=2, stream=9), hss_compress(Op(), T, 1e-8, seed=2, stream=9)
    assert np.array_equal(hss_dense(H1), hss_dense(H2)) and H1.samples == H2.samples


def _problem(kind):
    if kind == "poisson":
        return poisson_dirichlet(32, p=1, seed=0)
    return helmholtz_impedance(24, 2, 12.0, seed=0)


def _matfree_nodes(tree, fac):
    return [s for s in range(tree.nnodes) if s in fac.binv and tree.node_info[s, 5] > 0]


@pytest.fixture(scope="module", params=["poisson", "helmholtz"])
def setup(request):
    P = _problem(request.param)
    t = build_tree(P.coords, P.A.indptr, P.A.indices, 32)
    fac = mf.factor_matfree(t, P.A, hss_levels=3, eps=1e-11, beta=16)
    return P, t, fac


def _dense_front(P, t, fac, s):
    """Eq. 3.4 assembled densely from the children's reconstructed S."""
    Sd = {k: hss_dense(fac.hss[k]) for k in t.children(s) if k in fac.hss}
    for k in t.children(s):
        if k not in Sd:
            Sd[k] = np.zeros((0, 0))
    return assemble_front(t, s, P.A, Sd)


def test_implicit_front_operators_equal_the_assembled_front(setup):
    P, t, fac = setup
    rng = np.random.default_rng(0)
    nodes = _matfree_nodes(t, fac)
    assert nodes
    for s in nodes:
        F = _dense_front(P, t, fac, s)
        front = mf.ImplicitFront(t, s, P.A, fac.hss)
        mi, mb = front.m_i, front.m_b
        scale = np.abs(F).max()
        Xb = rng.standard_normal((mb, 3))
        Xi = rng.standard_normal((mi, 3))
        tol = 1e-12 * scale * max(mi, mb, 1)
        if mb:
            assert np.abs(front.aib(Xb) - F[:mi, mi:] @ Xb).max() <= tol
            assert np.abs(front.abi(Xi) - F[mi:, :mi] @ Xi).max() <= tol
            assert np.abs(front.abb(Xb) - F[mi:, mi:] @ Xb).max() <= tol
            I, J = rng.integers(0, mb, 17), rng.integers(0, mb, 11)
            assert np.abs(front.abb_entries(I, J) - F[mi:, mi:][np.ix_(I, J)]).max() <= 1e-13 * scale


def test_alg33_block_inverse_equals_a_dense_solve(setup):
    P, t, fac = setup
    rng = np.random.default_rng(1)
    for s in _matfree_nodes(t, fac):
        F = _dense_front(P, t, fac, s)
        mi = int(t.node_info[s, 5])
        X = rng.standard_normal((mi, 2)) + (1j * rng.standard_normal((mi, 2)) if np.iscomplexobj(F) else 0)
        ref = np.linalg.solve(F[:mi, :mi], X)
        got = fac.binv[s].solve(X)
        assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref), s


def test_R_and_S_equal_the_dense_elimination(setup):
    """Eq. 3.7 and Eq. 3.5 from the implicit front, against the dense
    elimination of the assembled front (compression tolerance 1e-11)."""
    P, t, fac = setup
    for s in _matfree_nodes(t, fac):
        mi, mb = int(t.node_info[s, 5]), int(t.node_info[s, 7])
        if mb == 0:
            continue
        F = _dense_front(P, t, fac, s)
        Rd = -np.linalg.solve(F[:mi, :mi], F[:mi, mi:])
        Sd = F[mi:, mi:] + F[mi:, :mi] @ Rd
        R = fac.R[s]
        assert np.linalg.norm(R.X @ R.RJ - Rd) <= 1e-7 * np.linalg.norm(Rd), s
        Sh = hss_dense(fac.hss[s])
        assert np.linalg.norm(Sh - Sd) <= 1e-7 * np.linalg.norm(Sd), s
        assert np.linalg.norm(Sh - Sh.T) <= 1e-7 * np.linalg.norm(Sd)     # symmetric operator, symmetric S


def test_sampled_operators_equal_their_dense_definitions(setup):
    """The products and entries Alg. A.1 and the range finder draw on: S~
    (Alg. 3.3), R (Eq. 3.7) and S (Eq. 3.5), each against its definition on
    the assembled front.  (A.1 takes the HSS values from entries; a wrong
    product only shows as bases fitted to another matrix and a sampling
    loop that runs to its cap, so the products are pinned here directly.)"""
    P, t, fac = setup
    rng = np.random.default_rng(2)
    for s in _matfree_nodes(t, fac):
        F = _dense_front(P, t, fac, s)
        front = mf.ImplicitFront(t, s, P.A, fac.hss)
        mi, mb, n1 = front.m_i, front.m_b, front.n1
        binv = fac.binv[s]
        if n1 and mi > n1:
            St = F[n1:mi, n1:mi] - F[n1:mi, :n1] @ np.linalg.solve(F[:n1, :n1], F[:n1, n1:mi])
            op = mf.SchurOp(front.parts[1].Sii, binv.U1, front.A12, front.A21)
            X = rng.standard_normal((mi - n1, 3))
            assert np.linalg.norm(op.matmat(X) - St @ X) <= 1e-9 * np.linalg.norm(St @ X)
            I, J = rng.integers(0, mi - n1, 9), rng.integers(0, mi - n1, 7)
            assert np.abs(op.entries(I, J) - St[np.ix_(I, J)]).max() <= 1e-9 * np.abs(St).max()
        if not mb:
            continue
        Rd = -np.linalg.solve(F[:mi, :mi], F[:mi, mi:])
        rop = mf.ROp(front, binv)
        X = rng.standard_normal((mb, 3))
        assert np.linalg.norm(rop.matmat(X) - Rd @ X) <= 1e-8 * np.linalg.norm(Rd @ X)
        J = rng.integers(0, mi, 5)
        assert np.linalg.norm(rop.rows(J) - Rd[J]) <= 1e-8 * np.linalg.norm(Rd[J]) + 1e-14
        R = fac.R[s]
        Sr = F[mi:, mi:] + F[mi:, :mi] @ (R.X @ R.RJ)
        sop = mf.SOp(front, R)
        assert np.linalg.norm(sop.matmat(X) - Sr @ X) <= 1e-10 * np.linalg.norm(Sr @ X)
        I, J = rng.integers(0, mb, 9), rng.integers(0, mb, 7)
        assert np.abs(sop.entries(I, J) - Sr[np.ix_(I, J)]).max() <= 1e-10 * np.abs(Sr).max()


@pytest.mark.parametrize("kind", ["poisson", "helmholtz"])
def test_matfree_preconditioner_reaches_the_direct_solve(kind):
    P = _problem(kind)
    t = build_tree(P.coords, P.A.indptr, P.A.indices, 32)
    b = P.b[:, 0] if P.b.ndim > 1 else P.b
    x = spla.spsolve(P.A.tocsc(), b)
    fac = mf.factor_matfree(t, P.A, hss_levels=3, eps=1e-11, beta=16)
    assert fac.binv
    y = mf.apply_matfree(fac, b)
    assert np.linalg.norm(y - x) <= 1e-7 * np.linalg.norm(x)
    fac6 = mf.factor_matfree(t, P.A, hss_levels=3, eps=1e-6, beta=16)
    r = gmres(P.A, b, lambda v: mf.apply_matfree(fac6, v), tol=1e-8)
    assert r.converged and r.iters <= 4, (r.iters, r.true_relres)
    assert np.linalg.norm(r.x - x) <= 1e-6 * np.linalg.norm(x)


def test_no_front_above_the_switching_level_is_assembled(monkeypatch):
    P = helmholtz_impedance(24, 1, 10.0, seed=0)
    t = build_tree(P.coords, P.A.indptr, P.A.indices, 32)
    seen = []
    real = mf.assemble_front

    def spy(tree, s, A, S):
        seen.append(s)
        return real(tree, s, A, S)

    monkeypatch.setattr(mf, "assemble_front", spy)
    fac = mf.factor_matfree(t, P.A, hss_levels=3, eps=1e-6, beta=16)
    lev = t.node_info[:, 0]
    upper = [s for s in range(t.nnodes) if lev[s] < fac.L_hss and t.children(s)]
    assert upper and not set(upper) & set(seen)
    assert set(upper) == set(fac.binv)


def test_sec33_p1_cross_couplings_have_at_most_one_entry_outside_the_facing_cluster():
    """Sec. 3.3: with P1 continuous elements and facing DOFs numbered alike,
    a cluster of A~^(mu,nu)'s rows couples outside the facing column cluster
    through at most one entry (HSS rank <= 1), and likewise for columns.
    Checked on every node whose two interior parts have equal size (so the
    cluster trees match level by level)."""
    P = poisson_dirichlet(64, p=1, seed=0)
    t = build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    checked = 0
    for s in range(t.nnodes):
        kids = t.children(s)
        if len(kids) != 2:
            continue
        mi = int(t.node_info[s, 5])
        n1 = int(np.sum(t.emap_of(kids[0]) < mi))
        if n1 < 16 or mi - n1 != n1:
            continue
        lo, hi = t.e_off[s], t.e_off[s + 1]
        r, c = t.e_row[lo:hi], t.e_col[lo:hi]
        m = (r < n1) & (c >= n1) & (c < mi)
        At = sp.csr_matrix((np.ones(m.sum()), (r[m], c[m] - n1)), shape=(n1, n1)).toarray()
        T = cluster_tree(n1, None, 8)
        for cl in T[1:]:
            out_c = np.ones(n1, bool)
            out_c[cl.lo:cl.hi] = False
            assert np.count_nonzero(At[cl.lo:cl.hi][:, out_c]) <= 1
            assert np.count_nonzero(At[out_c][:, cl.lo:cl.hi]) <= 1
            checked += 1
    assert checked >= 20


def test_sec34_rank_bound_of_R(setup):
    """Sec. 3.4: rank R = rank A_ib <= rank S_ib^mu + rank S_ib^nu + nnz A~_ib^(mu,nu)
    + nnz A~_ib^(nu,mu), where the children's couplings S_ib are their HSS
    root couplings U_1 B_12 U_2^T (rank <= the smaller basis width).  The
    numerical rank of the dense R of the assembled front respects it."""
    P, t, fac = setup
    checked = 0
    for s in _matfree_nodes(t, fac):
        mi, mb = int(t.node_info[s, 5]), int(t.node_info[s, 7])
        if mb == 0:
            continue
        F = _dense_front(P, t, fac, s)
        R = np.linalg.solve(F[:mi, :mi], F[:mi, mi:])
        sv = np.linalg.svd(R, compute_uv=False)
        rank = int(np.sum(sv > 1e-10 * sv[0]))
        front = mf.ImplicitFront(t, s, P.A, fac.hss)
        bound = front.Sib.nnz
        for part in front.parts:
            cp = part.cp
            if part.ni and part.pb.size:
                bound += min(cp.D12.shape) if cp.D12 is not None else min(cp.B12.shape)
        assert rank <= bound, (s, rank, bound)
        assert rank < min(mi, mb) or bound >= min(mi, mb)
        checked += 1
    assert checked


def test_matfree_on_a_lattice_with_holes():
    """Empty boxes (size-0 leaves), leaves above the switching level and
    children without a Schur complement: the tier still reproduces the
    direct solve at a tight tolerance."""
    P = poisson_dirichlet(32, p=1, seed=0)
    keep = np.nonzero((P.coords[:, 0] < 10) | (P.coords[:, 0] > 20) | (P.coords[:, 1] < 12))[0]
    A = P.A[keep][:, keep].tocsr()
    A.sort_indices()
    coords = P.coords[keep]
    b = np.asarray(P.b if P.b.ndim == 1 else P.b[:, 0])[keep]
    t = build_tree(coords, A.indptr, A.indices, 20)
    assert np.any(t.f("m_i") + t.f("m_b") == 0)
    fac = mf.factor_matfree(t, A, hss_levels=1, eps=1e-11, beta=8)
    lev = t.node_info[:, 0]
    assert fac.binv
    assert any(not t.children(s) and lev[s] < fac.L_hss for s in range(t.nnodes))   # a leaf above L_HSS
    x = spla.spsolve(A.tocsc(), b)
    y = mf.apply_matfree(fac, b)
    assert np.linalg.norm(y - x) <= 1e-7 * np.linalg.norm(x)
