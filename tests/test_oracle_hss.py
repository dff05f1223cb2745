"""Pins of the oracle's HSS machinery (Sec. 2.1-2.3, App. A) and of the
compressed factorization (Alg. 3.4)."""
import os

import numpy as np
import pytest

from ndhss_inputs import helmholtz_impedance, poisson_dirichlet
from oracle.frontal import apply_inverse, factor_dense
from oracle.gmres import gmres
from oracle.hss import (HSS, apply_compressed, cluster_tree, factor_compressed, gaussian, hss_compress,
                        hss_dense, hss_matvec, lowrank_rows, philox4x32_10, row_id, ulv_factor, ulv_solve)
from oracle.tree import build_tree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        out = philox4x32_10(np.array([v[:4]], dtype=np.uint32), (v[4], v[5]))[0]
        assert [int(x) for x in out] == v[6:]


def test_gaussian_moments_and_determinism():
    G = gaussian(400, 50, seed=7, stream=3)
    assert abs(G.mean()) < 0.02 and abs(G.std() - 1.0) < 0.02
    assert np.array_equal(G, gaussian(400, 50, seed=7, stream=3))
    assert not np.array_equal(G, gaussian(400, 50, seed=7, stream=4))
    # column-major element order: a taller matrix extends, it does not reshuffle, the first column
    assert np.array_equal(gaussian(400, 1, 7, 3)[:, 0], G[:, 0])


def test_cluster_tree_fig4_split_and_leaf_size():
    T = cluster_tree(300, 130, 40)
    assert (T[0].lo, T[0].hi) == (0, 300)
    c1, c2 = T[0].children
    assert (T[c1].lo, T[c1].hi, T[c2].lo, T[c2].hi) == (0, 130, 130, 300)
    for c in T:
        if c.children:
            a, b = T[c.children[0]], T[c.children[1]]
            assert a.lo == c.lo and a.hi == b.lo and b.hi == c.hi
        else:
            assert c.size <= 40


def _random_hss(n, top, beta, k, seed, cplx=True):
    rng = np.random.default_rng(seed)
    T = cluster_tree(n, top, beta)
    H = HSS(n=n, tree=T, dtype=np.complex128 if cplx else np.float64)
    z = (lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)) if cplx else (lambda *s: rng.standard_normal(s))
    for i, c in enumerate(T):
        if i == 0:
            continue
        if not c.children:
            H.U[i] = z(c.size, k)
            D = z(c.size, c.size)
            H.D[i] = D + D.T
        else:
            H.U[i] = z(2 * k, k)
    for i, c in enumerate(T):
        if c.children:
            B = z(k, k)
            H.B12[i], H.B21[i] = B, B.T
    return H


@pytest.mark.parametrize("cplx", [False, True])
def test_exact_hss_recovery(cplx):
    """A matrix with exact HSS rank k (Def. 2.3) is recovered to round-off by Alg. A.1."""
    H = _random_hss(300, 130, 40, 6, seed=1, cplx=cplx)
    A = hss_dense(H)
    assert np.abs(A - A.T).max() <= 1e-10 * np.abs(A).max()
    Hc = hss_compress(A, H.tree, 1e-10, k0=8, r=8, seed=3)
    assert np.linalg.norm(hss_dense(Hc) - A) <= 1e-12 * np.linalg.norm(A)
    assert Hc.kmax() <= 6


def test_hss_matvec_is_linear_and_matches_dense():
    H = _random_hss(200, 90, 30, 5, seed=2)
    A = hss_dense(H)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((200, 3))
    assert np.allclose(hss_matvec(H, x), A @ x, rtol=1e-12, atol=1e-12 * np.abs(A).max())


def test_row_id_skeleton_rows_exact():
    rng = np.random.default_rng(4)
    S = rng.standard_normal((60, 8)) @ rng.standard_normal((8, 40))
    J, X = row_id(S, 1e-12, 40)
    assert len(J) == 8
    assert np.array_equal(X[J], np.eye(8))
    assert np.linalg.norm(X @ S[J] - S) <= 1e-10 * np.linalg.norm(S)


def test_estimator_detects_truncation():
    """Too small a rank budget leaves an error the estimator (Eq. 2.7) sees."""
    x = np.linspace(0, 1, 256)
    A = 1.0 / (1.0 + 30 * np.abs(x[:, None] - x[None, :]))      # smooth, numerically low HSS rank
    T = cluster_tree(256, 128, 32)
    H = hss_compress(A, T, 1e-10, k0=4, r=4, seed=5, rank_cap=6)
    err = np.linalg.norm(hss_dense(H) - A) / np.linalg.norm(A)
    assert err > 1e-8                                   # truncated by the rank cap
    H2 = hss_compress(A, T, 1e-8, k0=4, r=4, seed=5)
    assert np.linalg.norm(hss_dense(H2) - A) <= 1e-7 * np.linalg.norm(A)
    assert H2.rounds > 1                                # the adaptive loop grew the rank


def test_lowrank_rows():
    rng = np.random.default_rng(6)
    R = (rng.standard_normal((120, 15)) @ rng.standard_normal((15, 90))).astype(complex)
    lr = lowrank_rows(R, 1e-8, k0=8, r=8, seed=1)
    assert lr.X.shape[1] == 15
    assert np.linalg.norm(lr.matmat(np.eye(90)) - R) <= 1e-10 * np.linalg.norm(R)


@pytest.fixture(scope="module", params=["poisson", "helmholtz"])
def compressed(request):
    P = poisson_dirichlet(64) if request.param == "poisson" else helmholtz_impedance(48, 2, 12.0, seed=3)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    return P, T, factor_compressed(T, P.A, hss_levels=3, eps=1e-6)


def test_compressed_schur_within_tolerance(compressed):
    """Every compressed S meets the HSS tolerance measured directly (Sec. 3.2)."""
    P, T, fac = compressed
    assert fac.hss
    for s, H in fac.hss.items():
        Se = fac.S_exact[s]
        assert np.linalg.norm(hss_dense(H) - Se) <= 20 * 1e-6 * np.linalg.norm(Se), s


def test_compressed_preconditioner_converges_fast(compressed):
    P, T, fac = compressed
    r = gmres(P.A, P.b, lambda v: apply_compressed(fac, v), tol=1e-8)
    assert r.converged and r.iters <= 5
    # without compression the same routine is the exact factorization
    fac0 = factor_compressed(T, P.A, hss_levels=T.depth + 1)
    assert not fac0.hss
    x0 = apply_compressed(fac0, P.b)
    assert np.allclose(x0, apply_inverse(factor_dense(T, P.A), P.b), rtol=1e-10, atol=1e-14)


def _kernel_matrix(n, dtype, seed):
    rng = np.random.default_rng(seed)
    x = np.sort(rng.random(n))
    A = 1.0 / (1.0 + 40 * np.abs(x[:, None] - x[None, :])) + np.diag(0.5 + rng.random(n))
    if dtype == np.complex128:
        A = A + 1j * (np.cos(7 * x[:, None] + 7 * x[None, :]) / (1 + 30 * np.abs(x[:, None] - x[None, :])))
    return (A + A.T) / 2                               # symmetric, complex symmetric when complex


@pytest.mark.parametrize("dtype", [np.float64, np.complex128])
@pytest.mark.parametrize("n,top,beta,eps", [(300, 140, 40, 1e-10), (257, None, 24, 1e-4), (90, 30, 16, 1e-14),
                                            (50, None, 64, 1e-8)])
def test_ulv_solve_equals_dense_solve_of_the_hss_matrix(dtype, n, top, beta, eps):
    """The ULV factorization is exact for the HSS matrix it factors: its solve
    equals a dense solve of the reconstruction (to rounding), including
    nodes whose rank reaches their size (nothing to eliminate, eps 1e-14)
    and the single-block tree (beta >= n)."""
    A = _kernel_matrix(n, dtype, 1)
    H = hss_compress(A, cluster_tree(n, top, beta), eps, seed=5)
    F = ulv_factor(H)
    rng = np.random.default_rng(2)
    b = rng.standard_normal((n, 3)).astype(dtype)
    xd = np.linalg.solve(hss_dense(H), b)
    assert np.linalg.norm(ulv_solve(F, b) - xd) <= 1e-11 * np.linalg.norm(xd)
    assert np.linalg.norm(ulv_solve(F, b[:, 0]) - xd[:, 0]) <= 1e-11 * np.linalg.norm(xd[:, 0])


def test_ulv_uses_transposes_not_conjugates():
    """For a complex symmetric (not Hermitian) HSS matrix the column bases
    enter as U^T; the same factorization of the Hermitian-ised coupling
    (conjugated column bases) would solve a different matrix."""
    A = _kernel_matrix(200, np.complex128, 3)
    H = hss_compress(A, cluster_tree(200, 90, 32), 1e-10, seed=1)
    b = np.ones(200, dtype=np.complex128)
    x = ulv_solve(ulv_factor(H), b)
    assert np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b)
    Hc = HSS(n=H.n, tree=H.tree, U=dict(H.U), D=dict(H.D), B12={i: v.conj() for i, v in H.B12.items()},
             B21={i: v.conj() for i, v in H.B21.items()}, skel=H.skel, dtype=H.dtype)
    xc = ulv_solve(ulv_factor(Hc), b)
    assert np.linalg.norm(A @ xc - b) > 1e-3 * np.linalg.norm(b)


def test_ulv_preconditioner_matches_dense_diagonal_within_tolerance(compressed):
    """A_ii in HSS form with its ULV solve changes the preconditioner by the
    compression tolerance only, and GMRES still converges as fast."""
    P, T, fac = compressed
    facu = factor_compressed(T, P.A, hss_levels=3, eps=1e-6, ulv=True)
    assert facu.ulv and all(int(T.node_info[s, 0]) < facu.L_hss for s in facu.ulv)
    b = P.b if P.b.ndim == 1 else P.b[:, 0]
    y0, y1 = apply_compressed(fac, b), apply_compressed(facu, b)
    assert np.linalg.norm(y1 - y0) <= 1e-4 * np.linalg.norm(y0)
    r = gmres(P.A, b, lambda v: apply_compressed(facu, v), tol=1e-8)
    assert r.converged and r.iters <= 5


def test_stopping_rule_keeps_sampling_a_slowly_decaying_spectrum():
    """A spectrum decaying by 0.93 per index: r = 4 more samples never halve the
    estimate, but it is far above the float64 floor, so sampling goes on until
    eps is met (within the 100 eps that an eps-truncated interpolative
    decomposition of a slowly decaying tail reaches; a rule that stopped at any
    non-halving round returns rank 6 and an error of 0.85 here)."""
    from oracle.hss import MAX_SAMPLES, STAGNATION_FLOOR, _stop
    rng = np.random.default_rng(11)
    m, nb = 200, 180
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((nb, nb)))
    s = 0.93 ** np.arange(nb)
    R = (U[:, :nb] * s) @ V.T
    lr = lowrank_rows(R, 1e-6, k0=8, r=4, seed=3)
    err = np.linalg.norm(lr.matmat(np.eye(nb)) - R) / np.linalg.norm(R)
    assert err <= 100 * 1e-6, err
    assert lr.X.shape[1] > 150                      # the rank eps asks for (0.93^k ~ 1e-6 near k ~ 190)
    # the rule itself: stagnation stops only at the floor, the sample cap always
    assert not _stop(1e-3, 1.0, 1e-6, 1.5e-3, 64, 500, 16)
    assert _stop(STAGNATION_FLOOR / 2, 1.0, 1e-20, STAGNATION_FLOOR / 1.5, 64, 500, 16)
    assert _stop(1e-3, 1.0, 1e-6, 1.0, MAX_SAMPLES - 8, 500, 16)
    assert not _stop(1e-3, 1.0, 1e-6, 1.0, MAX_SAMPLES - 16, 500, 16)


def test_factor_compressed_subtree_equals_full_factorization_on_that_subtree():
    """A front depends only on its own subtree: factoring one subtree alone
    gives bit for bit the blocks the full factorization gives there."""
    from ndhss_inputs import helmholtz_impedance
    from oracle.hss import factor_compressed
    from oracle.tree import build_tree
    P = helmholtz_impedance(40, 1, 10.0, seed=3)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 32)
    full = factor_compressed(T, P.A, hss_levels=3, eps=1e-6, beta=32, k0=16, r=8, seed=4)
    lev = T.f("level")
    s0 = int(np.nonzero(lev == 1)[0][0])
    sub = factor_compressed(T, P.A, hss_levels=3, eps=1e-6, beta=32, k0=16, r=8, seed=4, subtree=s0)
    inside = [s for s in range(T.nnodes) if sub.S[s] is not None]
    def members(s):
        return [s] + [d for c in T.children(s) for d in members(c)]
    assert sorted(inside) == sorted(members(s0))
    assert all(sub.S[s] is None for s in range(T.nnodes) if s not in inside)
    lowrank = 0
    for s in inside:
        assert np.array_equal(sub.S[s], full.S[s])
        if hasattr(full.R[s], "matmat"):
            assert np.array_equal(sub.R[s].X, full.R[s].X) and np.array_equal(sub.R[s].RJ, full.R[s].RJ)
            lowrank += 1
        else:
            assert np.array_equal(sub.R[s], full.R[s])
    assert lowrank > 0


@pytest.mark.parametrize("case", ["poisson", "helmholtz"])
def test_compressed_apply_converges_to_the_exact_apply_as_eps_shrinks(case):
    """With compression active on every level at and above the switching level
    (HSS S, low-rank R and L = R^T above it) and eps = 1e-12, Alg. 3.1 on the
    compressed factor agrees with the exact dense factor's apply to ~1e-9;
    at eps = 1e-6 the difference is orders of magnitude larger.  A transposed
    or dropped low-rank block, or a sign error in the up or down sweep, fails
    the tight bound."""
    P = poisson_dirichlet(48) if case == "poisson" else helmholtz_impedance(40, 2, 10.0, seed=5)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 32)
    exact = apply_inverse(factor_dense(T, P.A), P.b)
    tight = factor_compressed(T, P.A, hss_levels=3, eps=1e-12)
    loose = factor_compressed(T, P.A, hss_levels=3, eps=1e-6)
    assert tight.hss and tight.kmax > 0
    lr_nodes = [s for s, R in tight.R.items() if hasattr(R, "matmat")] if isinstance(tight.R, dict) else \
               [s for s in range(T.nnodes) if tight.R[s] is not None and hasattr(tight.R[s], "matmat")]
    assert lr_nodes, "no low-rank Gauss transform was exercised"
    e_tight = np.linalg.norm(apply_compressed(tight, P.b) - exact) / np.linalg.norm(exact)
    e_loose = np.linalg.norm(apply_compressed(loose, P.b) - exact) / np.linalg.norm(exact)
    assert e_tight <= 1e-9, e_tight
    assert e_loose >= 100 * e_tight, (e_loose, e_tight)
