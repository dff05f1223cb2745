"""Pins of the oracle's exact front factorization (Sec. 3.1) and Algorithm 3.1."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from ndhss_inputs import helmholtz_impedance, poisson_dirichlet
from oracle.frontal import apply_inverse, factor_dense, factor_node
from oracle.tree import build_tree


@pytest.fixture(scope="module", params=["poisson", "helmholtz_p2", "helmholtz_p1_leaf16"])
def setup(request):
    if request.param == "poisson":
        P, leaf = poisson_dirichlet(40, seed=2), 64
    elif request.param == "helmholtz_p2":
        P, leaf = helmholtz_impedance(20, 2, 15.0, seed=1), 64
    else:
        P, leaf = helmholtz_impedance(30, 1, 12.0, seed=4), 16
    T = build_tree(P.coords, P.A.indptr, P.A.indices, leaf)
    return P, T, factor_dense(T, P.A)


def test_exact_mode_equals_direct_solve(setup):
    """No compression: P^{-1} b = A^{-1} b (a sparse direct solver, Sec. 3.2)."""
    P, T, fac = setup
    x = apply_inverse(fac, P.b)
    xd = spla.spsolve(P.A.tocsc(), P.b)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_schur_equals_dense_schur_of_box(setup):
    """S^s = A(BL,BL) - A(BL,E) A(E,E)^{-1} A(E,BL) with E = box(s) \\ BL(s) (Eq. 3.5)."""
    P, T, fac = setup
    A = P.A.toarray()
    lev = T.f("level")
    sel = [s for s in range(T.nnodes) if T.node_info[s, 7] > 0]
    sel = sel[:: max(1, len(sel) // 25)]
    for s in sel:
        x0, x1, y0, y1 = T.node_info[s, 8:12]
        c = P.coords
        box = np.nonzero((c[:, 0] >= x0) & (c[:, 0] < x1) & (c[:, 1] >= y0) & (c[:, 1] < y1))[0]
        Bold = T.perm[T.B(s)]
        E = np.setdiff1d(box, Bold)
        Sd = A[np.ix_(Bold, Bold)] - A[np.ix_(Bold, E)] @ np.linalg.solve(A[np.ix_(E, E)], A[np.ix_(E, Bold)])
        assert np.linalg.norm(fac.S[s] - Sd) <= 1e-11 * np.linalg.norm(Sd), (s, lev[s])


def test_symmetric_operator_gives_symmetric_factor(setup):
    """A = A^T  =>  L^s = (R^s)^T and S^s = (S^s)^T (Eq. 3.3 with A_ii^T = A_ii)."""
    P, T, fac = setup
    for s in range(T.nnodes):
        if T.node_info[s, 7] == 0:
            continue
        scale = max(np.abs(fac.R[s]).max(), 1e-300)
        assert np.abs(fac.L[s] - fac.R[s].T).max() <= 1e-11 * scale
        assert np.abs(fac.S[s] - fac.S[s].T).max() <= 1e-11 * max(np.abs(fac.S[s]).max(), 1e-300)


def test_front_block_identity():
    """For one dense front, [I 0; -L I] diag(A_ii, S) [I -R; 0 I] reproduces it (Eq. 3.2)."""
    rng = np.random.default_rng(0)
    m, m_i = 37, 21
    F = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)) + 8 * np.eye(m)
    lu, L, R, S = factor_node(F, m_i)
    Lh = np.eye(m, dtype=complex)
    Lh[m_i:, :m_i] = -L
    Rh = np.eye(m, dtype=complex)
    Rh[:m_i, m_i:] = -R
    D = np.zeros_like(F)
    D[:m_i, :m_i] = F[:m_i, :m_i]
    D[m_i:, m_i:] = S
    assert np.abs(Lh @ D @ Rh - F).max() <= 1e-12 * np.abs(F).max()


def test_planted_sign_error_is_caught(setup, monkeypatch):
    """A dropped minus sign in R (Eq. 3.3b) breaks the direct-solve pin."""
    P, T, _ = setup
    import oracle.frontal as fr
    orig = fr.factor_node

    def bad(F, m_i):
        lu, L, R, S = orig(F, m_i)
        return lu, L, -R, S

    monkeypatch.setattr(fr, "factor_node", bad)
    fac = fr.factor_dense(T, P.A)
    x = fr.apply_inverse(fac, P.b)
    xd = spla.spsolve(P.A.tocsc(), P.b)
    assert np.linalg.norm(x - xd) > 1e-6 * np.linalg.norm(xd)
