"""Pins of the SIPG elastic-wave generator (ndhss_inputs/elastic.py) by what
the mathematics fixes: symmetry, rigid motions in the kernel of the static
operator, exact consistency for linear displacements (the discrete operator
returns the boundary traction load), the mass and the absorbing boundary
term on translations."""
import numpy as np
import pytest

from ndhss_inputs.elastic import elastic_sipg


def _field(P, fn):
    """DOF vector of the displacement field fn(x, y) -> (ux, uy) at the vertices."""
    elem, xy = P.meta["elem"], P.meta["xy"]
    X = xy[elem]                                         # [ne, 3, 2]
    U = np.stack(fn(X[..., 0], X[..., 1]), axis=-1)     # [ne, 3, 2]
    return U.reshape(-1).astype(np.complex128)


def test_symmetric_and_sizes():
    P = elastic_sipg(6, seed=1)
    A = P.A
    assert A.shape == (6 * 2 * 36, 6 * 2 * 36)
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()
    # every unknown couples to its own element and to at most three neighbours
    nnz_row = np.diff(A.indptr)
    assert nnz_row.max() <= 24 and nnz_row.min() >= 12
    lam, mu = P.meta["lam"], P.meta["mu"]
    assert lam.min() >= 1.0 and lam.max() <= 4.0 and mu.min() >= 1.0 and mu.max() <= 4.0
    assert P.coords.shape == (A.shape[0], 2)


@pytest.mark.parametrize("seed", [0, 3])
def test_rigid_motions_are_in_the_kernel_of_the_static_operator(seed):
    P = elastic_sipg(7, seed=seed, omega=0.0)
    A = P.A
    for fn in (lambda x, y: (np.ones_like(x), np.zeros_like(x)),
               lambda x, y: (np.zeros_like(x), np.ones_like(x)),
               lambda x, y: (-y, x)):
        r = _field(P, fn)
        assert np.linalg.norm(A @ r) <= 1e-11 * abs(A).max() * np.linalg.norm(r)


def test_linear_displacement_gives_the_boundary_traction():
    lam, mu = 1.7, 0.9
    P = elastic_sipg(5, lam=lam, mu=mu, omega=0.0)
    G = np.array([[0.3, -1.1], [0.7, 0.4]])
    c0 = np.array([0.2, -0.5])
    u = _field(P, lambda x, y: (G[0, 0] * x + G[0, 1] * y + c0[0], G[1, 0] * x + G[1, 1] * y + c0[1]))
    eps = 0.5 * (G + G.T)
    sig = lam * np.trace(eps) * np.eye(2) + 2 * mu * eps
    # int over the boundary of (sigma n) . phi_a e_c, edge by edge
    elem, xy = P.meta["elem"], P.meta["xy"]
    b = np.zeros(P.A.shape[0])
    sides = [(lambda p: abs(p[1]) < 1e-12, (0.0, -1.0)), (lambda p: abs(p[0] - 1) < 1e-12, (1.0, 0.0)),
             (lambda p: abs(p[1] - 1) < 1e-12, (0.0, 1.0)), (lambda p: abs(p[0]) < 1e-12, (-1.0, 0.0))]
    for e in range(elem.shape[0]):
        for (i, j) in ((0, 1), (1, 2), (2, 0)):
            p, q = xy[elem[e, i]], xy[elem[e, j]]
            for on, n in sides:
                if on(p) and on(q):
                    t = sig @ np.array(n) * np.linalg.norm(q - p) / 2.0
                    for a in (i, j):
                        b[6 * e + 2 * a: 6 * e + 2 * a + 2] += t
    r = P.A @ u
    assert np.linalg.norm(r - b) <= 1e-11 * np.linalg.norm(b)


def test_mass_and_absorbing_terms_on_translations():
    rho = 1.3
    # lam = mu = 0: no stiffness, no penalty, no boundary term -> -omega^2 rho M
    P = elastic_sipg(6, lam=0.0, mu=0.0, rho=rho, omega=2.0)
    rx = _field(P, lambda x, y: (np.ones_like(x), np.zeros_like(x)))
    ry = _field(P, lambda x, y: (np.zeros_like(x), np.ones_like(x)))
    assert abs(rx @ (P.A @ rx) - (-4.0 * rho)) <= 1e-12
    assert abs(rx @ (P.A @ ry)) <= 1e-12
    # constant lam, mu: -omega^2 rho |Omega| - i omega rho (c_p |sides with n = +-e_x| + c_s |sides with t = +-e_x|)
    lam, mu, om = 2.0, 1.5, 3.0
    P = elastic_sipg(6, lam=lam, mu=mu, rho=rho, omega=om)
    cp, cs = np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho)
    rx = _field(P, lambda x, y: (np.ones_like(x), np.zeros_like(x)))
    want = -om * om * rho - 1j * om * rho * 2.0 * (cp + cs)
    assert abs(rx @ (P.A @ rx) - want) <= 1e-11 * abs(want)


def test_default_frequency_and_source():
    P = elastic_sipg(8, seed=2)
    cs = P.meta["cs"]
    assert np.isclose(P.meta["omega"], 2 * np.pi * cs.min() / (8.0 / 8))
    b = P.b
    assert b.shape == (P.A.shape[0],) and np.all(np.isfinite(b))
    # both components carry the same projected force
    assert np.allclose(b[0::2], b[1::2])
