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


def _manufactured_error(N, lam, mu, omega):
    """L2 error of the SIPG solution for u = u_c + u_g (u_c divergence-free,
    u_g a gradient) with the load f = -div sigma(u) - omega^2 u and the
    boundary data g = sigma(u) n - i omega (c_p n n^T + c_s t t^T) u that the
    weak form's absorbing condition takes (rho = 1)."""
    import scipy.sparse.linalg as spla
    from ndhss_inputs.fem import _gauss_triangle
    pi = np.pi
    s, c = np.sin, np.cos

    def u(x, y):
        return s(pi * x) * s(pi * y) + c(pi * x) * s(pi * y), c(pi * x) * c(pi * y) + s(pi * x) * c(pi * y)

    def grad(x, y):             # d u_i / d x_j
        return ((pi * c(pi * x) * s(pi * y) - pi * s(pi * x) * s(pi * y),
                 pi * s(pi * x) * c(pi * y) + pi * c(pi * x) * c(pi * y)),
                (-pi * s(pi * x) * c(pi * y) + pi * c(pi * x) * c(pi * y),
                 -pi * c(pi * x) * s(pi * y) - pi * s(pi * x) * s(pi * y)))

    def f(x, y):                # div sigma(u_c) = -2 pi^2 mu u_c, div sigma(u_g) = -2 pi^2 (lam + 2 mu) u_g
        a1, a2 = 2 * pi * pi * mu - omega ** 2, 2 * pi * pi * (lam + 2 * mu) - omega ** 2
        return (a1 * s(pi * x) * s(pi * y) + a2 * c(pi * x) * s(pi * y),
                a1 * c(pi * x) * c(pi * y) + a2 * s(pi * x) * c(pi * y))

    P = elastic_sipg(N, lam=lam, mu=mu, omega=omega)
    elem, xy, area = P.meta["elem"], P.meta["xy"], P.meta["area"]
    ne = elem.shape[0]
    X = xy[elem]
    xi, eta, wt = _gauss_triangle(5)
    lam_b = np.stack([1 - xi - eta, xi, eta])                              # [3, nq] barycentric = basis
    pts = X[:, 0, None, :] + xi[None, :, None] * (X[:, 1] - X[:, 0])[:, None] + eta[None, :, None] * (X[:, 2] - X[:, 0])[:, None]
    w = 2 * area[:, None] * wt[None]                                      # [ne, nq]
    F = np.stack(f(pts[..., 0], pts[..., 1]), axis=-1)                     # [ne, nq, 2]
    b = np.einsum("aq,eq,eqc->eac", lam_b, w, F).astype(np.complex128)
    # boundary edges (edges of one element only)
    loc = [(0, 1), (1, 2), (2, 0)]
    cnt = {}
    for e in range(ne):
        for a0, a1 in loc:
            k = tuple(sorted((elem[e, a0], elem[e, a1])))
            cnt[k] = cnt.get(k, 0) + 1
    tq, wq = np.polynomial.legendre.leggauss(4)
    tq, wq = 0.5 * (tq + 1), 0.5 * wq
    cp, cs = np.sqrt(lam + 2 * mu), np.sqrt(mu)
    for e in range(ne):
        for a0, a1 in loc:
            if cnt[tuple(sorted((elem[e, a0], elem[e, a1])))] != 1:
                continue
            P0, P1 = xy[elem[e, a0]], xy[elem[e, a1]]
            L = np.linalg.norm(P1 - P0)
            t = (P1 - P0) / L
            mid = 0.5 * (P0 + P1)
            n = np.array([-1.0 if mid[0] < 1e-12 else 1.0 if mid[0] > 1 - 1e-12 else 0.0,
                          -1.0 if mid[1] < 1e-12 else 1.0 if mid[1] > 1 - 1e-12 else 0.0])
            assert abs(n @ t) < 1e-12 and abs(np.linalg.norm(n) - 1) < 1e-12
            q = P0[None] + tq[:, None] * (P1 - P0)[None]
            (ux, uy), ((a, bb), (cc, d)) = u(q[:, 0], q[:, 1]), grad(q[:, 0], q[:, 1])
            div = a + d
            sig = np.array([[lam * div + 2 * mu * a, mu * (bb + cc)], [mu * (bb + cc), lam * div + 2 * mu * d]])
            uq = np.stack([ux, uy])                                         # [2, nq]
            Cmat = cp * np.outer(n, n) + cs * np.outer(t, t)
            g = np.einsum("ijq,j->iq", sig, n) - 1j * omega * (Cmat @ uq)   # [2, nq]
            for a_loc, phi in ((a0, 1 - tq), (a1, tq)):
                b[e, a_loc] += L * np.einsum("q,q,cq->c", wq, phi, g)
    uh = spla.spsolve(P.A.tocsc(), b.reshape(-1)).reshape(ne, 3, 2)
    Uh = np.einsum("aq,eac->eqc", lam_b, uh)
    Ue = np.stack(u(pts[..., 0], pts[..., 1]), axis=-1)
    err = np.sqrt(np.sum(w[..., None] * np.abs(Uh - Ue) ** 2))
    ref = np.sqrt(np.sum(w[..., None] * np.abs(Ue) ** 2))
    return err / ref


def test_manufactured_solution_converges_at_second_order():
    """P1 SIPG converges like h^2 in L2 for a smooth solution (the volume,
    consistency, penalty and absorbing terms all enter: a wrong sign or a
    dropped term stalls the error)."""
    errs = [_manufactured_error(N, 2.0, 1.0, 3.0) for N in (8, 16, 32, 64)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert errs[-1] < 2e-3, errs
    assert rates[0] > 1.5 and rates[1] > 1.8 and rates[2] > 1.9, (errs, rates)
