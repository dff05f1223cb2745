"""Pins of the seeded FEM fixtures: sizes, symmetry and textbook convergence orders."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from ndhss_inputs import helmholtz_impedance, poisson_dirichlet


def test_poisson_c1_size_and_symmetry():
    P = poisson_dirichlet(64, seed=0)
    assert P.n == 63 * 63
    # 5-point couplings plus the structural (+1,+1) diagonal couplings, explicit zeros kept
    assert P.A.nnz == 27281
    assert abs(P.A - P.A.T).max() == 0.0
    assert P.coords.dtype == np.int32 and P.coords.min() == 1 and P.coords.max() == 63


def _nodal_order(errs):
    return np.log2(errs[:-1] / errs[1:])


@pytest.mark.parametrize("p,min_order", [(1, 1.8), (2, 2.7)])
def test_poisson_manufactured_order(p, min_order):
    """u = sin(pi x) sin(pi y): nodal error falls like h^(p+1) (Eq. 4.1, CG Pp)."""
    errs = []
    for N in (8, 16, 32):
        P = poisson_dirichlet(N, p=p, f=lambda x, y: 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y))
        u = spla.spsolve(P.A.tocsc(), P.b)
        xy = P.meta["xy"]
        ue = np.sin(np.pi * xy[:, 0]) * np.sin(np.pi * xy[:, 1])
        errs.append(np.abs(u - ue).max())
    assert np.all(_nodal_order(np.array(errs)) > min_order), errs


@pytest.mark.parametrize("p,min_order", [(1, 1.9), (2, 2.9)])
def test_helmholtz_plane_wave_order(p, min_order):
    """u = exp(i k d.x) with matching impedance data du/dn - i k u = g (Eq. 4.2)."""
    k, th = 4.0, 0.3
    d = np.array([np.cos(th), np.sin(th)])

    def g(x, y, nx, ny):
        u = np.exp(1j * k * (d[0] * x + d[1] * y))
        return 1j * k * (d[0] * nx + d[1] * ny) * u - 1j * k * u

    errs = []
    for N in (8, 16, 32):
        P = helmholtz_impedance(N, p, k, g=g)
        assert abs(P.A - P.A.T).max() <= 1e-14 * abs(P.A).max()     # complex symmetric
        u = spla.spsolve(P.A.tocsc(), P.b)
        xy = P.meta["xy"]
        ue = np.exp(1j * k * (xy @ d))
        # discrete L2 (RMS nodal) error: the max-norm carries an extra |log h| for P1
        errs.append(np.sqrt(np.mean(np.abs(u - ue) ** 2)))
    assert np.all(_nodal_order(np.array(errs)) > min_order), errs


def test_helmholtz_c2_shape():
    P = helmholtz_impedance(64, 2, 10.0, seed=3)
    assert P.n == 129 * 129 and P.A.dtype == np.complex128
    assert P.b.shape == (P.n,)
    assert P.coords.max() == 128
    # the source is a Gaussian of width 0.02 inside [0.1, 0.9]^2
    xs = P.meta["sources"][0]
    assert np.all((xs >= 0.1) & (xs <= 0.9))
