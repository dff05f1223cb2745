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


def test_macro_generator_quadratic_forms_pin_the_coefficients():
    """helmholtz_macro on rectangular cells with wave speed piecewise constant
    on macro blocks (the batched workload's generator), pinned by exact
    quadratic forms: 1^T A 1 = -w^2 int c^-2 - i w int_{boundary} c^-1, and for
    the interpolant of u = x (exact in P1) u^T A u = int |grad x|^2 -
    w^2 int x^2 c^-2 - i w int_{boundary} x^2 c^-1, cell by cell."""
    from ndhss_inputs.fem import helmholtz_macro
    rng = np.random.default_rng(0)
    Nx, Ny, mb = 24, 17, 4
    cb = rng.uniform(1.0, 3.0, (mb, mb))
    P = helmholtz_macro(Nx, Ny, cb, nsrc=2)
    w, xy, A = P.meta["omega"], P.meta["xy"], P.A
    assert abs(w - 2 * np.pi / (10.0 / min(Nx, Ny))) <= 1e-12 * w        # 10 points per wavelength at c = 1
    hx, hy = 1.0 / Nx, 1.0 / Ny
    ia = np.arange(Nx)[:, None]
    ib = np.arange(Ny)[None, :]
    c = cb[ia * mb // Nx, ib * mb // Ny]                                  # [Nx, Ny] per cell
    one = np.ones(A.shape[0])
    mass = (hx * hy / c ** 2).sum()
    bnd = (hx / c[:, 0]).sum() + (hx / c[:, -1]).sum() + (hy / c[0, :]).sum() + (hy / c[-1, :]).sum()
    ref = -w * w * mass - 1j * w * bnd
    assert abs(one @ (A @ one) - ref) <= 1e-10 * abs(ref)
    u = xy[:, 0].astype(np.complex128)
    x2 = ((np.arange(Nx) + 1.0) ** 3 - np.arange(Nx) ** 3) * hx ** 3 / 3.0     # int x^2 over each cell column
    vol = (x2[:, None] * hy / c ** 2).sum()
    bnd2 = (x2 / c[:, 0]).sum() + (x2 / c[:, -1]).sum() + (hy / c[-1, :]).sum()   # x = 0 on the left side
    ref2 = 1.0 - w * w * vol - 1j * w * bnd2
    assert abs(u @ (A @ u) - ref2) <= 1e-9 * abs(ref2)
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()
    assert P.b.shape == (A.shape[0], 2)


def test_batch_generator_recipe():
    from ndhss_inputs.fem import helmholtz_batch
    probs = helmholtz_batch(6, seed=3, nsrc=4)
    again = helmholtz_batch(6, seed=3, nsrc=4)
    for P, Q in zip(probs, again):
        Nx, Ny = P.meta["Nx"], P.meta["Ny"]
        assert 64 <= Nx <= 256 and 64 <= Ny <= 256
        cb = P.meta["c_blocks"]
        assert cb.shape == (8, 8) and cb.min() >= 1.0 and cb.max() <= 3.0
        assert P.A.shape[0] == (Nx + 1) * (Ny + 1) and P.b.shape == (P.A.shape[0], 4)
        src = P.meta["sources"]
        assert src.min() >= 0.1 and src.max() <= 0.9
        assert (P.A != Q.A).nnz == 0 and np.array_equal(P.b, Q.b)      # seeded
    assert len({(P.meta["Nx"], P.meta["Ny"]) for P in probs}) > 1     # uneven sizes


def test_block_slowness_generator_quadratic_form():
    """helmholtz_blocks (the adjoint workload's generator): squared slowness m
    piecewise constant on nb x nb blocks enters as -k^2 m in the mass term and
    -i k sqrt(m) on the boundary: 1^T A 1 = -k^2 int m - i k int_{boundary} sqrt(m)."""
    from ndhss_inputs.fem import helmholtz_blocks
    rng = np.random.default_rng(1)
    N, nb, k = 20, 4, 7.0
    m = rng.uniform(0.3, 1.0, (nb, nb))
    P = helmholtz_blocks(N, k, m)
    A = P.A
    h = 1.0 / N
    ia = np.arange(N)
    mc = m[ia[:, None] * nb // N, ia[None, :] * nb // N]                 # per cell (a, b)
    one = np.ones(A.shape[0])
    ref = -k * k * (h * h * mc).sum() - 1j * k * h * (np.sqrt(mc[:, 0]).sum() + np.sqrt(mc[:, -1]).sum()
                                                       + np.sqrt(mc[0, :]).sum() + np.sqrt(mc[-1, :]).sum())
    assert abs(one @ (A @ one) - ref) <= 1e-10 * abs(ref)
