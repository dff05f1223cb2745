"""Pins of the oracle's adjoint gradient (misfit J(m) of a Helmholtz problem
with squared slowness on blocks): central finite differences of J, and the
linearity of dJ/dm in the misfit's data residual."""
import numpy as np

from ndhss_inputs.fem import helmholtz_blocks
from oracle.adjoint import misfit_and_gradient


def _setup(N=16, nb=4, k=8.0, seed=0):
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.3, 1.0, (nb, nb))
    src = np.array([[0.3, 0.2], [0.7, 0.25]])
    P = helmholtz_blocks(N, k, m, src_xy=src)
    xy = P.meta["xy"]
    rec = np.nonzero(np.abs(xy[:, 1] - 0.75) < 1e-12)[0][::2]
    Pt = helmholtz_blocks(N, k, m + 0.05 * rng.uniform(-1, 1, m.shape), src_xy=src)
    import scipy.sparse.linalg as spla
    d = np.stack([spla.spsolve(Pt.A.tocsc(), Pt.b[:, s])[rec] for s in range(2)], axis=1)
    return P, m, src, rec, d, k, N


def test_adjoint_gradient_matches_central_differences():
    P, m, src, rec, d, k, N = _setup()
    J, g = misfit_and_gradient(P, rec, d)
    assert J > 0
    for j in (0, 5, 10, 15):                      # boundary and interior blocks
        h = 1e-5 * m.ravel()[j]
        mp, mm = m.copy(), m.copy()
        mp.ravel()[j] += h
        mm.ravel()[j] -= h
        Jp, _ = misfit_and_gradient(helmholtz_blocks(N, k, mp, src_xy=src), rec, d)
        Jm, _ = misfit_and_gradient(helmholtz_blocks(N, k, mm, src_xy=src), rec, d)
        fd = (Jp - Jm) / (2 * h)
        assert abs(g[j] - fd) <= 1e-6 * np.abs(g).max(), (j, g[j], fd)


def test_gradient_vanishes_at_the_true_model():
    """With data from the same model the residual and therefore the gradient are zero."""
    P, m, src, rec, _, k, N = _setup()
    import scipy.sparse.linalg as spla
    d = np.stack([spla.spsolve(P.A.tocsc(), P.b[:, s])[rec] for s in range(2)], axis=1)
    J, g = misfit_and_gradient(P, rec, d)
    assert J < 1e-20 and np.abs(g).max() < 1e-12
