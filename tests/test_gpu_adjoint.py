"""Gradients through the GPU solve (autograd Function with the adjoint
solve on the same factor) against the oracle's adjoint gradient (sparse
direct solves), central finite differences of the misfit, and the
right-hand-side gradient A^{-H} g."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from ndhss_inputs.fem import helmholtz_blocks
from oracle.adjoint import misfit_and_gradient

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_07791_gb300 import build, ndhss
    build.build()
    ndhss.load()
    return ndhss


def _problem(N=24, nb=4, k=10.0, seed=0):
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.3, 1.0, (nb, nb))
    src = np.array([[0.3, 0.2], [0.7, 0.25]])
    P = helmholtz_blocks(N, k, m, src_xy=src)
    rec = np.nonzero(np.abs(P.meta["xy"][:, 1] - 0.75) < 1e-12)[0][::2]
    Pt = helmholtz_blocks(N, k, m + 0.05 * rng.uniform(-1, 1, m.shape), src_xy=src)
    d = np.stack([spla.spsolve(Pt.A.tocsc(), Pt.b[:, s])[rec] for s in range(2)], axis=1)
    return P, m, src, rec, d, k, N


def _model(nd, P, k, N, src, prec, hss_levels):
    from paper_2105_07791_gb300.autograd import HelmholtzBlockModel
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    nb = P.meta["nb"]
    opts = nd.make_factor_opts(prec=prec, hss_levels=hss_levels)
    return HelmholtzBlockModel(tree, lambda mb: helmholtz_blocks(N, k, mb.reshape(nb, nb), src_xy=src).A, k,
                               P.meta["elem"], P.meta["Me"], P.meta["eblk"], P.meta["edges"], P.meta["Ee"],
                               P.meta["edge_blk"], nb * nb, opts=opts, tol=1e-11)


def _misfit(nd, model, m_t, B, rec, d):
    from paper_2105_07791_gb300.autograd import HelmholtzSolve
    X = HelmholtzSolve.apply(m_t, B, model)
    r = X[torch.from_numpy(rec).cuda()] - torch.from_numpy(d).cuda()
    return 0.5 * (r.abs() ** 2).sum(), X


@pytest.mark.parametrize("prec,hss_levels", [(0, -1), (1, -1), (1, 2)])
def test_coefficient_gradient_matches_oracle_and_differences(nd, prec, hss_levels):
    P, m, src, rec, d, k, N = _problem()
    model = _model(nd, P, k, N, src, prec, hss_levels)
    m_t = torch.tensor(m.ravel(), dtype=torch.float64, requires_grad=True)
    B = torch.from_numpy(np.ascontiguousarray(P.b)).cuda().requires_grad_(True)
    J, X = _misfit(nd, model, m_t, B, rec, d)
    J.backward()
    g = m_t.grad.numpy()
    Jo, go = misfit_and_gradient(P, rec, d)
    assert abs(J.item() - Jo) <= 1e-8 * Jo
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)
    # right-hand-side gradient: A^{-H} R^T (R x - d), column by column
    Xh = X.detach().cpu().numpy()
    for s in range(2):
        gs = np.zeros(P.A.shape[0], dtype=np.complex128)
        gs[rec] = Xh[rec, s] - d[:, s]
        lam = np.conj(spla.spsolve(P.A.tocsc(), np.conj(gs)))
        gb = B.grad[:, s].cpu().numpy()
        assert np.linalg.norm(gb - lam) <= 1e-6 * np.linalg.norm(lam)
    # central differences of the GPU misfit on a boundary and an interior block
    for j in (0, 5):
        h = 1e-4 * m.ravel()[j]
        vals = []
        for sgn in (1, -1):
            mp = m.ravel().copy()
            mp[j] += sgn * h
            with torch.no_grad():
                Jp, _ = _misfit(nd, model, torch.tensor(mp), B.detach(), rec, d)
            vals.append(Jp.item())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-5 * np.abs(go).max(), (j, fd, g[j])


@pytest.mark.slow
def test_c5_sized_gradient_matches_oracle():
    """The adjoint workload's full size: P1 on 512 x 512 cells, k = 80,
    squared slowness on 32 x 32 blocks ~ U[0.3, 1], 16 sources and receivers
    on the line y = 0.9, data from a seeded perturbed model; compressed FP32
    factor with float64 GMRES.  Gradient of all 1024 blocks against the
    oracle's adjoint gradient (sparse direct) to 1e-5."""
    import time
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_07791_gb300 import build, ndhss
    build.build()
    ndhss.load()
    N, k, nb, ns = 512, 80.0, 32, 16
    rng = np.random.default_rng(5)
    m = rng.uniform(0.3, 1.0, (nb, nb))
    y_line = round(0.9 * N) / N
    src = np.stack([(np.arange(ns) + 0.5) / ns, np.full(ns, y_line)], axis=1)
    P = helmholtz_blocks(N, k, m, src_xy=src)
    xy = P.meta["xy"]
    rec = np.array([np.argmin((xy[:, 0] - x) ** 2 + (xy[:, 1] - y_line) ** 2) for x in src[:, 0]])
    Pt = helmholtz_blocks(N, k, m + 0.05 * rng.uniform(-1, 1, m.shape), src_xy=src)
    lu = spla.splu(Pt.A.tocsc())
    d = np.stack([lu.solve(Pt.b[:, s])[rec] for s in range(ns)], axis=1)
    model = _model(ndhss, P, k, N, src, 1, 4)
    t_asm = [0.0]
    assemble = model.assemble

    def timed_assemble(mb):
        t = time.time()
        A = assemble(mb)
        t_asm[0] += time.time() - t
        return A

    model.assemble = timed_assemble
    m_t = torch.tensor(m.ravel(), dtype=torch.float64, requires_grad=True)
    B = torch.from_numpy(np.ascontiguousarray(P.b)).cuda()
    for rep in range(2):  # the first pass also pays one-time set-up (memory pool, module load)
        m_t.grad = None
        t_asm[0] = 0.0
        torch.cuda.synchronize()
        t0 = time.time()
        J, X = _misfit(ndhss, model, m_t, B, rec, d)
        J.backward()
        torch.cuda.synchronize()
        t_gpu = time.time() - t0
    t0 = time.time()
    Jo, go = misfit_and_gradient(P, rec, d)
    t_cpu = time.time() - t0
    g = m_t.grad.numpy()
    print(f"C5 gradient: {t_gpu:.2f} s on the GPU path, of which {t_asm[0]:.2f} s host assembly of A(m); "
          f"oracle (sparse direct, A given) {t_cpu:.2f} s")
    assert abs(J.item() - Jo) <= 1e-7 * Jo
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


@pytest.mark.parametrize("host", [False, True])
def test_conj_transpose_solves_the_adjoint_system(nd, host):
    """ndhss_gmres with conj_transpose solves A^H x = b on the factor of A
    (device and host buffers); the caller's b is left as it was."""
    P = _problem()[0]
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    M = nd.DeviceCSR(P.A)
    f = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, nd.make_factor_opts(prec=nd.NDHSS_FP32, hss_levels=2))
    rng = np.random.default_rng(4)
    g = rng.standard_normal(P.n) + 1j * rng.standard_normal(P.n)
    if host:
        b, x = g.copy(), np.zeros_like(g)
    else:
        b = torch.from_numpy(g).cuda()
        x = torch.zeros_like(b)
    st = nd.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x, tol=1e-10, conj_transpose=True)
    xh = x if host else x.cpu().numpy()
    bh = b if host else b.cpu().numpy()
    assert st["converged"] and st["true_relres"] <= 1e-10
    assert np.array_equal(bh, g)
    AH = P.A.conj().T.tocsr()
    assert np.linalg.norm(AH @ xh - g) <= 1e-9 * np.linalg.norm(g)
    # the plain solve on the same factor is a different system
    y = np.zeros_like(g)
    nd.ndhss_gmres(f, M.rowptr, M.col, M.vals, g.copy(), y, tol=1e-10)
    assert np.linalg.norm(P.A @ y - g) <= 1e-9 * np.linalg.norm(g)
    assert np.linalg.norm(y - xh) > 1e-3 * np.linalg.norm(y)


def test_conj_transpose_changes_nothing_for_a_real_matrix(nd):
    from ndhss_inputs import poisson_dirichlet
    P = poisson_dirichlet(40, p=1, seed=0)
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    M = nd.DeviceCSR(P.A)
    f = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, nd.make_factor_opts(prec=nd.NDHSS_FP32))
    b = torch.from_numpy(np.ascontiguousarray(P.b if P.b.ndim == 1 else P.b[:, 0])).cuda()
    x0, x1 = torch.zeros_like(b), torch.zeros_like(b)
    nd.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x0, tol=1e-10)
    nd.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x1, tol=1e-10, conj_transpose=True)
    assert torch.equal(x0, x1)
