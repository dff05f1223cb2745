"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances.  FP64 fronts: a block of the factor is a rational function of the
front entries computed by a different (blocked Gauss-Jordan) elimination order
than the oracle's LU; its normwise relative difference is bounded by
~ m * u64 * kappa(A_ii) and checked at 1e-9.  FP32 fronts: u32 = 6e-8, the same
bound with front conditioning up to ~1e3 gives ~1e-3 normwise for the blocks;
the end-to-end solution is refined by float64 GMRES to a true relative
residual of 1e-8 either way.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from ndhss_inputs import helmholtz_impedance, poisson_dirichlet
from oracle.frontal import apply_inverse, factor_dense
from oracle.gmres import gmres as oracle_gmres
from oracle.tree import build_tree
from closeness import rel as _rel

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


CASES = {
    "c1_poisson_p1_64": lambda: (poisson_dirichlet(64), 64),
    "helm_p2_24_k12": lambda: (helmholtz_impedance(24, 2, 12.0, seed=1), 64),
    "helm_p1_45_leaf16": lambda: (helmholtz_impedance(45, 1, 9.0, seed=2), 16),
    "poisson_p2_21_leaf32": lambda: (poisson_dirichlet(21, p=2, seed=5), 32),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, nd):
    P, leaf = CASES[request.param]()
    T = build_tree(P.coords, P.A.indptr, P.A.indices, leaf)
    fac = factor_dense(T, P.A)
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, leaf)
    M = nd.DeviceCSR(P.A)
    return dict(name=request.param, P=P, T=T, fac=fac, tree=tree, M=M)


def _gpu_factor(nd, c, prec, panel=0):
    M = c["M"]
    f = nd.ndhss_factor(c["tree"], M.vtype, M.rowptr, M.col, M.vals, nd.make_factor_opts(prec=prec, panel=panel))
    torch.cuda.synchronize()
    return f


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-3), (2, 5e-2)])
def test_factor_blocks_match_oracle(nd, case, prec, tol):
    """FP64 to rounding; FP32 and the TF32 tensor-core update (10-bit
    mantissa products, FP32 accumulation) by their arithmetic's tolerance."""
    f = _gpu_factor(nd, case, prec)
    T, fac = case["T"], case["fac"]
    nodes = list(range(T.nnodes))
    if len(nodes) > 60:
        nodes = nodes[:: len(nodes) // 60] + [T.nnodes - 1]
    for s in nodes:
        mi, mb = int(T.node_info[s, 5]), int(T.node_info[s, 7])
        if mi == 0:
            continue
        X = nd.ndhss_factor_get_block(f, s, 0, mi, mb)
        Xo = np.linalg.inv(fac.Aii[s])
        assert _rel(X, Xo) <= tol * 10, (s, "Aii^-1", _rel(X, Xo))
        if mb:
            for which, ref in ((1, fac.R[s]), (2, fac.L[s]), (3, fac.S[s])):
                blk = nd.ndhss_factor_get_block(f, s, which, mi, mb)
                assert _rel(blk, ref) <= tol, (s, which, _rel(blk, ref))


@pytest.mark.parametrize("panel", [1, 4, 0])
def test_factor_independent_of_pivot_block_width(nd, case, panel):
    """Blocking is an implementation choice: every panel width gives the same S (FP64)."""
    f = _gpu_factor(nd, case, 0, panel=panel)
    T, fac = case["T"], case["fac"]
    s = int(np.argmax(T.f("m_b") * (T.f("m_i") > 0)))
    mi, mb = int(T.node_info[s, 5]), int(T.node_info[s, 7])
    assert _rel(nd.ndhss_factor_get_block(f, s, 3, mi, mb), fac.S[s]) <= 1e-9


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_apply_matches_oracle_and_direct_solve(nd, case, prec):
    P, fac = case["P"], case["fac"]
    f = _gpu_factor(nd, case, prec)
    b = P.b if P.b.ndim == 1 else P.b[:, 0]
    dt = torch.complex128 if np.iscomplexobj(b) or case["M"].vtype == 1 else torch.float64
    xb = torch.from_numpy(np.ascontiguousarray(b.astype(np.complex128 if dt == torch.complex128 else np.float64))).cuda()
    y = torch.empty_like(xb)
    nd.ndhss_apply(f, xb, y)
    torch.cuda.synchronize()
    yo = apply_inverse(fac, b)
    yd = spla.spsolve(P.A.tocsc(), b)
    # TF32 operands carry a 10-bit mantissa (unit roundoff 2^-11 ~ 4.9e-4), BF16
    # a 7-bit one (2^-8 ~ 3.9e-3); the fronts' condition numbers (~1e2 on C1)
    # scale that into the inverse
    tol = {0: 1e-10, 1: 1e-3, 2: 1e-1, 3: 2e-1}[prec]
    assert _rel(y.cpu().numpy(), yo) <= tol
    assert _rel(y.cpu().numpy(), yd) <= tol
    # host buffers through the same entry point
    yh = np.zeros_like(xb.cpu().numpy())
    nd.ndhss_apply(f, xb.cpu().numpy(), yh)
    assert np.array_equal(yh, y.cpu().numpy())


def test_spmv_matches_scipy(nd, case):
    P, M = case["P"], case["M"]
    rng = np.random.default_rng(7)
    x = rng.standard_normal(P.n)
    if M.vtype == 1:
        x = x + 1j * rng.standard_normal(P.n)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    nd.ndhss_spmv(P.n, M.vtype, M.rowptr, M.col, M.vals, xd, yd)
    torch.cuda.synchronize()
    ref = P.A @ x
    assert _rel(yd.cpu().numpy(), ref) <= 1e-14


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_gmres_solution_and_iterations(nd, case, prec):
    P, fac = case["P"], case["fac"]
    M = case["M"]
    f = _gpu_factor(nd, case, prec)
    b = P.b if P.b.ndim == 1 else P.b[:, 0]
    bd = torch.from_numpy(np.ascontiguousarray(b.astype(np.complex128 if M.vtype == 1 else np.float64))).cuda()
    xd = torch.zeros_like(bd)
    st = nd.ndhss_gmres(f, M.rowptr, M.col, M.vals, bd, xd, restart=30, maxit=300, tol=1e-8)
    x = xd.cpu().numpy()
    assert st["converged"] and st["true_relres"] <= 1e-8
    assert np.linalg.norm(b - P.A @ x) / np.linalg.norm(b) <= 1e-8
    ro = oracle_gmres(P.A, b, lambda v: apply_inverse(fac, v), tol=1e-8)
    if prec <= 1:
        assert st["iters"] <= ro.iters + 2, (st, ro.iters)
    else:
        # TF32 / BF16 operands leave a preconditioner accurate to ~1e-2 (10- / 7-bit
        # mantissas): the float64 restarts refine it, at a few more iterations than
        # the exact oracle factor needs
        assert st["iters"] <= ro.iters + (9 if prec == 2 else 12), (st, ro.iters)
    xdir = spla.spsolve(P.A.tocsc(), b)
    assert _rel(x, ro.x) <= (1e-8 if prec == 0 else 1e-6)
    assert _rel(x, xdir) <= (1e-8 if prec == 0 else 1e-6)


def test_single_leaf_and_tiny_problems(nd):
    """n <= leaf size (root is a leaf, m_b = 0) and a 1-DOF system."""
    for P, leaf in ((poisson_dirichlet(5), 64), (poisson_dirichlet(2), 4)):
        tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, leaf)
        M = nd.DeviceCSR(P.A)
        f = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals)
        xb = torch.from_numpy(P.b.copy()).cuda()
        y = torch.empty_like(xb)
        nd.ndhss_apply(f, xb, y)
        assert _rel(y.cpu().numpy(), spla.spsolve(P.A.tocsc(), P.b)) <= 1e-12


def test_singular_front_is_reported(nd):
    """A zero row/column makes A_ii singular: SINGULAR status, no fault."""
    P = poisson_dirichlet(12)
    A = P.A.tolil()
    A[5, :] = 0.0
    A[:, 5] = 0.0
    A = A.tocsr()
    # keep the structural pattern (explicit zeros) so the tree is unchanged
    A = P.A.copy()
    A.data[A.indptr[5]:A.indptr[6]] = 0.0
    A.data[A.indices == 5] = 0.0
    tree = nd.ndhss_build_tree(P.coords, A.indptr, A.indices, 16)
    M = nd.DeviceCSR(A)
    with pytest.raises(nd.NdhssError) as ei:
        nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals)
    assert ei.value.code == 3 and "node" in str(ei.value)
    # the context is still usable afterwards
    x = torch.ones(4, device="cuda")
    assert float(x.sum()) == 4.0
