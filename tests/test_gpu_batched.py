"""Batched workload on the GPU: a forest of independent problems
(ndhss_build_tree_batched) factored in one call, the 32-column apply
(ndhss_apply_multi) and the lockstep GMRES (ndhss_gmres_batched), all through
the C ABI, against the FP64 oracle run problem by problem.

Tolerances.  FP64 fronts: the multi apply sums each tile in another order than
the one-column apply and the oracle; normwise relative differences stay at a
few u64 x kappa of the fronts, checked at 1e-10.  FP32 fronts: u32 x kappa,
checked at 1e-4 against the one-column FP32 apply (same factor, other order)
and at 2e-3 against the FP64 oracle.  Solutions: true relative residual 1e-8
per system; the forward error against a sparse direct solve is at most
cond(A) x 1e-8 and is checked at 1e-5 on these well-conditioned problems.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from ndhss_inputs import helmholtz_batch, poisson_dirichlet
from oracle.frontal import apply_inverse, factor_dense
from oracle.gmres import gmres as oracle_gmres
from oracle.tree import build_tree
from closeness import rel as _rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LEAF = 32


@pytest.fixture(scope="module")
def nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_07791_gb300 import build, ndhss
    build.build()
    ndhss.load()
    return ndhss


@pytest.fixture(scope="module")
def batch(nd):
    """Five problems of uneven size (grids 12..40 cells, wave speed on 4 x 4
    macro blocks), 6 right-hand sides each."""
    probs = helmholtz_batch(5, seed=3, nmin=12, nmax=40, nsrc=6, mb=4)
    tree = nd.ndhss_build_tree_batched([(P.coords, P.A.indptr, P.A.indices) for P in probs], LEAF)
    A, off = nd.batch_csr([P.A for P in probs])
    M = nd.DeviceCSR(A)
    facs = [factor_dense(build_tree(P.coords, P.A.indptr, P.A.indices, LEAF), P.A) for P in probs]
    return dict(probs=probs, tree=tree, A=A, off=off, M=M, facs=facs)


def _factor(nd, tree, M, prec, hss_levels=-1):
    f = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, nd.make_factor_opts(prec=prec, hss_levels=hss_levels))
    torch.cuda.synchronize()
    return f


def _rand(n, k, seed, cplx=True):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, k))
    if cplx:
        X = X + 1j * rng.standard_normal((n, k))
    return X


@pytest.mark.parametrize("prec,tol_o", [(0, 1e-10), (1, 2e-3)])
def test_forest_multi_apply_is_each_problems_oracle_apply(nd, batch, prec, tol_o):
    f = _factor(nd, batch["tree"], batch["M"], prec)
    n, off = batch["A"].shape[0], batch["off"]
    for k in (32, 7, 1):
        X = _rand(n, k, 10 + k)
        Xd = torch.from_numpy(X).cuda().contiguous()
        Yd = torch.empty_like(Xd)
        nd.ndhss_apply_multi(f, Xd, Yd)
        Y = Yd.cpu().numpy()
        for s, fac in enumerate(batch["facs"]):
            a, b = off[s], off[s + 1]
            Yo = apply_inverse(fac, X[a:b])
            assert _rel(Y[a:b], Yo) <= tol_o, (k, s, _rel(Y[a:b], Yo))
    # the one-column dataflow apply on the same forest factor agrees
    X = _rand(n, 3, 5)
    Xd = torch.from_numpy(X).cuda().contiguous()
    Yd = torch.empty_like(Xd)
    nd.ndhss_apply_multi(f, Xd, Yd)
    for c in range(3):
        x1 = torch.from_numpy(np.ascontiguousarray(X[:, c])).cuda()
        y1 = torch.empty_like(x1)
        nd.ndhss_apply(f, x1, y1)
        assert _rel(Yd[:, c].cpu().numpy(), y1.cpu().numpy()) <= (1e-12 if prec == 0 else 1e-4)


def test_multi_apply_single_problem_real_and_ragged(nd):
    """A real (Poisson) factor: float64 vectors, FP64 and FP32 fronts."""
    P = poisson_dirichlet(37, seed=3)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    fac = factor_dense(T, P.A)
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    M = nd.DeviceCSR(P.A)
    X = _rand(P.n, 32, 1, cplx=False)
    Yo = apply_inverse(fac, X)
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        f = _factor(nd, tree, M, prec)
        Xd = torch.from_numpy(X).cuda().contiguous()
        Yd = torch.empty_like(Xd)
        nd.ndhss_apply_multi(f, Xd, Yd)
        assert _rel(Yd.cpu().numpy(), Yo) <= tol


def test_multi_apply_argument_checks(nd, batch):
    f = _factor(nd, batch["tree"], batch["M"], 1)
    n = batch["A"].shape[0]
    X = torch.zeros((n, 33), dtype=torch.complex128, device="cuda")
    with pytest.raises(nd.NdhssError, match="INVALID_ARG"):
        nd.ndhss_apply_multi(f, X, torch.empty_like(X))
    # ULV factorizations are applied column by column only
    P = helmholtz_batch(1, seed=9, nmin=64, nmax=64, nsrc=1)[0]
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 32)
    M = nd.DeviceCSR(P.A)
    fu = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals,
                         nd.make_factor_opts(prec=1, hss_levels=2, ulv=True))
    X = torch.zeros((P.n, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(nd.NdhssError, match="column"):
        nd.ndhss_apply_multi(fu, X, torch.empty_like(X))


@pytest.mark.parametrize("prec,tol_o,tol_1", [(0, 1e-4, 1e-12), (1, 1e-3, 1e-4)])
def test_multi_apply_compressed_factor(nd, prec, tol_o, tol_1):
    """Compressed fronts (low-rank R and L above the switching level): the
    32-column apply against the oracle's compressed preconditioner
    (apply_compressed, same Philox streams; the tolerance of the one-vector
    compressed apply) and column by column against ndhss_apply."""
    from oracle.hss import apply_compressed, factor_compressed
    P = helmholtz_batch(1, seed=9, nmin=96, nmax=96, nsrc=1)[0]
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 32)
    fac = factor_compressed(T, P.A, hss_levels=3, eps=1e-6, beta=64, k0=32, r=16, seed=11)
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 32)
    M = nd.DeviceCSR(P.A)
    f = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals,
                        nd.make_factor_opts(prec=prec, hss_levels=3, eps_hss=1e-6, beta=64, k0=32, r=16, seed=11))
    assert nd.ndhss_factor_stats_get(f)["kmax"] > 0
    for k in (32, 5):
        X = _rand(P.n, k, 20 + k)
        Xd = torch.from_numpy(X).cuda().contiguous()
        Yd = torch.empty_like(Xd)
        nd.ndhss_apply_multi(f, Xd, Yd)
        Y = Yd.cpu().numpy()
        assert _rel(Y, apply_compressed(fac, X)) <= tol_o, _rel(Y, apply_compressed(fac, X))
        for c in range(min(k, 3)):
            x1 = torch.from_numpy(np.ascontiguousarray(X[:, c])).cuda()
            y1 = torch.empty_like(x1)
            nd.ndhss_apply(f, x1, y1)
            assert _rel(Y[:, c], y1.cpu().numpy()) <= tol_1, (c, _rel(Y[:, c], y1.cpu().numpy()))


@pytest.mark.parametrize("prec", [0, 1])
def test_gmres_batched_solves_every_system(nd, batch, prec):
    f = _factor(nd, batch["tree"], batch["M"], prec)
    probs, off, M = batch["probs"], batch["off"], batch["M"]
    n = batch["A"].shape[0]
    nrhs = 6
    Bh = np.zeros((nrhs, n), dtype=np.complex128)
    for s, P in enumerate(probs):
        Bh[:, off[s]:off[s + 1]] = P.b.T
    Bh[2, off[1]:off[2]] = 0.0                      # one zero right-hand side: x = 0, converged at once
    B = torch.from_numpy(Bh).cuda()
    X = torch.zeros_like(B)
    st = nd.ndhss_gmres_batched(f, M.rowptr, M.col, M.vals, off, B, X, tol=1e-8)
    Xh = X.cpu().numpy()
    for s, P in enumerate(probs):
        lu = spla.splu(P.A.tocsc())
        for c in range(nrhs):
            S = st[s][c]
            assert S["converged"] and S["true_relres"] <= 1e-8, (s, c, S)
            xs = Xh[c, off[s]:off[s + 1]]
            bs = Bh[c, off[s]:off[s + 1]]
            if not np.any(bs):
                assert S["iters"] == 0 and not np.any(xs)
                continue
            assert _rel(xs, lu.solve(bs)) <= 1e-5, (s, c)
            assert np.linalg.norm(bs - P.A @ xs) <= 1.01e-8 * np.linalg.norm(bs)
    # iteration counts: the oracle GMRES with the oracle's exact dense factor
    # on one system per problem, within +2 (FP64) / the FP32 bound of the
    # one-system path
    for s, P in enumerate(probs):
        ro = oracle_gmres(P.A, P.b[:, 0], lambda v: apply_inverse(batch["facs"][s], v), tol=1e-8)
        slack = 2 if prec == 0 else 4
        assert st[s][0]["iters"] <= ro.iters + slack, (s, st[s][0]["iters"], ro.iters)


def test_gmres_batched_matches_one_system_solver(nd, batch):
    """On the same forest factor, the lockstep solver and ndhss_gmres take
    the same number of steps per system (same arithmetic, other reduction
    order)."""
    f = _factor(nd, batch["tree"], batch["M"], 0)
    probs, off, M = batch["probs"], batch["off"], batch["M"]
    n = batch["A"].shape[0]
    Bh = np.zeros((2, n), dtype=np.complex128)
    for s, P in enumerate(probs):
        Bh[:, off[s]:off[s + 1]] = P.b[:, :2].T
    B = torch.from_numpy(Bh).cuda()
    X = torch.zeros_like(B)
    st = nd.ndhss_gmres_batched(f, M.rowptr, M.col, M.vals, off, B, X, tol=1e-8)
    for s in range(len(probs)):
        b1 = np.zeros(n, dtype=np.complex128)
        b1[off[s]:off[s + 1]] = Bh[0, off[s]:off[s + 1]]
        bd = torch.from_numpy(b1).cuda()
        x1 = torch.zeros_like(bd)
        s1 = nd.ndhss_gmres(f, M.rowptr, M.col, M.vals, bd, x1, tol=1e-8)
        assert abs(s1["iters"] - st[s][0]["iters"]) <= 1, (s, s1["iters"], st[s][0]["iters"])
        assert not np.any(x1.cpu().numpy()[np.r_[0:off[s], off[s + 1]:n]])


def test_gmres_batched_argument_checks(nd, batch):
    f = _factor(nd, batch["tree"], batch["M"], 1)
    M, off = batch["M"], batch["off"]
    n = batch["A"].shape[0]
    B = torch.zeros((2, n), dtype=torch.complex128, device="cuda")
    X = torch.zeros_like(B)
    bad = off.copy()
    bad[-1] -= 1
    with pytest.raises(nd.NdhssError, match="sys_off"):
        nd.ndhss_gmres_batched(f, M.rowptr, M.col, M.vals, bad, B, X)
    with pytest.raises(nd.NdhssError, match="restart"):
        nd.ndhss_gmres_batched(f, M.rowptr, M.col, M.vals, off, B, X, restart=40)


def test_level_wider_than_the_grid_limit(nd):
    """70000 single-front problems: one level holds more fronts than a grid's
    y / z dimension (65535), so the factorization runs it in chunks."""
    P = poisson_dirichlet(4)                        # 9 unknowns, one leaf
    S = 70000
    tree = nd.ndhss_build_tree_batched([(P.coords, P.A.indptr, P.A.indices)] * S, 64)
    assert tree.nnodes == S and tree.depth == 0
    A, off = nd.batch_csr([P.A] * S)
    M = nd.DeviceCSR(A)
    f = _factor(nd, tree, M, 0)
    x = _rand(A.shape[0], 1, 3, cplx=False)[:, 0]
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    nd.ndhss_apply(f, xd, yd)
    want = np.linalg.solve(P.A.toarray()[None], x.reshape(S, 9, 1))[..., 0].ravel()
    assert _rel(yd.cpu().numpy(), want) <= 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_gmres_batched_real_problems(nd, prec):
    """float64 vectors: a forest of three Poisson problems of different sizes,
    five random right-hand sides each, against sparse direct solves."""
    probs = [poisson_dirichlet(N, seed=N) for N in (17, 30, 9)]
    tree = nd.ndhss_build_tree_batched([(P.coords, P.A.indptr, P.A.indices) for P in probs], 32)
    A, off = nd.batch_csr([P.A for P in probs])
    M = nd.DeviceCSR(A)
    assert M.vtype == 0
    f = _factor(nd, tree, M, prec)
    n = A.shape[0]
    Bh = np.ascontiguousarray(_rand(n, 5, 21, cplx=False).T)
    B = torch.from_numpy(Bh).cuda()
    X = torch.zeros_like(B)
    st = nd.ndhss_gmres_batched(f, M.rowptr, M.col, M.vals, off, B, X, tol=1e-10)
    Xh = X.cpu().numpy()
    for s, P in enumerate(probs):
        lu = spla.splu(P.A.tocsc())
        for c in range(5):
            assert st[s][c]["converged"] and st[s][c]["true_relres"] <= 1e-10
            a, b = off[s], off[s + 1]
            assert _rel(Xh[c, a:b], lu.solve(Bh[c, a:b])) <= 1e-8


@pytest.mark.parametrize("prec", [0, 1])
def test_gmres_batched_compressed_forest(nd, batch, prec):
    """The lockstep GMRES on a compressed forest factor (the 32-column apply
    with low-rank tiles): every system to a float64 true residual of 1e-8,
    solutions within 1e-5 of a direct solve."""
    tree, M, probs, off = batch["tree"], batch["M"], batch["probs"], batch["off"]
    f = _factor(nd, tree, M, prec, hss_levels=2)
    assert nd.ndhss_factor_stats_get(f)["kmax"] > 0          # low-rank tiles are exercised
    n = batch["A"].shape[0]
    nrhs = 4
    Bh = np.zeros((nrhs, n), dtype=np.complex128)
    for s, P in enumerate(probs):
        Bh[:, off[s]:off[s + 1]] = P.b[:, :nrhs].T
    B = torch.from_numpy(Bh).cuda()
    X = torch.zeros_like(B)
    st = nd.ndhss_gmres_batched(f, M.rowptr, M.col, M.vals, off, B, X, tol=1e-8)
    Xh = X.cpu().numpy()
    for s, P in enumerate(probs):
        lu = spla.splu(P.A.tocsc())
        for c in range(nrhs):
            S = st[s][c]
            assert S["converged"] and S["true_relres"] <= 1e-8, (s, c, S)
            xs, bs = Xh[c, off[s]:off[s + 1]], Bh[c, off[s]:off[s + 1]]
            assert _rel(xs, lu.solve(bs)) <= 1e-5, (s, c)


@pytest.mark.parametrize("tiles", ["64,64,64,64", "32,64,32,64"])
def test_multi_apply_tile_shapes_agree(nd, batch, tiles, monkeypatch):
    """Both tile shapes of the 32-column apply (chosen per front-size bucket
    by the autotuned table, overridden here) give the same result up to the
    summation order of their K chunks (the same chunks: bit-identical)."""
    f64 = _factor(nd, batch["tree"], batch["M"], 1)
    n = batch["A"].shape[0]
    X = _rand(n, 32, 77)
    Xd = torch.from_numpy(X).cuda().contiguous()
    Ya = torch.empty_like(Xd)
    nd.ndhss_apply_multi(f64, Xd, Ya)
    monkeypatch.setenv("NDHSS_MAPPLY_TILES", tiles)
    f32 = _factor(nd, batch["tree"], batch["M"], 1)
    Yb = torch.empty_like(Xd)
    nd.ndhss_apply_multi(f32, Xd, Yb)
    assert torch.equal(Ya, Yb)
