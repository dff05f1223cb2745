"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Every comparison bounds both the normwise and the entrywise relative
difference (tests/closeness.py).  The module runs the FP32-storage
precisions with NDHSS_TC_MIN_MI=16, so every level whose largest interior
block has 16 or more unknowns takes the two-level sweep with tensor-core
block exchanges; one test compares it with the rank-kb sweep on CUDA cores.

Tolerances.  A block of the factor is a rational function of the front
entries computed in another elimination order than the oracle's LU; its
relative difference is about c * kappa * u, u the unit roundoff of the
products.  FP64: u = 1.1e-16, checked at 1e-9.  FP32-accurate products
(NDHSS_FP32: two TF32 parts; NDHSS_FP32_BF16: three BF16 parts): each
operand is represented to ~2^-22 relative, so u_eff ~ 8 u32 = 4.8e-7; the
measured block differences on these problems are <= 7e-6 (c kappa ~ 15),
checked at 1e-4 (one more decade for A_ii^{-1}).  NDHSS_FP32_TF32 (one
rounded TF32 part): u = 2^-11 = 4.9e-4, measured <= 3.1e-3, checked at
2e-2.  One apply: measured <= 1e-5 (FP32-accurate) and <= 5.1e-3 (TF32),
checked at 1e-4 and 5e-2.  GMRES: the end-to-end solution is refined by
float64 GMRES to a true relative residual of 1e-8 either way; iterations
within oracle + 2, except TF32: a preconditioner of one-apply accuracy
delta <= 5e-2 reduces the residual by ~delta per step, so it needs up to
log(1e-8) / log(5e-2) ~ 6.2 steps more than the exact oracle factor's one
(measured: oracle + 3); checked at oracle + 7.
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


@pytest.fixture(autouse=True)
def tensor_core_levels(monkeypatch):
    """The small parity problems take the tensor-core sweep on every level
    with 16 or more interior unknowns (the default threshold is 96)."""
    monkeypatch.setenv("NDHSS_TC_MIN_MI", "16")
    monkeypatch.delenv("NDHSS_FRONT_UPDATE", raising=False)


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


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-4), (2, 2e-2), (3, 1e-4)])
def test_factor_blocks_match_oracle(nd, case, prec, tol):
    """FP64 to rounding; the tensor-core precisions by their products'
    tolerance (module docstring)."""
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
    # one apply: FP32-accurate products measured <= 1e-5, one TF32 part <= 5.1e-3
    tol = {0: 1e-10, 1: 1e-4, 2: 5e-2, 3: 1e-4}[prec]
    assert _rel(y.cpu().numpy(), yo) <= tol
    assert _rel(y.cpu().numpy(), yd) <= tol
    # host buffers through the same entry point
    yh = np.zeros_like(xb.cpu().numpy())
    nd.ndhss_apply(f, xb.cpu().numpy(), yh)
    assert np.array_equal(yh, y.cpu().numpy())


@pytest.mark.parametrize("prec", [1, 3])
def test_tensor_core_sweep_matches_rank_kb_sweep(nd, case, prec, monkeypatch):
    """The two-level sweep (rank-kb steps on a slab, tensor-core block
    exchange of the rest) composes the same exchanges as the rank-kb sweep
    over whole fronts on the CUDA cores: both factors agree to the
    FP32-accurate tolerance, block by block."""
    fa = _gpu_factor(nd, case, prec)
    monkeypatch.setenv("NDHSS_FRONT_UPDATE", "simt")
    fb = _gpu_factor(nd, case, prec)
    T = case["T"]
    st = nd.ndhss_factor_stats_get(fa)
    assert st["tc_flops"] > 0 and nd.ndhss_factor_stats_get(fb)["tc_flops"] == 0
    mi_all, mb_all = T.f("m_i"), T.f("m_b")
    big = [s for s in range(T.nnodes) if mi_all[s] >= 16 and mb_all[s] > 0]
    assert big
    for s in big[:40]:
        mi, mb = int(mi_all[s]), int(mb_all[s])
        for w in range(4):
            a = nd.ndhss_factor_get_block(fa, s, w, mi, mb)
            b = nd.ndhss_factor_get_block(fb, s, w, mi, mb)
            assert _rel(a, b) <= (1e-3 if w == 0 else 1e-4), (s, w, _rel(a, b))


@pytest.mark.parametrize("prec", [0, 1])
def test_register_panel_matches_shared_memory_panel(nd, case, prec, monkeypatch):
    """Panels of at most 512 candidate rows with elements of at most 8 bytes
    run with each row in one thread's registers, tracking positions instead
    of moving rows.  Pivots, ties and the exchange arithmetic are those of
    the shared-memory panel (NDHSS_PANEL=smem): real factors agree bit for
    bit.  Complex products may be contracted into FMAs differently in the
    two kernels (measured: one FP32 ulp, 7.7e-8 relative), checked at 1e-6;
    complex FP64 takes the shared-memory panel both times."""
    fa = _gpu_factor(nd, case, prec)
    monkeypatch.setenv("NDHSS_PANEL", "smem")
    fb = _gpu_factor(nd, case, prec)
    T = case["T"]
    mi_all, mb_all = T.f("m_i"), T.f("m_b")
    nodes = [s for s in range(T.nnodes) if mi_all[s] > 0]
    if len(nodes) > 80:
        nodes = nodes[:: len(nodes) // 80] + [T.nnodes - 1]
    for s in nodes:
        mi, mb = int(mi_all[s]), int(mb_all[s])
        for w in range(4 if mb else 1):
            a = nd.ndhss_factor_get_block(fa, s, w, mi, mb)
            b = nd.ndhss_factor_get_block(fb, s, w, mi, mb)
            if np.iscomplexobj(a):
                assert _rel(a, b) <= 1e-6, (s, w, _rel(a, b))
            else:
                assert np.array_equal(a, b), (s, w, _rel(a, b))


@pytest.mark.parametrize("prob,prec", [("poisson", 0), ("poisson", 1), ("helmholtz", 1)])
def test_register_panel_matches_shared_memory_panel_large_fronts(nd, prob, prec, monkeypatch):
    """A root front of ~600 interior unknowns: its first panels have more
    than 512 candidate rows and take the 1024-thread register panel, which
    is 16 columns wide.  Both factors use 16-column panels (the blocking
    decides the rounding of the updates); same comparison as above, on the
    top fronts.  The complex contraction differences (one FP32 ulp) grow
    through these larger eliminations like any rounding difference:
    measured 1.04e-6, checked at 1e-5."""
    P = poisson_dirichlet(100, p=2, seed=3) if prob == "poisson" else helmholtz_impedance(100, 2, 30.0, seed=3)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    mi_all, mb_all = T.f("m_i"), T.f("m_b")
    assert mi_all.max() > 512
    c = dict(tree=nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64), M=nd.DeviceCSR(P.A))
    fa = _gpu_factor(nd, c, prec, panel=16)
    monkeypatch.setenv("NDHSS_PANEL", "smem")
    fb = _gpu_factor(nd, c, prec, panel=16)
    top = [int(s) for s in np.argsort(-mi_all)[:7]]
    for s in top:
        mi, mb = int(mi_all[s]), int(mb_all[s])
        for w in range(4 if mb else 1):
            a = nd.ndhss_factor_get_block(fa, s, w, mi, mb)
            b = nd.ndhss_factor_get_block(fb, s, w, mi, mb)
            if np.iscomplexobj(a):
                assert _rel(a, b) <= 1e-5, (s, w, _rel(a, b))
            else:
                assert np.array_equal(a, b), (s, w, _rel(a, b))


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
    # oracle + 2; one TF32 part: oracle + 7 (module docstring)
    assert st["iters"] <= ro.iters + (7 if prec == 2 else 2), (st, ro.iters)
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


def test_fma_peak_measurement(nd):
    """The ALU roofline denominators: FP32 well above FP64 on GB300's CUDA
    cores, both within physical bounds (152 SMs x 128 FP32 lanes x 2 flops
    x 2.1 GHz = 82 TFLOP/s at most)."""
    f64 = nd.ndhss_measure_fma_peak(0)
    f32 = nd.ndhss_measure_fma_peak(1)
    assert 0.1 < f64 < 10.0, f64
    assert 10.0 < f32 < 85.0, f32
    assert f32 > 8 * f64
    with pytest.raises(ValueError):
        nd.ndhss_measure_fma_peak(2)
