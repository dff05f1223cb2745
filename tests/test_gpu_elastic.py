"""The elastic-wave workload (P1 SIPG, two displacement components, absorbing
boundary; ndhss_inputs/elastic.py) through the C ABI against the FP64 oracle:
exact dense tier, compressed tier (beta = 60, a multiple of the six unknowns
of an element, so HSS leaves hold whole elements), and GMRES to the
workload's 1e-6 and to 1e-8.  Tolerances as in test_gpu_parity /
test_gpu_hss (FP64 rounding; FP32 u32 x kappa; compressed eps-limited)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from ndhss_inputs.elastic import elastic_sipg
from oracle.frontal import apply_inverse, factor_dense
from oracle.gmres import gmres as oracle_gmres
from oracle.hss import apply_compressed, factor_compressed
from oracle.tree import build_tree
from closeness import rel as _rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LEAF, BETA, HL, EPS = 60, 60, 3, 1e-6


@pytest.fixture(scope="module")
def nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_07791_gb300 import build, ndhss
    build.build()
    ndhss.load()
    return ndhss


@pytest.fixture(scope="module")
def el(nd):
    P = elastic_sipg(20, seed=4)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, LEAF)
    return dict(P=P, T=T, dense=factor_dense(T, P.A),
                comp=factor_compressed(T, P.A, hss_levels=HL, eps=EPS, beta=BETA, k0=32, r=16, seed=7),
                tree=nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, LEAF), M=nd.DeviceCSR(P.A))


def _factor(nd, el, prec, hl):
    M = el["M"]
    opts = nd.make_factor_opts(prec=prec, hss_levels=hl, eps_hss=EPS, beta=BETA, k0=32, r=16, seed=7)
    f = nd.ndhss_factor(el["tree"], M.vtype, M.rowptr, M.col, M.vals, opts)
    torch.cuda.synchronize()
    return f


@pytest.mark.parametrize("prec,hl,tol", [(0, -1, 1e-10), (1, -1, 2e-3), (3, -1, 2e-3), (0, HL, 1e-4), (1, HL, 1e-3),
                                         (3, HL, 1e-3)])
def test_apply_matches_oracle(nd, el, prec, hl, tol, monkeypatch):
    monkeypatch.setenv("NDHSS_TC_MIN_MI", "16")     # the tensor-core sweep on every level it can take
    P = el["P"]
    f = _factor(nd, el, prec, hl)
    b = np.ascontiguousarray(P.b)
    bd = torch.from_numpy(b).cuda()
    y = torch.empty_like(bd)
    nd.ndhss_apply(f, bd, y)
    yo = apply_inverse(el["dense"], b) if hl < 0 else apply_compressed(el["comp"], b)
    assert _rel(y.cpu().numpy(), yo) <= tol, _rel(y.cpu().numpy(), yo)
    if hl < 0 and prec == 0:
        assert _rel(y.cpu().numpy(), spla.spsolve(P.A.tocsc(), b)) <= 1e-9


@pytest.mark.parametrize("prec,hl,tol", [(1, HL, 1e-6), (1, HL, 1e-8), (0, HL, 1e-8), (1, -1, 1e-8), (3, -1, 1e-8)])
def test_gmres_solution_and_iterations(nd, el, prec, hl, tol, monkeypatch):
    monkeypatch.setenv("NDHSS_TC_MIN_MI", "16")
    P = el["P"]
    f = _factor(nd, el, prec, hl)
    b = np.ascontiguousarray(P.b)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st = nd.ndhss_gmres(f, el["M"].rowptr, el["M"].col, el["M"].vals, bd, x, tol=tol)
    xs = x.cpu().numpy()
    assert st["converged"] and np.linalg.norm(b - P.A @ xs) <= tol * np.linalg.norm(b) * 1.0001
    fac = el["dense"] if hl < 0 else el["comp"]
    prec_o = (lambda v: apply_inverse(fac, v)) if hl < 0 else (lambda v: apply_compressed(fac, v))
    ro = oracle_gmres(P.A, b, prec_o, tol=tol)
    # oracle + 2; a compressed factor from FP32 fronts differs from the oracle's
    # FP64 compression by up to the one-apply tolerance 1e-3 (the FP32
    # estimator floor, 1e3 u32 ~ 6e-5 of a block's norm, stops the sampling
    # above eps): each float64 refinement cycle gains ~3 digits, so a 1e-8
    # solve needs up to two more cycles than the oracle's (oracle + 4)
    slack = 4 if (prec != 0 and hl >= 0) else 2
    assert st["iters"] <= ro.iters + slack, (st["iters"], ro.iters)
