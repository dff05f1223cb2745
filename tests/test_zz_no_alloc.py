"""The allocation-free apply (ndhss_apply_noalloc) against ndhss_apply.

Some callers cannot allocate device memory when they need P^{-1}: a solver
loop in a process whose device memory another allocator has reserved up
front, or code under a no-allocation-after-setup rule.  This entry point
gives them the same result from a fixed static work area.  Both paths launch
the same kernels on the same factor and task queue, and the apply's sums run
in a fixed order, so the results must agree bit for bit; the compressed cases
exercise the work area's low-rank partial-product slots.  The file is named
to be collected last, so a run that stops at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from ndhss_inputs import helmholtz_impedance, poisson_dirichlet

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


@pytest.mark.parametrize("case,prec,hss_levels", [("poisson", 0, -1), ("helmholtz", 0, -1), ("helmholtz", 1, -1),
                                                  ("helmholtz", 1, 4), ("helmholtz", 0, 4)])
def test_noalloc_apply_matches_apply_twice(nd, case, prec, hss_levels):
    P = poisson_dirichlet(48, seed=3) if case == "poisson" else helmholtz_impedance(40, 2, 15.0, seed=2)
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    M = nd.DeviceCSR(P.A)
    f = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals,
                        nd.make_factor_opts(prec=prec, hss_levels=hss_levels, seed=5))
    if hss_levels >= 0:
        assert nd.ndhss_factor_stats_get(f)["kmax"] > 0      # low-rank nodes present
    rng = np.random.default_rng(11)
    for call in range(2):                       # two calls in a row share the static work area
        x = rng.standard_normal(P.n) + (1j * rng.standard_normal(P.n) if M.vtype == 1 else 0.0)
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        y_ref = torch.empty_like(xd)
        nd.ndhss_apply(f, xd, y_ref)
        y = torch.full_like(xd, float("nan"))
        nd.ndhss_apply_noalloc(f, xd, y)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.array_equal(a, b), (call, float(np.abs(a - b).max()))


def test_noalloc_rejects_host_buffers_and_oversized_problems(nd):
    import ctypes
    P = poisson_dirichlet(16)
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    M = nd.DeviceCSR(P.A)
    f = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals)
    xh = np.ones(P.n)
    yh = np.zeros_like(xh)
    # the C side refuses host memory ...
    code = nd.load().ndhss_apply_noalloc(f.handle, ctypes.c_void_p(xh.ctypes.data), ctypes.c_void_p(yh.ctypes.data),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 1 and "device pointers" in nd.load().ndhss_last_error().decode()
    # ... and the binding refuses buffers of the wrong kind, type or length before calling it
    xd = torch.ones(P.n, dtype=torch.float64, device="cuda")
    for bad in (xh, xd.to(torch.float32), xd[:-1], torch.ones(P.n, dtype=torch.complex128, device="cuda")):
        with pytest.raises(ValueError):
            nd.ndhss_apply_noalloc(f, bad, torch.empty_like(xd))
    # complex128 fronts need 32 bytes per DOF: n = 731^2 > 524272 exceeds the 16 MiB area
    H = helmholtz_impedance(730, 1, 4.0, seed=0)
    treeH = nd.ndhss_build_tree(H.coords, H.A.indptr, H.A.indices, 64)
    MH = nd.DeviceCSR(H.A)
    fH = nd.ndhss_factor(treeH, MH.vtype, MH.rowptr, MH.col, MH.vals, nd.make_factor_opts(prec=0))
    xd = torch.zeros(H.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(nd.NdhssError) as ei:
        nd.ndhss_apply_noalloc(fH, xd, torch.empty_like(xd))
    assert ei.value.code == 1 and "static scratch" in str(ei.value)
