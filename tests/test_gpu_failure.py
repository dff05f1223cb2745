"""Failure detection of the persistent apply without a GPU fault.

Every wait of the dataflow apply kernel is bounded.  The testing hook raises
one completion requirement beyond what any task will signal (a counter that
nothing sets), so the next apply's down-sweep tasks wait until the bound runs
out; the kernel then returns early and the host reads the status.  The
context must stay usable: a fresh factorization on the same device still
solves, and the marked one fails fast from then on.
"""
import time

import numpy as np
import pytest

from ndhss_inputs import poisson_dirichlet

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


def test_stalled_apply_times_out_and_context_survives(nd):
    P = poisson_dirichlet(32)
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    M = nd.DeviceCSR(P.A)
    f = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, nd.make_factor_opts(prec=0))
    b = np.ascontiguousarray(P.b, dtype=np.float64)
    y = np.zeros_like(b)
    nd.ndhss_apply(f, b, y)                      # healthy first
    nd.ndhss_testing_stall_apply(f)
    t0 = time.time()
    with pytest.raises(nd.NdhssError) as e:
        nd.ndhss_apply(f, b, y)
    assert e.value.code == 6 and "gave up" in str(e.value)
    assert time.time() - t0 < 30
    t0 = time.time()
    with pytest.raises(nd.NdhssError) as e:     # marked: later applies return at once
        nd.ndhss_apply(f, b, y)
    assert e.value.code == 6 and time.time() - t0 < 1.5
    del f
    g = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, nd.make_factor_opts(prec=0))
    y2 = np.zeros_like(b)
    nd.ndhss_apply(g, b, y2)
    r = P.A @ y2 - b
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)


def test_noalloc_apply_timeout_surfaces_at_the_next_synchronising_call(nd):
    # the allocation-free apply never synchronises: a wait that gives up inside
    # it marks the factorization, and the next synchronising call reports it
    P = poisson_dirichlet(24)
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    M = nd.DeviceCSR(P.A)
    f = nd.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, nd.make_factor_opts(prec=0))
    xd = torch.from_numpy(np.ascontiguousarray(P.b, dtype=np.float64)).cuda()
    yd = torch.empty_like(xd)
    nd.ndhss_testing_stall_apply(f)
    t0 = time.time()
    nd.ndhss_apply_noalloc(f, xd, yd)            # returns OK: nothing waited on yet
    torch.cuda.synchronize()
    assert time.time() - t0 < 30
    b = np.ascontiguousarray(P.b, dtype=np.float64)
    with pytest.raises(nd.NdhssError) as e:
        nd.ndhss_apply(f, b, np.zeros_like(b))   # host buffers: this call synchronises
    assert e.value.code == 6
