"""The parameter-study driver (paper_2105_07791_gb300/sweeps.py): its report
and exponent fit on the CPU; one tiny sweep of each kind on the GPU."""
import numpy as np
import pytest

from paper_2105_07791_gb300 import sweeps


def test_fit_exponent_recovers_a_power_law():
    n = np.array([1e4, 4e4, 1.6e5, 6.4e5])
    assert abs(sweeps.fit_exponent(n, 3.0 * n ** 1.5) - 1.5) < 1e-12
    assert abs(sweeps.fit_exponent(n, 2.0 * n * np.log(n)) - 1.0) < 0.2


def test_report_has_every_row_and_the_fits():
    h = [dict(problem="poisson", N=N, n=N * N, depth=5, apply_ms=1e-5 * N * N, factor_ms=1e-6 * (N * N) ** 1.5,
              factor_bytes=100 * N * N, iters=3, kmax=20) for N in (256, 512, 1024)]
    k = [dict(N=32, kappa=kk, ppw=10.0, n=4225, iters=4, kmax=30, true_relres=1e-10) for kk in (2, 4)]
    d = [dict(N=32, kappa=4, levels_above_leaf=L, iters=4, kmax=30, factor_ms=1.0) for L in (2, 3)]
    text = sweeps.report(k, d, h)
    assert text.count("| poisson |") == 3 + 1                  # three rows and the fitted exponents
    assert "| poisson | 1.50 | 1.00 | 1.00 |" in text
    assert text.count("| 32 | 4 |") == 1 + 2


@pytest.mark.gpu
def test_tiny_sweeps_run_on_the_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_07791_gb300 import build, ndhss
    build.build()
    ndhss.load()
    kr = sweeps.kappa_sweep(meshes=(12,), kappas=(2, 4, 64))
    assert [r["kappa"] for r in kr] == [2, 4]                    # kappa 64 has < 6 points per wavelength
    dr = sweeps.depth_sweep(N=12, kappas=(4,), levels=(1, 2))
    hr = sweeps.h_sweep(meshes=(16, 24))
    for r in kr + dr + hr:
        assert r["converged"] and r["true_relres"] <= 1e-9 and r["factor_ms"] > 0
    assert len(hr) == 8
