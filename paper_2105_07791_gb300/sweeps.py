"""The paper's parameter studies on synthetic meshes, run through the C ABI on
one GPU (Sec. 4.3 - 4.6):

* ``kappa``: GMRES iterations and k_max (the largest rank of any compressed
  Schur complement block or Gauss transform) for wavenumbers kappa = 2 ... 256
  at p = 2 on several meshes (Fig. 9);
* ``depth``: iterations against kappa for several switching levels (levels
  above the leaf at which compression starts; Figs. 8 and 13);
* ``h``: factorization time, application time, factor memory, iterations and
  k_max under h-refinement for Poisson, Helmholtz at fixed kappa and Helmholtz
  at fixed kappa h (Tables 2 and 3).

The discretization is this package's continuous Galerkin one with impedance
conditions for Helmholtz (the paper's tables use an interior-penalty DG
discretization with Dirichlet conditions), so the numbers compare in trend,
not in value.  Usage::

    python -m paper_2105_07791_gb300.sweeps --which all --out sweeps.md
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np


def run_case(P, *, leaf=64, hss_levels=4, prec=None, tol=1e-9, eps_hss=1e-6, beta=64, maxit=300):
    """Factor P.A and solve A x = b (first right-hand side); times by CUDA events."""
    import torch

    from . import ndhss
    if prec is None:
        prec = ndhss.NDHSS_FP32
    tree = ndhss.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, leaf)
    M = ndhss.DeviceCSR(P.A)
    b0 = P.b if P.b.ndim == 1 else P.b[:, 0]
    b = torch.from_numpy(np.ascontiguousarray(b0)).cuda()
    x = torch.zeros_like(b)
    opts = ndhss.make_factor_opts(prec=prec, hss_levels=hss_levels, eps_hss=eps_hss, beta=beta)
    stream = torch.cuda.current_stream()
    ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, opts, stream=stream)     # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    f = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, opts, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    st = ndhss.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x, tol=tol, maxit=maxit, timing=True, stream=stream)
    fs = ndhss.ndhss_factor_stats_get(f)
    return dict(n=int(P.n), depth=int(tree.depth), factor_ms=e0.elapsed_time(e1),
                apply_ms=st["apply_ms"] / max(st["napply"], 1), iters=int(st["iters"]), converged=bool(st["converged"]),
                true_relres=float(st["true_relres"]), kmax=int(fs["kmax"]), factor_bytes=int(fs["factor_bytes"]),
                apply_bytes=int(fs["apply_bytes"]))


def kappa_sweep(meshes=(32, 64, 128), kappas=(2, 4, 8, 16, 32, 64, 128, 256), p=2, min_ppw=6.0, **kw):
    """Fig. 9: iterations and k_max against kappa; a (mesh, kappa) pair is run
    when the P-p nodal lattice keeps >= min_ppw points per wavelength."""
    from ndhss_inputs import helmholtz_impedance
    rows = []
    for N in meshes:
        for k in kappas:
            ppw = (2 * math.pi / k) * p * N
            if ppw < min_ppw:
                continue
            r = run_case(helmholtz_impedance(N, p, float(k), seed=0), **kw)
            r.update(N=N, p=p, kappa=k, ppw=ppw)
            rows.append(r)
    return rows


def depth_sweep(N=64, p=2, kappas=(4, 8, 16, 32, 64), levels=(2, 3, 4, 5, 6), **kw):
    """Figs. 8 / 13: iterations against kappa for several switching levels."""
    from ndhss_inputs import helmholtz_impedance
    rows = []
    for k in kappas:
        P = helmholtz_impedance(N, p, float(k), seed=0)
        for L in levels:
            r = run_case(P, hss_levels=L, **kw)
            r.update(N=N, p=p, kappa=k, levels_above_leaf=L)
            rows.append(r)
    return rows


def h_sweep(meshes=(32, 64, 128, 256, 512), p=1, **kw):
    """Tables 2 and 3: Poisson; Helmholtz with kappa = 10; Helmholtz with
    kappa h = 1/4 and 1/2 (h = 1/N)."""
    from ndhss_inputs import helmholtz_impedance, poisson_dirichlet
    rows = []
    for name in ("poisson", "helmholtz_k10", "helmholtz_kh0.25", "helmholtz_kh0.5"):
        for N in meshes:
            if name == "poisson":
                P = poisson_dirichlet(N, p=p, seed=0)
            elif name == "helmholtz_k10":
                P = helmholtz_impedance(N, p, 10.0, seed=0)
            else:
                kh = float(name.split("kh")[1])
                P = helmholtz_impedance(N, p, kh * N, seed=0)
            r = run_case(P, **kw)
            r.update(problem=name, N=N, p=p)
            rows.append(r)
    return rows


def fit_exponent(ns, ts):
    """Least-squares slope of log t against log n."""
    ns, ts = np.log(np.asarray(ns, float)), np.log(np.asarray(ts, float))
    return float(np.polyfit(ns, ts, 1)[0]) if ns.size >= 2 else float("nan")


def _table(rows, cols):
    out = ["| " + " | ".join(c for c, _ in cols) + " |", "|" + "---|" * len(cols)]
    for r in rows:
        out.append("| " + " | ".join(f(r) for _, f in cols) + " |")
    return "\n".join(out)


def report(kappa_rows=None, depth_rows=None, h_rows=None) -> str:
    parts = []
    if kappa_rows:
        parts.append("### Iterations and k_max against kappa (p = 2, tol 1e-9, compression 4 levels above the leaf)\n")
        parts.append(_table(kappa_rows, [("1/h", lambda r: str(r["N"])), ("kappa", lambda r: str(r["kappa"])),
                                         ("points/wavelength", lambda r: f"{r['ppw']:.1f}"), ("n", lambda r: str(r["n"])),
                                         ("iters", lambda r: str(r["iters"])), ("k_max", lambda r: str(r["kmax"])),
                                         ("true relres", lambda r: f"{r['true_relres']:.1e}")]))
    if depth_rows:
        parts.append("\n\n### Iterations against kappa for several switching levels (p = 2)\n")
        parts.append(_table(depth_rows, [("1/h", lambda r: str(r["N"])), ("kappa", lambda r: str(r["kappa"])),
                                         ("levels above leaf", lambda r: str(r["levels_above_leaf"])),
                                         ("iters", lambda r: str(r["iters"])), ("k_max", lambda r: str(r["kmax"])),
                                         ("factor ms", lambda r: f"{r['factor_ms']:.1f}")]))
    if h_rows:
        parts.append("\n\n### h-refinement (p = 1, compression 4 levels above the leaf, tol 1e-9)\n")
        parts.append(_table(h_rows, [("problem", lambda r: r["problem"]), ("1/h", lambda r: str(r["N"])),
                                     ("n", lambda r: str(r["n"])), ("depth", lambda r: str(r["depth"])),
                                     ("apply ms", lambda r: f"{r['apply_ms']:.3f}"),
                                     ("factor ms", lambda r: f"{r['factor_ms']:.1f}"),
                                     ("factor MB", lambda r: f"{r['factor_bytes'] / 1e6:.0f}"),
                                     ("iters", lambda r: str(r["iters"])), ("k_max", lambda r: str(r["kmax"]))]))
        fits = []
        for name in sorted({r["problem"] for r in h_rows}):
            rs = [r for r in h_rows if r["problem"] == name and r["n"] >= 50000]
            if len(rs) >= 2:
                fits.append(f"| {name} | {fit_exponent([r['n'] for r in rs], [r['factor_ms'] for r in rs]):.2f} | "
                            f"{fit_exponent([r['n'] for r in rs], [r['apply_ms'] for r in rs]):.2f} | "
                            f"{fit_exponent([r['n'] for r in rs], [r['factor_bytes'] for r in rs]):.2f} |")
        if fits:
            parts.append("\n\nFitted exponents t ~ n^a over the meshes with n >= 5e4:\n\n"
                         "| problem | factor | apply | memory |\n|---|---|---|---|\n" + "\n".join(fits))
    return "\n".join(parts) + "\n"


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--which", choices=["kappa", "depth", "h", "all"], default="all")
    ap.add_argument("--out", default=None, help="write the markdown report here (default: stdout)")
    a = ap.parse_args(argv)
    from . import build, ndhss
    build.build()
    ndhss.load()
    t0 = time.time()
    kr = kappa_sweep() if a.which in ("kappa", "all") else None
    dr = depth_sweep() if a.which in ("depth", "all") else None
    hr = h_sweep() if a.which in ("h", "all") else None
    text = report(kr, dr, hr) + f"\n(sweeps took {time.time() - t0:.0f} s)\n"
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text)
    print(text)


if __name__ == "__main__":
    main()
