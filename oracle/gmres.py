"""Oracle: restarted, left-preconditioned GMRES in float64 / complex128.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 4 runs restarted GMRES on P^{-1} A x = P^{-1} b (Eq. 1.2) and stops on
the preconditioned relative residual ||P^{-1}(A x - b)|| / ||P^{-1} b||.
Readings used here (restart length, tolerance and the true-residual rule are
not fixed by the paper for these workloads):

* x0 = 0; Arnoldi with classical Gram-Schmidt applied twice (CGS2);
  complex Givens rotations G = [[c, s], [-conj(s), c]] with real c.
* A cycle ends when |g_{j+1}| <= inner * tol * ||P^{-1} b|| (inner test),
  after ``restart`` steps, on breakdown, or at ``maxit`` total steps.  The
  default inner = 0.1 follows Sec. 4, which stops on a preconditioned
  residual one decade below the accuracy it reports (1e-9); it keeps a
  preconditioner applied in reduced precision from ending cycles on an
  estimate that the float64 residual does not yet meet.
* Optionally (cycle_rtol > 0) a cycle also ends once |g_{j+1}| <= cycle_rtol *
  beta_cycle: with a preconditioner applied in reduced precision the Krylov
  estimate is not trustworthy beyond what one application resolves, and the
  float64 restart performs the refinement instead.
* After each cycle the float64 true residual ||b - A x|| / ||b|| is checked;
  the solve is converged only when it is <= tol.  Otherwise the method
  restarts from the current x (so the outer loop acts as iterative
  refinement), with at least one Arnoldi step per cycle.
* The iteration count is the number of Arnoldi steps (products with P^{-1} A).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    converged: bool
    true_relres: float
    cycles: int
    history: list = field(default_factory=list)    # |g_{j+1}| / ||P^{-1} b|| per step


def givens(a, b):
    """(c, s) with c real such that [[c, s], [-conj(s), c]] @ [a, b] = [r, 0]."""
    if b == 0:
        return 1.0, 0.0 * a
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = np.hypot(abs(a), abs(b))
    return abs(a) / t, (a / abs(a)) * np.conj(b) / t


def gmres(A, b, prec, tol: float = 1e-8, restart: int = 30, maxit: int = 300, inner: float = 0.1,
          cycle_rtol: float = 0.0) -> GmresResult:
    """Solve A x = b; ``prec(v)`` applies P^{-1}; ``A`` supports ``A @ v``."""
    dtype = np.result_type(A.dtype, b.dtype, np.float64)
    n = b.shape[0]
    x = np.zeros(n, dtype=dtype)
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return GmresResult(x=x, iters=0, converged=True, true_relres=0.0, cycles=0)
    zbnorm = np.linalg.norm(prec(b.astype(dtype)))
    its = 0
    cycles = 0
    hist = []
    while True:
        r = b - A @ x
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            return GmresResult(x=x, iters=its, converged=True, true_relres=float(rel), cycles=cycles, history=hist)
        if its >= maxit:
            return GmresResult(x=x, iters=its, converged=False, true_relres=float(rel), cycles=cycles, history=hist)
        cycles += 1
        z = prec(r)
        beta = np.linalg.norm(z)
        V = np.zeros((n, restart + 1), dtype=dtype)
        H = np.zeros((restart + 1, restart), dtype=dtype)
        cs = np.zeros(restart)
        sn = np.zeros(restart, dtype=dtype)
        g = np.zeros(restart + 1, dtype=dtype)
        g[0] = beta
        V[:, 0] = z / beta
        j_end = 0
        for j in range(restart):
            w = prec(A @ V[:, j])
            its += 1
            h = V[:, :j + 1].conj().T @ w                  # CGS, first pass
            w = w - V[:, :j + 1] @ h
            h2 = V[:, :j + 1].conj().T @ w                 # second pass
            w = w - V[:, :j + 1] @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0:
                V[:, j + 1] = w / hn
            for i in range(j):                             # previous rotations
                t0 = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                t1 = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j], H[i + 1, j] = t0, t1
            c, s = givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j] = c * H[j, j] + s * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            res = abs(g[j + 1]) / zbnorm
            hist.append(float(res))
            j_end = j + 1
            if res <= inner * tol or abs(g[j + 1]) <= cycle_rtol * beta or hn == 0 or its >= maxit:
                break
        y = sla.solve_triangular(H[:j_end, :j_end], g[:j_end], lower=False)
        x = x + V[:, :j_end] @ y
