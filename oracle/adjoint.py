"""Oracle: the gradient of a data misfit with respect to piecewise-constant
squared-slowness coefficients by the adjoint state.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For A(m) x_s = b_s (A complex symmetric, Eq. 4.2 with m on blocks) and
J(m) = 0.5 sum_s ||R x_s - d_s||^2 (R samples receiver DOFs):
  g_s = R^T (R x_s - d_s)                 gradient of J in x_s (conjugate-Wirtinger
                                          convention: dJ = Re(g^H dx))
  lambda_s = A^{-H} g_s                   the adjoint state
  dJ/dm_j = -sum_s Re(lambda_s^H (dA/dm_j) x_s),
  dA/dm_j = -k^2 sum_{e in j} M_e - i k / (2 sqrt(m_j)) sum_{edges in j} E_e.
Solves are sparse direct (no iteration tolerance in the reference).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def block_qform(meta, lam: np.ndarray, x: np.ndarray, nblk: int):
    """Per block j: q_M[j] = sum_{e in j} lam_e^H M_e x_e and q_E[j] likewise
    over the boundary edges (lam, x: [n] complex)."""
    e, Me, eb = meta["elem"], meta["Me"], meta["eblk"]
    qe = np.einsum("ea,eab,eb->e", np.conj(lam[e]), Me, x[e])
    qM = np.bincount(eb, weights=qe.real, minlength=nblk) + 1j * np.bincount(eb, weights=qe.imag, minlength=nblk)
    ed, Ee, ebk = meta["edges"], meta["Ee"], meta["edge_blk"]
    qd = np.einsum("ea,eab,eb->e", np.conj(lam[ed]), Ee, x[ed])
    qE = np.bincount(ebk, weights=qd.real, minlength=nblk) + 1j * np.bincount(ebk, weights=qd.imag, minlength=nblk)
    return qM, qE


def coefficient_gradient(meta, lam: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dJ/dm_j = -Re(lam^H dA/dm_j x) for one (lam, x) pair."""
    mb = meta["m_blocks"].ravel()
    k = meta["k"]
    qM, qE = block_qform(meta, lam, x, mb.size)
    return -np.real(-k * k * qM - 1j * k / (2.0 * np.sqrt(mb)) * qE)


def misfit_and_gradient(P, rec: np.ndarray, d: np.ndarray):
    """J and dJ/dm (flattened blocks) for the problem P (b: [n, nsrc]),
    receivers ``rec`` (DOF indices) and data d [len(rec), nsrc]."""
    A = P.A.tocsc()
    B = P.b.reshape(A.shape[0], -1)
    lu = spla.splu(A)
    J = 0.0
    grad = np.zeros(P.meta["m_blocks"].size)
    for s in range(B.shape[1]):
        x = lu.solve(B[:, s])
        r = x[rec] - d[:, s]
        J += 0.5 * float(np.vdot(r, r).real)
        g = np.zeros_like(x)
        g[rec] = r
        lam = np.conj(lu.solve(np.conj(g)))          # A^{-H} g = conj(A^{-1} conj(g)) since A^T = A
        grad += coefficient_gradient(P.meta, lam, x)
    return J, grad
