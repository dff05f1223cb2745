"""Time-harmonic elastic waves (the Navier equation, Sec. 4.4 / Eq. 4.6) with a
P1 symmetric interior-penalty DG discretization on the N x N cell grid of
[0,1]^2 (each cell cut by its (+1, +1) diagonal into two triangles).

Bilinear (not sesquilinear) form, so the matrix is complex symmetric:

    a(u, v) = sum_K int_K sigma(u) : eps(v) - omega^2 int rho u . v
              - sum_F int_F ({sigma(u) n} . [v] + {sigma(v) n} . [u])
              + sum_F sigma_F int_F [u] . [v]
              - i omega sum_{F on dOmega} int_F rho (c_p (u.n)(v.n) + c_s (u.t)(v.t))

with sigma(u) = lam div(u) I + 2 mu eps(u), interior faces F (normal n out of
the first element, [u] = u_first - u_second, {.} the average), penalty
sigma_F = 10 (lam + 2 mu)_max,F (p + 1)^2 / h_F, h_F the face length, and the
first-order absorbing condition sigma(u) n = i omega rho (c_p n n^T + c_s t t^T) u
(c_p = sqrt((lam + 2 mu) / rho), c_s = sqrt(mu / rho), t the tangent).
lam and mu are constant per element (taken at the centroid).

Degrees of freedom: element e, vertex a (its three vertices in the mesh's
counter-clockwise order), component c -> 6 e + 2 a + c, so an element's six
unknowns are contiguous and a cell's twelve too; every unknown's lattice
coordinate is its cell (a, b), as the tree builder wants for DG (elements are
never split between boxes).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fem import Problem, _finish, _mesh, gaussian_source


def fourier_field(N: int, xy_c: np.ndarray, rng, nmodes: int = 16, lo: float = 1.0, hi: float = 4.0):
    """lo + (hi - lo) (1 + f) / 2 at the points xy_c, f the sum of nmodes seeded
    Fourier modes a_m cos(2 pi k_m . x + phi_m) (k_m integer in 1..4, a_m ~
    U[0.5, 1]) divided by sum |a_m|, so the values lie in [lo, hi]."""
    k = rng.integers(1, 5, size=(nmodes, 2))
    a = rng.uniform(0.5, 1.0, size=nmodes)
    ph = rng.uniform(0.0, 2 * np.pi, size=nmodes)
    f = np.zeros(xy_c.shape[0])
    for m in range(nmodes):
        f += a[m] * np.cos(2 * np.pi * (k[m, 0] * xy_c[:, 0] + k[m, 1] * xy_c[:, 1]) + ph[m])
    f /= np.abs(a).sum()
    return lo + (hi - lo) * 0.5 * (1.0 + f)


def elastic_sipg(N: int, *, seed: int = 0, lam=None, mu=None, rho: float = 1.0, omega=None, ppw: float = 8.0,
                 nsrc: int = 1, width: float = 0.02, src_xy=None) -> Problem:
    """The SIPG elastic-wave system on N x N cells.  ``lam`` / ``mu``: per-element
    arrays or scalars (default: seeded Fourier fields in [1, 4]); ``omega``:
    default 2 pi min(c_s) / (ppw h) (ppw points per shear wavelength).
    Right-hand sides: a Gaussian body force (both components) of the given
    width at ``src_xy`` [nsrc, 2] (default drawn ~ U[0.1, 0.9]^2 from the
    seed), projected on the DG space (element mass matrix times the force at
    the vertices)."""
    elem, cell, lattice, xy, Lx, Ly = _mesh(N, N, 1)
    ne = elem.shape[0]
    X = xy[elem]                                                   # [ne, 3, 2]
    xc = X.mean(axis=1)
    rng = np.random.default_rng(seed)
    lam_e = fourier_field(N, xc, rng) if lam is None else np.broadcast_to(np.asarray(lam, float), (ne,)).copy()
    mu_e = fourier_field(N, xc, rng) if mu is None else np.broadcast_to(np.asarray(mu, float), (ne,)).copy()
    h = 1.0 / N
    cs = np.sqrt(mu_e / rho)
    cp = np.sqrt((lam_e + 2 * mu_e) / rho)
    if omega is None:
        omega = 2 * np.pi * float(cs.min()) / (ppw * h)
    # P1 basis phi_a(x) = alpha_a + g_a . x on every element
    d1, d2 = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    area = 0.5 * np.abs(det)
    g = np.empty((ne, 3, 2))
    g[:, 1, 0], g[:, 1, 1] = d2[:, 1] / det, -d2[:, 0] / det
    g[:, 2, 0], g[:, 2, 1] = -d1[:, 1] / det, d1[:, 0] / det
    g[:, 0] = -(g[:, 1] + g[:, 2])
    alpha = 1.0 - np.einsum("eak,eak->ea", g, X)

    def dof(e, a, c):
        return 6 * np.asarray(e) + 2 * np.asarray(a) + np.asarray(c)

    rows, cols, vals = [], [], []
    # volume: stiffness and mass, per element 6 x 6
    ai, ci, bj, dj = np.meshgrid(np.arange(3), np.arange(2), np.arange(3), np.arange(2), indexing="ij")
    ai, ci, bj, dj = (t.ravel() for t in (ai, ci, bj, dj))
    ga, gb = g[:, ai, :], g[:, bj, :]                             # [ne, 36, 2]
    dot = np.einsum("eqk,eqk->eq", ga, gb)
    gac = np.take_along_axis(ga, np.broadcast_to(ci[None, :, None], (ne, 36, 1)), 2)[..., 0]
    gad = np.take_along_axis(ga, np.broadcast_to(dj[None, :, None], (ne, 36, 1)), 2)[..., 0]
    gbc = np.take_along_axis(gb, np.broadcast_to(ci[None, :, None], (ne, 36, 1)), 2)[..., 0]
    gbd = np.take_along_axis(gb, np.broadcast_to(dj[None, :, None], (ne, 36, 1)), 2)[..., 0]
    Kv = (lam_e[:, None] * gac * gbd + mu_e[:, None] * ((ci == dj)[None] * dot + gbc * gad)) * area[:, None]
    Mv = rho * (ci == dj)[None] * (area[:, None] / 12.0) * (1.0 + (ai == bj)[None])
    e_idx = np.repeat(np.arange(ne), 36)
    rows.append(dof(e_idx, np.tile(ai, ne), np.tile(ci, ne)))
    cols.append(dof(e_idx, np.tile(bj, ne), np.tile(dj, ne)))
    vals.append((Kv - omega * omega * Mv).ravel().astype(np.complex128))
    # faces: every edge with its one or two elements
    loc = np.array([[0, 1], [1, 2], [2, 0]])
    ev = elem[:, loc]                                              # [ne, 3, 2] vertex ids per local edge
    key = np.sort(ev, axis=2).reshape(-1, 2)
    order = np.lexsort((key[:, 1], key[:, 0]))
    ks = key[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    first = order[:-1][same]                                       # (element * 3 + local edge) pairs
    second = order[1:][same]
    paired = np.zeros(key.shape[0], bool)
    paired[first] = paired[second] = True
    bnd = np.nonzero(~paired)[0]
    tq, wq = np.polynomial.legendre.leggauss(2)
    tq, wq = 0.5 * (tq + 1.0), 0.5 * wq

    def face_geom(fe):
        e, le = fe // 3, fe % 3
        P0, P1 = xy[ev[e, le, 0]], xy[ev[e, le, 1]]
        tvec = P1 - P0
        L = np.linalg.norm(tvec, axis=1)
        t = tvec / L[:, None]
        n = np.stack([t[:, 1], -t[:, 0]], axis=1)                 # outward for counter-clockwise elements
        pts = P0[:, None, :] + tq[None, :, None] * tvec[:, None, :]   # [nf, 2 quad points, 2]
        return e, L, n, t, pts

    def phi(e, pts):
        """[nf, 3 basis, nq] values of element e's basis at the points."""
        return alpha[e][:, :, None] + np.einsum("fak,fqk->faq", g[e], pts)

    def sig_n(e, n):
        """(sigma(phi_b e_d) n)_c of element e: [nf, 3 (b), 2 (d), 2 (c)]."""
        gb_ = g[e]                                                 # [nf, 3, 2]
        gn = np.einsum("fbk,fk->fb", gb_, n)
        out = lam_e[e][:, None, None, None] * gb_[:, :, :, None] * n[:, None, None, :]
        eye = np.eye(2)[None, None]
        out = out + mu_e[e][:, None, None, None] * (eye * gn[:, :, None, None]
                                                     + gb_[:, :, None, :] * n[:, None, :, None])
        return out                                                 # indexed [f, b, d, c]

    # interior faces
    eP, L, n, t, pts = face_geom(first)
    eM = second // 3
    phP, phM = phi(eP, pts), phi(eM, pts)                          # [nf, 3, nq]
    sP, sM = sig_n(eP, n), sig_n(eM, n)
    sigF = 10.0 * np.maximum(lam_e[eP] + 2 * mu_e[eP], lam_e[eM] + 2 * mu_e[eM]) * 4.0 / L
    sides = ((eP, phP, sP, 1.0), (eM, phM, sM, -1.0))
    for (eI, phI, sI, si) in sides:
        for (eJ, phJ, sJ, sj) in sides:
            intI = np.einsum("faq,q->fa", phI, wq) * L[:, None]                    # int phi_a^I
            intJ = np.einsum("fbq,q->fb", phJ, wq) * L[:, None]
            mass = np.einsum("faq,fbq,q->fab", phI, phJ, wq) * L[:, None, None]   # int phi_a^I phi_b^J
            blk = np.zeros((eI.size, 3, 2, 3, 2))                                 # [f, a, c, b, d]
            # - int {sigma(u) n} . [v]:  u = phi_b^J e_d, v = phi_a^I e_c
            blk -= 0.5 * si * np.einsum("fa,fbdc->facbd", intI, sJ)
            # - int {sigma(v) n} . [u]
            blk -= 0.5 * sj * np.einsum("fb,facd->facbd", intJ, sI)
            # + sigma_F int [u] . [v]
            blk += (si * sj) * sigF[:, None, None, None, None] * np.einsum("fab,cd->facbd", mass, np.eye(2))
            A_, C_, B_, D_ = np.meshgrid(np.arange(3), np.arange(2), np.arange(3), np.arange(2), indexing="ij")
            rows.append(dof(eI[:, None], A_.ravel()[None], C_.ravel()[None]).ravel())
            cols.append(dof(eJ[:, None], B_.ravel()[None], D_.ravel()[None]).ravel())
            vals.append(blk.reshape(eI.size, 36).ravel().astype(np.complex128))
    # boundary faces: absorbing term
    eB, LB, nB, tB, ptsB = face_geom(bnd)
    phB = phi(eB, ptsB)
    massB = np.einsum("faq,fbq,q->fab", phB, phB, wq) * LB[:, None, None]
    coef = rho * (cp[eB][:, None, None] * np.einsum("fc,fd->fcd", nB, nB)
                  + cs[eB][:, None, None] * np.einsum("fc,fd->fcd", tB, tB))
    blkB = -1j * omega * np.einsum("fab,fcd->facbd", massB, coef)
    A_, C_, B_, D_ = np.meshgrid(np.arange(3), np.arange(2), np.arange(3), np.arange(2), indexing="ij")
    rows.append(dof(eB[:, None], A_.ravel()[None], C_.ravel()[None]).ravel())
    cols.append(dof(eB[:, None], B_.ravel()[None], D_.ravel()[None]).ravel())
    vals.append(blkB.reshape(eB.size, 36).ravel())
    ndof = 6 * ne
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(ndof, ndof)).tocsr()
    A.sort_indices()
    # right-hand sides: Gaussian body force (1, 1), projected
    if src_xy is None:
        src_xy = rng.uniform(0.1, 0.9, size=(nsrc, 2))
    src_xy = np.asarray(src_xy, float)
    Me_loc = (area[:, None, None] / 12.0) * (np.ones((3, 3)) + np.eye(3))[None]      # [ne, 3, 3]
    B = np.zeros((ndof, src_xy.shape[0]), dtype=np.complex128)
    for s in range(src_xy.shape[0]):
        fv = gaussian_source(X.reshape(-1, 2), src_xy[s], width).reshape(ne, 3)
        proj = np.einsum("eab,eb->ea", Me_loc, fv)
        for c in range(2):
            B[dof(np.arange(ne)[:, None], np.arange(3)[None], c).ravel(), s] = proj.ravel()
    coords = np.repeat(cell.astype(np.int32), 6, axis=0)
    return Problem(A=_finish(A), b=np.ascontiguousarray(B[:, 0] if B.shape[1] == 1 else B), coords=coords,
                   name=f"elastic_sipg_p1_{N}x{N}",
                   meta=dict(N=N, omega=omega, lam=lam_e, mu=mu_e, rho=rho, cs=cs, cp=cp, elem=elem, xy=xy,
                             sources=src_xy, area=area))
