"""Seeded synthetic finite-element inputs (test and benchmark fixtures only).

This module builds the sparse Galerkin systems ``A x = b`` that the
preconditioner is applied to (Section 1, Eq. 1.1): continuous Galerkin P1/P2
discretizations of the Poisson problem (Eq. 4.1) and of the Helmholtz problem
(Eq. 4.2) with a first-order impedance condition, on a uniform triangulation
of the unit square in which every cell is cut by its (+1,+1) diagonal.

It holds none of the preconditioner's arithmetic (no nested dissection, no
fronts, no compression, no Krylov method); both the CPU oracle and the CUDA
path consume its output.  Every random number it draws comes from
``numpy.random.default_rng(seed)``.

Besides ``A`` and ``b`` each problem carries the integer lattice coordinate of
every degree of freedom: vertex ``(a, b)`` of the cell grid sits at lattice
point ``(p*a, p*b)`` and the P2 edge midpoints at the odd lattice points in
between, so one lattice unit is ``h/p``.  The nested dissection boxes are
drawn on that lattice.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """One sparse linear system plus the geometry the tree builder needs."""

    A: sp.csr_matrix          # n x n, float64 or complex128, structurally symmetric
    b: np.ndarray             # right-hand side(s), shape (n,) or (n, nrhs)
    coords: np.ndarray        # int32 [n, 2] lattice coordinates of every DOF
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]


# ----------------------------------------------------------------------------
# reference-element data, derived from the barycentric coordinates
#   l0 = 1 - xi - eta, l1 = xi, l2 = eta
# ----------------------------------------------------------------------------

def _gauss_triangle(order: int):
    """Quadrature on the reference triangle by collapsing the unit square.

    (u, v) in [0,1]^2 maps to (xi, eta) = (u, v (1 - u)) with Jacobian (1 - u);
    a tensor Gauss-Legendre rule with ``order`` points per direction is exact
    for polynomials of degree 2*order - 2 on the triangle.
    """
    t, w = np.polynomial.legendre.leggauss(order)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    U, V = np.meshgrid(t, t, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    xi = U.ravel()
    eta = (V * (1.0 - U)).ravel()
    wt = (WU * WV * (1.0 - U)).ravel()
    return xi, eta, wt


def _basis(p: int, xi: np.ndarray, eta: np.ndarray):
    """Values [nq, nb] and reference gradients [nq, nb, 2] of the Lagrange basis."""
    l0 = 1.0 - xi - eta
    l1 = xi
    l2 = eta
    g0 = np.array([-1.0, -1.0])
    g1 = np.array([1.0, 0.0])
    g2 = np.array([0.0, 1.0])
    nq = xi.size
    if p == 1:
        val = np.stack([l0, l1, l2], axis=1)
        grad = np.broadcast_to(np.stack([g0, g1, g2], axis=0), (nq, 3, 2)).copy()
        return val, grad
    if p == 2:
        L = [l0, l1, l2]
        G = [g0, g1, g2]
        vals = [L[i] * (2.0 * L[i] - 1.0) for i in range(3)]
        grads = [np.outer(4.0 * L[i] - 1.0, G[i]) for i in range(3)]
        for (i, j) in ((0, 1), (1, 2), (2, 0)):       # edge midpoints 3, 4, 5
            vals.append(4.0 * L[i] * L[j])
            grads.append(4.0 * (np.outer(L[j], G[i]) + np.outer(L[i], G[j])))
        return np.stack(vals, axis=1), np.stack(grads, axis=1)
    raise ValueError("p must be 1 or 2")


def _edge_basis(p: int, t: np.ndarray):
    """1D Lagrange basis on an edge: [end0, end1] (+ [mid] for p = 2)."""
    if p == 1:
        return np.stack([1.0 - t, t], axis=1)
    return np.stack([(1.0 - t) * (1.0 - 2.0 * t), t * (2.0 * t - 1.0), 4.0 * t * (1.0 - t)], axis=1)


# ----------------------------------------------------------------------------
# mesh
# ----------------------------------------------------------------------------

def _mesh(Nx: int, Ny: int, p: int):
    """Triangles of the Nx x Ny cell grid on [0,1]^2, as lattice-node ids.

    Returns (elem [ne, nb] node ids, cell [ne, 2] cell index, lattice [nn, 2],
    xy [nn, 2] physical coordinates, Lx, Ly).
    """
    Lx, Ly = p * Nx + 1, p * Ny + 1
    jj, ii = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    lattice = np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.int64)
    xy = lattice.astype(np.float64) / np.array([p * Nx, p * Ny], dtype=np.float64)

    def nid(i, j):
        return j * Lx + i

    bb, aa = np.meshgrid(np.arange(Ny), np.arange(Nx), indexing="ij")
    a = aa.ravel()
    b = bb.ravel()
    v00 = (p * a, p * b)
    v10 = (p * (a + 1), p * b)
    v11 = (p * (a + 1), p * (b + 1))
    v01 = (p * a, p * (b + 1))
    tris = []
    for (P, Q, R) in ((v00, v10, v11), (v00, v11, v01)):     # counter-clockwise
        nodes = [nid(*P), nid(*Q), nid(*R)]
        if p == 2:
            for (U, V) in ((P, Q), (Q, R), (R, P)):
                nodes.append(nid((U[0] + V[0]) // 2, (U[1] + V[1]) // 2))
        tris.append(np.stack(nodes, axis=1))
    # interleave so element 2c is the lower-right and 2c+1 the upper-left triangle of cell c
    ne = 2 * a.size
    elem = np.empty((ne, tris[0].shape[1]), dtype=np.int64)
    elem[0::2] = tris[0]
    elem[1::2] = tris[1]
    cell = np.repeat(np.stack([a, b], axis=1), 2, axis=0)
    return elem, cell, lattice, xy, Lx, Ly


def _boundary_edges(Nx: int, Ny: int, p: int, Lx: int):
    """Boundary edges as node ids [ne, 2 or 3] (ends, then midpoint) plus a side tag."""
    def nid(i, j):
        return j * Lx + i

    edges, side = [], []
    for a in range(Nx):                                  # bottom, top
        for (j, s) in ((0, 0), (p * Ny, 2)):
            e = [nid(p * a, j), nid(p * (a + 1), j)]
            if p == 2:
                e.append(nid(p * a + 1, j))
            edges.append(e)
            side.append(s)
    for b in range(Ny):                                  # left, right
        for (i, s) in ((0, 3), (p * Nx, 1)):
            e = [nid(i, p * b), nid(i, p * (b + 1))]
            if p == 2:
                e.append(nid(i, p * b + 1))
            edges.append(e)
            side.append(s)
    return np.array(edges, dtype=np.int64), np.array(side, dtype=np.int64)


def _edge_cells(Nx, Ny):
    """Cell index (a, b) adjacent to each boundary edge (same order as _boundary_edges)."""
    out = []
    for a in range(Nx):
        out.append((a, 0))
        out.append((a, Ny - 1))
    for b in range(Ny):
        out.append((0, b))
        out.append((Nx - 1, b))
    return np.array(out, dtype=np.int64)


# ----------------------------------------------------------------------------
# assembly
# ----------------------------------------------------------------------------

def assemble(Nx: int, Ny: int, p: int, *, mass_coef=None, impedance_k=None):
    """Assemble K + diag-free mass term + impedance term on the full lattice.

    ``mass_coef`` is a per-element array (or scalar) c_e so that the bilinear
    form is  a(u, v) = int grad u . grad v + c_e int u v - i int_{dOmega} k_e u v,
    the boundary term being present only when ``impedance_k`` (per boundary
    edge, or scalar) is given.  The form is bilinear (no conjugation), so the
    matrix is complex symmetric.  Returns (A_full csr, M_full csr, Medge csr,
    lattice, xy, elem).
    """
    elem, cell, lattice, xy, Lx, Ly = _mesh(Nx, Ny, p)
    nn = lattice.shape[0]
    ne, nb = elem.shape
    xi, eta, wq = _gauss_triangle(4)
    val, grad = _basis(p, xi, eta)                        # [nq, nb], [nq, nb, 2]
    X = xy[elem]                                          # [ne, nb, 2]
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]], axis=2)   # [ne, 2, 2], columns
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    Jinv_T = np.empty_like(J)
    Jinv_T[:, 0, 0] = J[:, 1, 1] / det
    Jinv_T[:, 0, 1] = -J[:, 1, 0] / det
    Jinv_T[:, 1, 0] = -J[:, 0, 1] / det
    Jinv_T[:, 1, 1] = J[:, 0, 0] / det
    area = np.abs(det)
    # K_e[a, b] = sum_q w_q (Jinv_T grad_a) . (Jinv_T grad_b) = sum_{jk} C_e[j, k] Q[j, k, a, b]
    # with C_e = Jinv_T^T Jinv_T (2 x 2 per element) and Q the reference-gradient moments
    Q = np.einsum("q,qaj,qbk->jkab", wq, grad, grad).reshape(4, nb * nb)
    C = np.einsum("eij,eik->ejk", Jinv_T, Jinv_T).reshape(ne, 4)
    Ke = (C @ Q).reshape(ne, nb, nb) * area[:, None, None]
    Me = np.einsum("q,qa,qb->ab", wq, val, val)[None, :, :] * area[:, None, None]

    rows = np.repeat(elem, nb, axis=1).ravel()
    cols = np.tile(elem, (1, nb)).ravel()
    M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(nn, nn)).tocsr()
    vals = Ke.astype(np.complex128 if impedance_k is not None else np.float64)
    if mass_coef is not None:
        c = np.broadcast_to(np.asarray(mass_coef, dtype=np.float64), (ne,))
        vals = vals + Me * c[:, None, None]
    R, C, V = [rows], [cols], [vals.ravel()]
    edges, side = _boundary_edges(Nx, Ny, p, Lx)
    t, w = np.polynomial.legendre.leggauss(4)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    eb = _edge_basis(p, t)
    Em = np.einsum("q,qa,qb->ab", w, eb, eb)               # reference edge mass
    length = np.where((side == 0) | (side == 2), 1.0 / Nx, 1.0 / Ny)
    ke = edges.shape[1]
    er = np.repeat(edges, ke, axis=1).ravel()
    ec = np.tile(edges, (1, ke)).ravel()
    Medge = sp.coo_matrix(((Em[None] * length[:, None, None]).ravel(), (er, ec)), shape=(nn, nn)).tocsr()
    if impedance_k is not None:
        kb = np.broadcast_to(np.asarray(impedance_k, dtype=np.float64), (edges.shape[0],))
        R.append(er)
        C.append(ec)
        V.append((-1j * Em[None] * (length * kb)[:, None, None]).ravel())
    # one COO -> CSR pass: duplicates are summed and structural zeros are kept
    A = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))),
                      shape=(nn, nn)).tocsr()
    A.sort_indices()
    return A, M, Medge, lattice, xy, elem, cell, (edges, side)


def _restrict(A, keep):
    A = A[keep][:, keep].tocsr()
    A.sort_indices()
    return A


def _finish(A):
    A = sp.csr_matrix(A)
    A.indices = A.indices.astype(np.int32)
    A.indptr = A.indptr.astype(np.int32)
    A.sort_indices()
    return A


# ----------------------------------------------------------------------------
# named problems
# ----------------------------------------------------------------------------

def poisson_dirichlet(N: int, p: int = 1, seed: int = 0, f=None) -> Problem:
    """-lap u = f on [0,1]^2 with u = 0 on the boundary (Eq. 4.1), CG Pp.

    Boundary nodes are removed.  By default f_i ~ U[-1, 1] i.i.d. per lattice
    node (drawn on the full lattice from ``seed``) and b = (M f) restricted to
    the interior; a callable ``f(x, y)`` is interpolated instead when given.
    """
    A, M, _, lattice, xy, *_ = assemble(N, N, p)
    Lx = p * N + 1
    interior = ((lattice[:, 0] > 0) & (lattice[:, 0] < Lx - 1)
                & (lattice[:, 1] > 0) & (lattice[:, 1] < Lx - 1))
    keep = np.nonzero(interior)[0]
    if f is None:
        rng = np.random.default_rng(seed)
        fv = rng.uniform(-1.0, 1.0, size=lattice.shape[0])
    else:
        fv = f(xy[:, 0], xy[:, 1])
    b = (M @ fv)[keep]
    return Problem(A=_finish(_restrict(A, keep)), b=np.ascontiguousarray(b),
                   coords=lattice[keep].astype(np.int32), name=f"poisson_p{p}_{N}x{N}",
                   meta=dict(N=N, p=p, seed=seed, xy=xy[keep], h=1.0 / N))


def gaussian_source(xy, xs, width=0.02):
    """Gaussian point source of the given width, peak 1, centred at xs."""
    d2 = (xy[:, 0] - xs[0]) ** 2 + (xy[:, 1] - xs[1]) ** 2
    return np.exp(-d2 / (2.0 * width * width))


def helmholtz_impedance(N: int, p: int, k: float, seed: int = 0, *, nsrc: int = 1,
                        slowness2=None, width: float = 0.02, g=None, f=None) -> Problem:
    """-lap u - k^2 m u = f on [0,1]^2 with du/dn - i k sqrt(m) u = g (Eq. 4.2).

    Weak form  int grad u . grad v - k^2 int m u v - i k int_{dOmega} sqrt(m) u v
    = int f v + int_{dOmega} g v, bilinear so A is complex symmetric.
    ``g(x, y, nx, ny)`` receives the outward normal of the edge it is integrated on.
    ``slowness2`` (squared slowness m) is a per-element array or None (m = 1).
    By default f is a Gaussian source of width ``width`` at x_s ~ U[0.1, 0.9]^2
    drawn from ``seed`` (``nsrc`` sources give ``nsrc`` right-hand sides),
    interpolated at the nodes and multiplied by the mass matrix.
    """
    elem, cell, lattice, xy, Lx, Ly = _mesh(N, N, p)
    ne = elem.shape[0]
    m_e = np.ones(ne) if slowness2 is None else np.asarray(slowness2, dtype=np.float64)
    edges, side = _boundary_edges(N, N, p, Lx)
    ecell = _edge_cells(N, N)
    # an edge's coefficient is the element's (both triangles of a cell share m)
    m_edge = m_e[2 * (ecell[:, 1] * N + ecell[:, 0])]
    A, M, Medge, lattice, xy, *_ = assemble(N, N, p, mass_coef=-(k * k) * m_e,
                                            impedance_k=k * np.sqrt(m_edge))
    rng = np.random.default_rng(seed)
    if f is None and g is None:
        xs = rng.uniform(0.1, 0.9, size=(nsrc, 2))
        F = np.stack([gaussian_source(xy, xs[s], width) for s in range(nsrc)], axis=1)
        b = (M @ F).astype(np.complex128)
        meta_src = xs
    else:
        b = np.zeros(lattice.shape[0], dtype=np.complex128)
        if f is not None:
            b = b + M @ f(xy[:, 0], xy[:, 1])
        if g is not None:
            # edge by edge, so each side uses its own outward normal
            normals = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])
            t, w = np.polynomial.legendre.leggauss(4)
            t = 0.5 * (t + 1.0)
            w = 0.5 * w
            eb = _edge_basis(p, t)
            Em = np.einsum("q,qa,qb->ab", w, eb, eb)
            length = np.where((side == 0) | (side == 2), 1.0 / N, 1.0 / N)
            nrm = normals[side]
            gv = g(xy[edges, 0], xy[edges, 1], nrm[:, None, 0], nrm[:, None, 1])   # [ne, ke]
            contrib = np.einsum("ab,eb->ea", Em, gv) * length[:, None]
            np.add.at(b, edges.ravel(), contrib.ravel())
        meta_src = None
    if b.ndim == 2 and b.shape[1] == 1:
        b = b[:, 0]
    return Problem(A=_finish(A), b=np.ascontiguousarray(b), coords=lattice.astype(np.int32),
                   name=f"helmholtz_p{p}_{N}x{N}_k{k:g}",
                   meta=dict(N=N, p=p, k=k, seed=seed, xy=xy, h=1.0 / N, sources=meta_src))


def helmholtz_blocks(N: int, k: float, m_blocks, *, p: int = 1, seed: int = 0, nsrc: int = 1,
                     width: float = 0.02, src_xy=None) -> Problem:
    """Helmholtz with squared slowness m piecewise constant on an nb x nb grid
    of blocks (``m_blocks`` [nb, nb], block (i, j) covering cells with
    i = a * nb // N, j = b * nb // N), impedance on all sides, Gaussian
    sources (at ``src_xy`` [nsrc, 2] or drawn from ``seed``).

    Besides A(m) and b, meta holds what the derivative of A with respect to
    one block's m needs:  dA/dm_j = -k^2 sum_{e in j} M_e - i k / (2 sqrt(m_j))
    sum_{edges in j} E_e, with ``elem`` / ``Me`` the element DOFs and unit
    mass matrices, ``eblk`` their blocks, ``edges`` / ``Ee`` / ``edge_blk``
    the boundary edges' DOFs, unit edge mass matrices and blocks.
    """
    mb = np.asarray(m_blocks, dtype=np.float64)
    nb = mb.shape[0]
    elem, cell, lattice, xy, Lx, Ly = _mesh(N, N, p)
    eblk = (cell[:, 0] * nb // N) * nb + (cell[:, 1] * nb // N)
    m_e = mb.ravel()[eblk]
    if src_xy is None:
        src_xy = np.random.default_rng(seed).uniform(0.1, 0.9, size=(nsrc, 2))
    src_xy = np.asarray(src_xy, dtype=np.float64)
    P = helmholtz_impedance(N, p, k, seed, slowness2=m_e, f=lambda x, y: 0.0 * x)     # b set below
    _, M, *_ = assemble(N, N, p)
    F = np.stack([gaussian_source(xy, src_xy[s], width) for s in range(src_xy.shape[0])], axis=1)
    b = (M @ F).astype(np.complex128)
    # element data
    xi, eta, wq = _gauss_triangle(4)
    val, _ = _basis(p, xi, eta)
    X = xy[elem]
    det = (X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1]) - (X[:, 2, 0] - X[:, 0, 0]) * (X[:, 1, 1] - X[:, 0, 1])
    Me = np.einsum("q,qa,qb->ab", wq, val, val)[None, :, :] * np.abs(det)[:, None, None]
    edges, side = _boundary_edges(N, N, p, Lx)
    ecell = _edge_cells(N, N)
    edge_blk = (ecell[:, 0] * nb // N) * nb + (ecell[:, 1] * nb // N)
    t, w = np.polynomial.legendre.leggauss(4)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    eb = _edge_basis(p, t)
    Em = np.einsum("q,qa,qb->ab", w, eb, eb)
    Ee = Em[None] * np.full(edges.shape[0], 1.0 / N)[:, None, None]
    P.b = np.ascontiguousarray(b[:, 0] if b.shape[1] == 1 else b)
    P.name = f"helmholtz_blocks_p{p}_{N}x{N}_k{k:g}_nb{nb}"
    P.meta.update(m_blocks=mb, nb=nb, elem=elem, Me=Me, eblk=eblk, edges=edges, Ee=Ee, edge_blk=edge_blk,
                  sources=src_xy, k=k)
    return P


def helmholtz_macro(Nx: int, Ny: int, c_blocks, *, p: int = 1, ppw: float = 10.0, src_xy=None, nsrc: int = 32,
                    seed: int = 0, width: float = 0.02) -> Problem:
    """Helmholtz with impedance on all sides on an Nx x Ny cell grid of
    [0,1]^2 (cells h_x = 1/Nx by h_y = 1/Ny), wave speed c piecewise constant
    on the macro blocks of ``c_blocks`` [mb, mb] (cell (a, b) in block
    (a mb // Nx, b mb // Ny)), angular frequency omega = 2 pi / (ppw max(h_x, h_y))
    so that the slowest wave (c >= 1) has ``ppw`` points per wavelength, and
    local wavenumber k = omega / c in the mass and the impedance terms.
    Right-hand sides: Gaussian sources of the given width at ``src_xy``
    [nsrc, 2] (default: drawn ~ U[0.1, 0.9]^2 from ``seed``), interpolated
    and multiplied by the mass matrix.
    """
    cb = np.asarray(c_blocks, dtype=np.float64)
    mb = cb.shape[0]
    elem, cell, lattice, xy, Lx, Ly = _mesh(Nx, Ny, p)
    omega = 2.0 * np.pi / (ppw * max(1.0 / Nx, 1.0 / Ny))
    c_e = cb[cell[:, 0] * mb // Nx, cell[:, 1] * mb // Ny]
    ecell = _edge_cells(Nx, Ny)
    c_edge = cb[ecell[:, 0] * mb // Nx, ecell[:, 1] * mb // Ny]
    A, M, *_ = assemble(Nx, Ny, p, mass_coef=-(omega / c_e) ** 2, impedance_k=omega / c_edge)
    if src_xy is None:
        src_xy = np.random.default_rng(seed).uniform(0.1, 0.9, size=(nsrc, 2))
    src_xy = np.asarray(src_xy, dtype=np.float64)
    F = np.stack([gaussian_source(xy, src_xy[s], width) for s in range(src_xy.shape[0])], axis=1)
    b = (M @ F).astype(np.complex128)
    return Problem(A=_finish(A), b=np.ascontiguousarray(b), coords=lattice.astype(np.int32),
                   name=f"helmholtz_macro_p{p}_{Nx}x{Ny}",
                   meta=dict(Nx=Nx, Ny=Ny, p=p, omega=omega, c_blocks=cb, xy=xy, sources=src_xy))


def helmholtz_batch(count: int, seed: int = 0, *, nmin: int = 64, nmax: int = 256, nsrc: int = 32,
                    mb: int = 8, cmin: float = 1.0, cmax: float = 3.0, p: int = 1) -> list:
    """``count`` independent Helmholtz problems (helmholtz_macro) of the
    batched workload: problem s draws from seed + s its grid
    N_x, N_y ~ U{nmin..nmax}, its wave speeds c ~ U[cmin, cmax] on mb x mb
    macro blocks and its ``nsrc`` source positions ~ U[0.1, 0.9]^2."""
    out = []
    for s in range(count):
        rng = np.random.default_rng([seed, s])
        Nx, Ny = (int(v) for v in rng.integers(nmin, nmax + 1, size=2))
        cb = rng.uniform(cmin, cmax, size=(mb, mb))
        src = rng.uniform(0.1, 0.9, size=(nsrc, 2))
        out.append(helmholtz_macro(Nx, Ny, cb, p=p, src_xy=src))
    return out
