"""Differentiation through the preconditioned solve (adjoint state).

``HelmholtzSolve.apply(m, B, model)`` returns X with A(m) X = B for the
Helmholtz model of Sec. 4 (Eq. 4.2) whose squared slowness m is piecewise
constant on blocks: the forward pass factors A(m) with ``ndhss_factor`` and
solves every column with ``ndhss_gmres``.  The backward pass needs
Lambda = A^{-H} G; A is complex symmetric (A^T = A), so
A^{-H} G = conj(A^{-1} conj(G)) and the adjoint solve (``ndhss_gmres`` with
``conj_transpose``) reuses the forward pass's factor and GMRES.  Then (PyTorch's conjugate-Wirtinger convention,
dJ = Re(G^H dX)):

    grad_B   = Lambda
    grad_m_j = -Re sum_s lambda_s^H (dA/dm_j) x_s,
    dA/dm_j  = -k^2 sum_{e in block j} M_e - i k / (2 sqrt(m_j)) sum_{boundary edges in j} E_e,

with the block sums of the element quadratic forms computed on the device
by ``ndhss_elem_qform``.  The matrix A(m) itself comes from the model's
``assemble`` callable (the problem's discretisation, not this library).
"""
from __future__ import annotations

import numpy as np
import torch

from . import ndhss


class HelmholtzBlockModel:
    """What the solve and its derivative need about the discretisation:
    ``assemble(m) -> scipy CSR A(m)`` for the flattened block values m, the
    nested-dissection tree of A's pattern (fixed in m), the wavenumber k, the
    elements (DOFs ``elem`` [ne, nloc], unit mass matrices ``Me``, blocks
    ``eblk``) and the boundary edges (``edges``, ``Ee``, ``edge_blk``)."""

    def __init__(self, tree, assemble, k, elem, Me, eblk, edges, Ee, edge_blk, nblk, opts=None, tol=1e-10,
                 device="cuda"):
        self.tree = tree
        self.assemble = assemble
        self.k = float(k)
        self.nblk = int(nblk)
        self.opts = opts if opts is not None else ndhss.make_factor_opts(prec=ndhss.NDHSS_FP64)
        self.tol = tol
        self.device = device
        self.elems = self._groups(elem, Me, eblk)
        self.edges = self._groups(edges, Ee, edge_blk)

    def _groups(self, idx, mats, blk):
        order = np.argsort(blk, kind="stable")
        goff = np.zeros(self.nblk + 1, dtype=np.int32)
        np.add.at(goff, np.asarray(blk)[order] + 1, 1)
        goff = np.cumsum(goff).astype(np.int32)
        dev = self.device
        return dict(goff=torch.from_numpy(goff).to(dev),
                    idx=torch.from_numpy(np.ascontiguousarray(np.asarray(idx)[order], dtype=np.int32)).to(dev),
                    mats=torch.from_numpy(np.ascontiguousarray(np.asarray(mats)[order], dtype=np.float64)).to(dev),
                    nloc=int(np.asarray(idx).shape[1]))

    def qform(self, grp, lam, x):
        q = torch.empty(self.nblk, dtype=torch.complex128, device=self.device)
        return ndhss.ndhss_elem_qform(grp["goff"], grp["nloc"], grp["idx"], grp["mats"], lam, x, q)

    def coefficient_gradient(self, m, lam, x):
        """-Re(lam^H dA/dm_j x) for every block j (one right-hand side)."""
        qM = self.qform(self.elems, lam, x)
        qE = self.qform(self.edges, lam, x)
        k = self.k
        dA = -(k * k) * qM - 1j * k / (2.0 * torch.sqrt(m)) * qE
        return -dA.real


def _solve_columns(f, M, B, tol, adjoint=False):
    X = torch.empty_like(B)
    for s in range(B.shape[1]):
        x = torch.zeros(B.shape[0], dtype=B.dtype, device=B.device)
        st = ndhss.ndhss_gmres(f, M.rowptr, M.col, M.vals, B[:, s].contiguous(), x, tol=tol, conj_transpose=adjoint)
        if not st["converged"]:
            raise RuntimeError(f"ndhss_gmres did not converge: {st}")
        X[:, s] = x
    return X


class HelmholtzSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, B, model):
        one = B.dim() == 1
        Bc = (B.unsqueeze(1) if one else B).to(device=model.device, dtype=torch.complex128)
        A = model.assemble(m.detach().cpu().numpy().astype(np.float64))
        M = ndhss.DeviceCSR(A)
        f = ndhss.ndhss_factor(model.tree, M.vtype, M.rowptr, M.col, M.vals, model.opts)
        X = _solve_columns(f, M, Bc, model.tol)
        ctx.model, ctx.f, ctx.M, ctx.one = model, f, M, one
        ctx.save_for_backward(m, X)
        return X[:, 0] if one else X

    @staticmethod
    def backward(ctx, G):
        m, X = ctx.saved_tensors
        model = ctx.model
        G2 = (G.unsqueeze(1) if ctx.one else G).resolve_conj().to(torch.complex128)
        # A^{-H} G by the library's adjoint solve (conj(A^{-1} conj(G)) for complex symmetric A)
        Lam = _solve_columns(ctx.f, ctx.M, G2.contiguous(), model.tol, adjoint=True)
        md = m.detach().to(device=model.device, dtype=torch.float64)
        gm = torch.zeros(model.nblk, dtype=torch.float64, device=model.device)
        for s in range(X.shape[1]):
            gm += model.coefficient_gradient(md, Lam[:, s].contiguous(), X[:, s].contiguous())
        gB = Lam[:, 0] if ctx.one else Lam
        return gm.to(device=m.device, dtype=m.dtype), gB, None
