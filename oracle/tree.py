"""Oracle: box nested dissection and the elimination tree (Def. 3.1, Sec. 3.1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` leg of ``bench.py`` may import this package; the product
path never does.

The tree is built by recursive bisection of boxes on the integer DOF lattice
(Fig. 3, Sec. 4.1 "subsequent subdivisions", Sec. 4.5 "aspect ratio of the
boxes close to one").  Everything here is integer arithmetic, so the CUDA
library's host builder must reproduce it bit for bit.  Readings of points the
paper leaves open:

* Box: half-open integer rectangle [x0,x1) x [y0,y1); the root is the bounding
  box of all lattice coordinates (hi = max + 1).
* A box with at most ``leaf_size`` DOFs (or a single lattice point) is a leaf;
  otherwise its longer side is halved (x on ties) at mid = (lo + hi) >> 1, the
  low half being the first child mu, the high half the second child nu.
  Nodes are numbered in post-order (Fig. 1).
* BL(box) = DOFs of the box with a structural neighbour outside the box (the
  pattern is symmetrised; explicit zeros count).
  Leaf: I = box \\ BL(box).  Inner node sigma with children mu, nu:
  I^sigma = (BL(mu) u BL(nu)) \\ BL(sigma)   and   B^kappa = BL(kappa)
  (a superset of the coupled ancestor DOFs of Sec. 3.1, exact since the
  extra rows are merely zero couplings).
* Order (the numbering that keeps A~_ii^(mu,nu) of low HSS rank, Sec. 3.3,
  and exposes S_ii^(mu) in the parent-conforming block of Fig. 4):
  for a child kappa of sigma,
     F(kappa) = BL(kappa) \\ BL(sigma)  sorted by (coordinate along sigma's
                cut, distance to the cut, DOF id),
     G(kappa) = BL(kappa) n BL(sigma)   sorted by (cyclic counter-clockwise
                perimeter position on sigma's box, starting where the cut
                meets the bottom side (x-split) or the right side (y-split);
                distance to the nearest side; DOF id),
     B^kappa  = [F(kappa); G(kappa)],
     I^sigma  = [F(mu); F(nu)].
  Leaf interiors are ordered by DOF id.  The front of sigma is [I^sigma; B^sigma].
* The permutation lists I^sigma for sigma in post-order (new -> old).
* Every entry A(i, j) enters exactly one front: that of the lowest common
  ancestor of the leaves holding i and j (Eq. 3.2 for a leaf, the A~ blocks
  of Eq. 3.4 otherwise).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

NODE_FIELDS = ("level", "parent", "child0", "child1", "i_off", "m_i", "b_off", "m_b",
               "x0", "x1", "y0", "y1", "axis", "cut")
NF = len(NODE_FIELDS)


@dataclass
class Tree:
    n: int
    node_info: np.ndarray      # int32 [nnodes, NF]
    perm: np.ndarray           # int32 [n], new -> old
    iperm: np.ndarray          # int32 [n], old -> new
    blist: np.ndarray          # int32 [sum m_b], B^sigma as new indices, node after node
    emap: np.ndarray           # int32 [sum m_b], position of each B^kappa entry in the parent front
    e_off: np.ndarray          # int32 [nnodes + 1]
    e_row: np.ndarray          # int32 [nnz] front-local row of each entry
    e_col: np.ndarray          # int32 [nnz] front-local column
    e_idx: np.ndarray          # int32 [nnz] CSR position of the entry
    leaf_of: np.ndarray        # int32 [n] leaf node holding each DOF (old numbering)
    coords: np.ndarray = None  # int64 [n, 2] lattice coordinates (old numbering)

    @property
    def nnodes(self) -> int:
        return self.node_info.shape[0]

    def f(self, name: str) -> np.ndarray:
        return self.node_info[:, NODE_FIELDS.index(name)]

    @property
    def depth(self) -> int:
        return int(self.f("level").max())

    def I(self, s: int) -> np.ndarray:
        """I^s as new indices (a contiguous range)."""
        o, m = self.node_info[s, 4], self.node_info[s, 5]
        return np.arange(o, o + m)

    def B(self, s: int) -> np.ndarray:
        """B^s as new indices."""
        o, m = self.node_info[s, 6], self.node_info[s, 7]
        return self.blist[o:o + m]

    def emap_of(self, s: int) -> np.ndarray:
        o, m = self.node_info[s, 6], self.node_info[s, 7]
        return self.emap[o:o + m]

    def children(self, s: int):
        c0, c1 = self.node_info[s, 2], self.node_info[s, 3]
        return [c for c in (c0, c1) if c >= 0]

    def levels(self):
        """Node ids grouped by level, deepest level first."""
        lev = self.f("level")
        return [np.nonzero(lev == l)[0] for l in range(self.depth, -1, -1)]


def symmetric_pattern(n: int, rowptr: np.ndarray, col: np.ndarray):
    """Neighbour lists of the symmetrised structural pattern without the diagonal."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    r = np.concatenate([rows, col])
    c = np.concatenate([col, rows])
    keep = r != c
    P = sp.csr_matrix((np.ones(int(keep.sum()), dtype=np.int8), (r[keep], c[keep])), shape=(n, n))
    P.sum_duplicates()
    P.sort_indices()
    return P.indptr.astype(np.int64), P.indices.astype(np.int64)


def _boundary_layer(dofs, box, coords, nptr, nidx):
    """BL(box): the DOFs of ``dofs`` with a neighbour outside the half-open box."""
    if dofs.size == 0:
        return np.zeros(0, dtype=bool)
    x0, x1, y0, y1 = box
    cnt = nptr[dofs + 1] - nptr[dofs]
    owner = np.repeat(np.arange(dofs.size), cnt)
    starts = np.repeat(nptr[dofs], cnt)
    within = np.arange(owner.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    nb = nidx[starts + within]
    cx = coords[nb, 0]
    cy = coords[nb, 1]
    outside = (cx < x0) | (cx >= x1) | (cy < y0) | (cy >= y1)
    return np.bincount(owner[outside], minlength=dofs.size) > 0


def _perimeter(xs, ys, box, axis, cut):
    """(cyclic counter-clockwise perimeter position, distance to nearest side)."""
    x0, x1, y0, y1 = box
    X0, X1, Y0, Y1 = x0, x1 - 1, y0, y1 - 1
    W, H = X1 - X0, Y1 - Y0
    db, dr, dt, dl = ys - Y0, X1 - xs, Y1 - ys, xs - X0
    dmin = np.minimum(np.minimum(db, dr), np.minimum(dt, dl))
    p = np.where(db == dmin, xs - X0,
        np.where(dr == dmin, W + (ys - Y0),
        np.where(dt == dmin, W + H + (X1 - xs), 2 * W + H + (Y1 - ys))))
    Pl = 2 * W + 2 * H
    ps = (cut - X0) if axis == 0 else (W + (cut - Y0))
    q = np.mod(p - ps, Pl) if Pl > 0 else np.zeros_like(p)
    return q, dmin


def build_tree(coords: np.ndarray, rowptr: np.ndarray, col: np.ndarray, leaf_size: int) -> Tree:
    """Box nested dissection (Fig. 3) producing the post-ordered elimination tree."""
    coords = np.asarray(coords, dtype=np.int64)
    n = coords.shape[0]
    if n < 1 or leaf_size < 1:
        raise ValueError("need n >= 1 and leaf_size >= 1")
    nptr, nidx = symmetric_pattern(n, rowptr, col)

    nodes = []            # in post-order: dict(box, level, parent, children, dofs, bl, axis, cut)

    def split(box, dofs, level):
        x0, x1, y0, y1 = box
        W, H = x1 - x0, y1 - y0
        rec = dict(box=box, level=level, dofs=dofs, children=[], axis=-1, cut=0)
        if dofs.size > leaf_size and (W > 1 or H > 1):
            axis = 0 if W >= H else 1
            lo, hi = (x0, x1) if axis == 0 else (y0, y1)
            c = (lo + hi) >> 1
            low = dofs[coords[dofs, axis] < c]
            high = dofs[coords[dofs, axis] >= c]
            if axis == 0:
                bl, bh = (x0, c, y0, y1), (c, x1, y0, y1)
            else:
                bl, bh = (x0, x1, y0, c), (x0, x1, c, y1)
            k0 = split(bl, low, level + 1)
            k1 = split(bh, high, level + 1)
            rec.update(axis=axis, cut=c, children=[k0, k1])
        rec["id"] = len(nodes)
        nodes.append(rec)
        for k in rec["children"]:
            nodes[k]["parent"] = rec["id"]
        return rec["id"]

    root_box = (int(coords[:, 0].min()), int(coords[:, 0].max()) + 1,
                int(coords[:, 1].min()), int(coords[:, 1].max()) + 1)
    root = split(root_box, np.arange(n, dtype=np.int64), 0)
    nodes[root]["parent"] = -1
    nn = len(nodes)

    for rec in nodes:
        rec["blmask"] = _boundary_layer(rec["dofs"], rec["box"], coords, nptr, nidx)
        rec["bl"] = rec["dofs"][rec["blmask"]]

    # F(kappa), G(kappa) for every non-root node, ordered by the parent's cut
    I_list = [None] * nn
    B_list = [None] * nn
    nF = np.zeros(nn, dtype=np.int64)
    for rec in nodes:
        s = rec["id"]
        if not rec["children"]:
            inner = rec["dofs"][~rec["blmask"]]
            I_list[s] = np.sort(inner)
            continue
        par_bl = set(rec["bl"].tolist())
        axis, cut = rec["axis"], rec["cut"]
        parts = []
        for which, k in enumerate(rec["children"]):
            blk = nodes[k]["bl"]
            in_par = np.fromiter((d in par_bl for d in blk.tolist()), dtype=bool, count=blk.size)
            Fk = blk[~in_par]
            Gk = blk[in_par]
            # F: (coordinate along the cut, distance to the cut, id)
            t = coords[Fk, 1 - axis]
            a = coords[Fk, axis]
            d = (cut - 1) - a if which == 0 else a - cut
            Fk = Fk[np.lexsort((Fk, d, t))]
            # G: (cyclic perimeter position on sigma's box, depth, id)
            q, dm = _perimeter(coords[Gk, 0], coords[Gk, 1], rec["box"], axis, cut)
            Gk = Gk[np.lexsort((Gk, dm, q))]
            B_list[k] = np.concatenate([Fk, Gk])
            nF[k] = Fk.size
            parts.append(Fk)
        I_list[s] = np.concatenate(parts)
    B_list[root] = np.zeros(0, dtype=np.int64)

    # permutation: I^sigma in post-order
    m_i = np.array([I_list[s].size for s in range(nn)], dtype=np.int64)
    m_b = np.array([B_list[s].size for s in range(nn)], dtype=np.int64)
    i_off = np.concatenate([[0], np.cumsum(m_i)[:-1]])
    b_off = np.concatenate([[0], np.cumsum(m_b)[:-1]])
    perm = np.concatenate(I_list).astype(np.int64)
    if perm.size != n or np.unique(perm).size != n:
        raise RuntimeError("elimination sets do not partition the DOFs")
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    blist = np.concatenate([iperm[B_list[s]] for s in range(nn)]) if m_b.sum() else np.zeros(0, np.int64)

    # position of each B^kappa entry in the parent's front
    emap = np.zeros(int(m_b.sum()), dtype=np.int64)
    for rec in nodes:
        s = rec["id"]
        if not rec["children"]:
            continue
        Bpos = {int(g): i for i, g in enumerate(blist[b_off[s]:b_off[s] + m_b[s]].tolist())}
        base = 0
        for k in rec["children"]:
            Bk = blist[b_off[k]:b_off[k] + m_b[k]]
            out = np.empty(m_b[k], dtype=np.int64)
            f = nF[k]
            out[:f] = base + np.arange(f)
            out[f:] = m_i[s] + np.array([Bpos[int(g)] for g in Bk[f:].tolist()], dtype=np.int64)
            emap[b_off[k]:b_off[k] + m_b[k]] = out
            base += f

    # entries: each A(i, j) goes to the front of LCA(leaf(i), leaf(j))
    level = np.array([rec["level"] for rec in nodes], dtype=np.int64)
    parent = np.array([rec["parent"] for rec in nodes], dtype=np.int64)
    leaf_of = np.empty(n, dtype=np.int64)
    for rec in nodes:
        if not rec["children"]:
            leaf_of[rec["dofs"]] = rec["id"]
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    nnz = col.size
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    a = leaf_of[rows].copy()
    b = leaf_of[col].copy()
    for _ in range(2 * (level.max() + 1)):
        ua = level[a] > level[b]
        a[ua] = parent[a[ua]]
        ub = level[b] > level[a]
        b[ub] = parent[b[ub]]
        both = (a != b) & (level[a] == level[b])
        a[both] = parent[a[both]]
        b[both] = parent[b[both]]
    if np.any(a != b):
        raise RuntimeError("LCA search did not converge")
    lca = a
    # front position of DOF d (old id) at node s
    key_node = np.concatenate([np.repeat(np.arange(nn), m_b)])
    key_dof = perm[blist] if blist.size else np.zeros(0, np.int64)
    key_pos = np.concatenate([m_i[s] + np.arange(m_b[s]) for s in range(nn)]) if blist.size else np.zeros(0, np.int64)
    keys = key_node * n + key_dof
    order = np.argsort(keys, kind="stable")
    keys_sorted = keys[order]
    elim = np.repeat(np.arange(nn), m_i)[iperm]          # node eliminating each DOF (old id)

    def front_pos(d, s):
        pos = np.empty(d.size, dtype=np.int64)
        isI = elim[d] == s
        pos[isI] = iperm[d[isI]] - i_off[s[isI]]
        q = ~isI
        kk = s[q] * n + d[q]
        loc = np.searchsorted(keys_sorted, kk)
        if np.any(loc >= keys_sorted.size) or np.any(keys_sorted[np.minimum(loc, keys_sorted.size - 1)] != kk):
            raise RuntimeError("entry outside its front: tree is not well separated")
        pos[q] = key_pos[order[loc]]
        return pos

    e_r = front_pos(rows, lca)
    e_c = front_pos(col, lca)
    eorder = np.lexsort((np.arange(nnz), lca))
    e_off = np.concatenate([[0], np.cumsum(np.bincount(lca, minlength=nn))])

    node_info = np.zeros((nn, NF), dtype=np.int64)
    for rec in nodes:
        s = rec["id"]
        ch = rec["children"] + [-1, -1]
        node_info[s] = [rec["level"], rec["parent"], ch[0], ch[1], i_off[s], m_i[s], b_off[s], m_b[s],
                        *rec["box"], rec["axis"], rec["cut"]]
    i32 = lambda v: np.ascontiguousarray(v, dtype=np.int32)
    return Tree(n=n, node_info=i32(node_info), perm=i32(perm), iperm=i32(iperm), blist=i32(blist),
                emap=i32(emap), e_off=i32(e_off), e_row=i32(e_r[eorder]), e_col=i32(e_c[eorder]),
                e_idx=i32(eorder), leaf_of=i32(leaf_of), coords=coords)
