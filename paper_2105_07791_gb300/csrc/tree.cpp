// Box nested dissection and elimination tree (Def. 3.1, Fig. 3, Sec. 3.1,
// numbering of Sec. 3.3 / Fig. 4).  Host-only integer code.
//
// Rules (all integer arithmetic, deterministic):
//  * boxes are half-open lattice rectangles [x0,x1) x [y0,y1); the root is the
//    bounding box of all coordinates;
//  * a box with <= leaf_size DOFs (or a single lattice point) is a leaf,
//    otherwise its longer side (x on ties) is halved at (lo + hi) >> 1, the low
//    half being the first child; nodes are numbered in post-order;
//  * BL(box) = DOFs of the box with a structural neighbour outside it;
//    leaf: I = box \ BL, sorted by DOF id; inner node sigma with children
//    mu, nu: F(k) = BL(k) \ BL(sigma) sorted by (coordinate along the cut,
//    distance to the cut, id), G(k) = BL(k) n BL(sigma) sorted by (cyclic
//    counter-clockwise perimeter position on sigma's box starting where the
//    cut meets the bottom (x-split) or right (y-split) side, distance to the
//    nearest side, id); B^k = [F(k); G(k)], I^sigma = [F(mu); F(nu)];
//  * every entry A(i,j) enters the front of LCA(leaf(i), leaf(j)).
#include "internal.h"

#include <algorithm>
#include <numeric>
#include <tuple>

namespace ndhss {

namespace {

struct BuildNode {
    int x0, x1, y0, y1;
    int level = 0, parent = -1, child0 = -1, child1 = -1, axis = -1, cut = 0;
    std::vector<int> dofs;   // sorted original ids
    std::vector<int> bl;     // BL(box), in dofs order
};

struct Builder {
    int n;
    const int32_t* coords;
    int leaf_size;
    std::vector<int64_t> nptr;
    std::vector<int> nidx;
    std::vector<BuildNode> nodes;

    int cx(int d) const { return coords[2 * (size_t)d]; }
    int cy(int d) const { return coords[2 * (size_t)d + 1]; }
    int cc(int d, int axis) const { return coords[2 * (size_t)d + axis]; }

    int split(int x0, int x1, int y0, int y1, std::vector<int>&& dofs, int level) {
        BuildNode rec;
        rec.x0 = x0; rec.x1 = x1; rec.y0 = y0; rec.y1 = y1;
        rec.level = level;
        int W = x1 - x0, H = y1 - y0;
        if ((int64_t)dofs.size() > leaf_size && (W > 1 || H > 1)) {
            int axis = (W >= H) ? 0 : 1;
            int lo = axis == 0 ? x0 : y0, hi = axis == 0 ? x1 : y1;
            int c = (lo + hi) >> 1;
            std::vector<int> low, high;
            for (int d : dofs) (cc(d, axis) < c ? low : high).push_back(d);
            int k0, k1;
            if (axis == 0) {
                k0 = split(x0, c, y0, y1, std::move(low), level + 1);
                k1 = split(c, x1, y0, y1, std::move(high), level + 1);
            } else {
                k0 = split(x0, x1, y0, c, std::move(low), level + 1);
                k1 = split(x0, x1, c, y1, std::move(high), level + 1);
            }
            rec.axis = axis;
            rec.cut = c;
            rec.child0 = k0;
            rec.child1 = k1;
        }
        rec.dofs = std::move(dofs);
        int id = (int)nodes.size();
        nodes.push_back(std::move(rec));
        if (nodes[id].child0 >= 0) {
            nodes[nodes[id].child0].parent = id;
            nodes[nodes[id].child1].parent = id;
        }
        return id;
    }
};

}  // namespace

ndhss_status build_tree_impl(int32_t n, const int32_t* coords, const int32_t* rowptr,
                             const int32_t* col, int32_t leaf_size, Tree* T) {
    if (n < 1 || leaf_size < 1 || !coords || !rowptr || !col)
        return set_error(NDHSS_ERR_INVALID_ARG, "build_tree: need n >= 1, leaf_size >= 1 and non-NULL arrays");
    int64_t nnz = rowptr[n];
    if (rowptr[0] != 0 || nnz < 0) return set_error(NDHSS_ERR_INVALID_ARG, "build_tree: bad rowptr");
    for (int i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) return set_error(NDHSS_ERR_INVALID_ARG, "build_tree: rowptr not monotone");
    for (int64_t k = 0; k < nnz; ++k)
        if (col[k] < 0 || col[k] >= n) return set_error(NDHSS_ERR_INVALID_ARG, "build_tree: column index out of range");

    T->coords.assign(coords, coords + 2 * (size_t)n);
    Builder B;
    B.n = n;
    B.coords = coords;
    B.leaf_size = leaf_size;

    // symmetrised structural pattern without the diagonal, unique neighbours
    {
        std::vector<int64_t> cnt(n + 1, 0);
        for (int i = 0; i < n; ++i)
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
                if (col[k] != i) { cnt[i + 1]++; cnt[col[k] + 1]++; }
        for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
        std::vector<int> tmp(cnt[n]);
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
                if (col[k] != i) { tmp[pos[i]++] = col[k]; tmp[pos[col[k]]++] = i; }
        B.nptr.assign(n + 1, 0);
        B.nidx.reserve(tmp.size());
        for (int i = 0; i < n; ++i) {
            auto b = tmp.begin() + cnt[i], e = tmp.begin() + cnt[i + 1];
            std::sort(b, e);
            auto u = std::unique(b, e);
            for (auto it = b; it != u; ++it) B.nidx.push_back(*it);
            B.nptr[i + 1] = (int64_t)B.nidx.size();
        }
    }

    int minx = coords[0], maxx = coords[0], miny = coords[1], maxy = coords[1];
    for (int d = 0; d < n; ++d) {
        minx = std::min(minx, B.cx(d)); maxx = std::max(maxx, B.cx(d));
        miny = std::min(miny, B.cy(d)); maxy = std::max(maxy, B.cy(d));
    }
    std::vector<int> all(n);
    std::iota(all.begin(), all.end(), 0);
    int root = B.split(minx, maxx + 1, miny, maxy + 1, std::move(all), 0);
    auto& nodes = B.nodes;
    const int nn = (int)nodes.size();
    (void)root;

    // boundary layers
    std::vector<char> inBL;  // scratch, per node
    for (auto& rec : nodes) {
        rec.bl.clear();
        for (int d : rec.dofs) {
            bool out = false;
            for (int64_t k = B.nptr[d]; k < B.nptr[d + 1] && !out; ++k) {
                int j = B.nidx[k];
                int x = B.cx(j), y = B.cy(j);
                out = (x < rec.x0) || (x >= rec.x1) || (y < rec.y0) || (y >= rec.y1);
            }
            if (out) rec.bl.push_back(d);
        }
    }

    std::vector<std::vector<int>> Ilist(nn), Blist(nn);
    std::vector<int64_t> nF(nn, 0);
    std::vector<char> mark(n, 0);
    for (int s = 0; s < nn; ++s) {
        auto& rec = nodes[s];
        if (rec.child0 < 0) {
            std::vector<int> inner;
            size_t j = 0;
            for (int d : rec.dofs) {
                if (j < rec.bl.size() && rec.bl[j] == d) { ++j; continue; }
                inner.push_back(d);
            }
            std::sort(inner.begin(), inner.end());
            Ilist[s] = std::move(inner);
            continue;
        }
        for (int d : rec.bl) mark[d] = 1;
        const int axis = rec.axis, cut = rec.cut;
        const int X0 = rec.x0, X1 = rec.x1 - 1, Y0 = rec.y0, Y1 = rec.y1 - 1;
        const int64_t W = X1 - X0, H = Y1 - Y0, Pl = 2 * W + 2 * H;
        const int64_t ps = axis == 0 ? (int64_t)(cut - X0) : W + (cut - Y0);
        std::vector<int> Iparts;
        int which = 0;
        for (int k : {rec.child0, rec.child1}) {
            std::vector<std::tuple<int64_t, int64_t, int>> Fk, Gk;
            for (int d : nodes[k].bl) {
                if (!mark[d]) {
                    int64_t t = B.cc(d, 1 - axis);
                    int64_t a = B.cc(d, axis);
                    int64_t dist = which == 0 ? (int64_t)(cut - 1) - a : a - cut;
                    Fk.emplace_back(t, dist, d);
                } else {
                    int64_t x = B.cx(d), y = B.cy(d);
                    int64_t db = y - Y0, dr = X1 - x, dt = Y1 - y, dl = x - X0;
                    int64_t dmin = std::min(std::min(db, dr), std::min(dt, dl));
                    int64_t p;
                    if (db == dmin) p = x - X0;
                    else if (dr == dmin) p = W + (y - Y0);
                    else if (dt == dmin) p = W + H + (X1 - x);
                    else p = 2 * W + H + (Y1 - y);
                    int64_t q = Pl > 0 ? (((p - ps) % Pl) + Pl) % Pl : 0;
                    Gk.emplace_back(q, dmin, d);
                }
            }
            std::sort(Fk.begin(), Fk.end());
            std::sort(Gk.begin(), Gk.end());
            auto& Bk = Blist[k];
            Bk.clear();
            for (auto& e : Fk) { Bk.push_back(std::get<2>(e)); Iparts.push_back(std::get<2>(e)); }
            for (auto& e : Gk) Bk.push_back(std::get<2>(e));
            nF[k] = (int64_t)Fk.size();
            ++which;
        }
        for (int d : rec.bl) mark[d] = 0;
        Ilist[s] = std::move(Iparts);
    }

    // permutation and node arrays
    T->n = n;
    T->nnodes = nn;
    T->node_info.assign((size_t)nn * NODE_NF, 0);
    std::vector<int64_t> m_i(nn), m_b(nn), i_off(nn), b_off(nn);
    int64_t acc_i = 0, acc_b = 0;
    for (int s = 0; s < nn; ++s) {
        m_i[s] = (int64_t)Ilist[s].size();
        m_b[s] = (int64_t)Blist[s].size();
        i_off[s] = acc_i; acc_i += m_i[s];
        b_off[s] = acc_b; acc_b += m_b[s];
    }
    if (acc_i != n) return set_error(NDHSS_ERR_INTERNAL, "build_tree: elimination sets do not partition the DOFs");
    T->perm.resize(n);
    T->iperm.assign(n, -1);
    for (int s = 0; s < nn; ++s)
        for (int64_t k = 0; k < m_i[s]; ++k) T->perm[i_off[s] + k] = Ilist[s][k];
    for (int i = 0; i < n; ++i) {
        if (T->iperm[T->perm[i]] != -1) return set_error(NDHSS_ERR_INTERNAL, "build_tree: duplicate DOF");
        T->iperm[T->perm[i]] = i;
    }
    T->blist.resize(acc_b);
    for (int s = 0; s < nn; ++s)
        for (int64_t k = 0; k < m_b[s]; ++k) T->blist[b_off[s] + k] = T->iperm[Blist[s][k]];

    // extend-add map: position of each B^kappa row in the parent's front
    T->emap.assign(acc_b, 0);
    for (int s = 0; s < nn; ++s) {
        auto& rec = nodes[s];
        if (rec.child0 < 0) continue;
        std::vector<std::pair<int, int>> bpos;   // (new index, position in B^s)
        bpos.reserve(m_b[s]);
        for (int64_t k = 0; k < m_b[s]; ++k) bpos.emplace_back(T->blist[b_off[s] + k], (int)k);
        std::sort(bpos.begin(), bpos.end());
        int64_t base = 0;
        for (int k : {rec.child0, rec.child1}) {
            for (int64_t r = 0; r < m_b[k]; ++r) {
                int64_t out;
                if (r < nF[k]) {
                    out = base + r;
                } else {
                    int g = T->blist[b_off[k] + r];
                    auto it = std::lower_bound(bpos.begin(), bpos.end(), std::make_pair(g, -1));
                    if (it == bpos.end() || it->first != g)
                        return set_error(NDHSS_ERR_INTERNAL, "build_tree: child boundary DOF missing in parent front (node %d)", s);
                    out = m_i[s] + it->second;
                }
                T->emap[b_off[k] + r] = (int32_t)out;
            }
            base += nF[k];
        }
    }

    // node info
    for (int s = 0; s < nn; ++s) {
        auto& rec = nodes[s];
        int32_t* ni = &T->node_info[(size_t)s * NODE_NF];
        ni[0] = rec.level; ni[1] = rec.parent; ni[2] = rec.child0; ni[3] = rec.child1;
        ni[4] = (int32_t)i_off[s]; ni[5] = (int32_t)m_i[s]; ni[6] = (int32_t)b_off[s]; ni[7] = (int32_t)m_b[s];
        ni[8] = rec.x0; ni[9] = rec.x1; ni[10] = rec.y0; ni[11] = rec.y1; ni[12] = rec.axis; ni[13] = rec.cut;
    }

    // entries -> LCA fronts
    std::vector<int> leaf_of(n, -1), elim(n, -1);
    for (int s = 0; s < nn; ++s) {
        if (nodes[s].child0 < 0)
            for (int d : nodes[s].dofs) leaf_of[d] = s;
        for (int64_t k = 0; k < m_i[s]; ++k) elim[Ilist[s][k]] = s;
    }
    std::vector<std::pair<int64_t, int>> keys;   // (node * n + dof, position in front)
    keys.reserve(acc_b);
    for (int s = 0; s < nn; ++s)
        for (int64_t k = 0; k < m_b[s]; ++k)
            keys.emplace_back((int64_t)s * n + Blist[s][k], (int)(m_i[s] + k));
    std::sort(keys.begin(), keys.end());
    auto front_pos = [&](int d, int s, int32_t* out) -> bool {
        if (elim[d] == s) { *out = (int32_t)(T->iperm[d] - i_off[s]); return true; }
        int64_t key = (int64_t)s * n + d;
        auto it = std::lower_bound(keys.begin(), keys.end(), std::make_pair(key, -1));
        if (it == keys.end() || it->first != key) return false;
        *out = it->second;
        return true;
    };
    std::vector<int> lca(nnz);
    std::vector<int64_t> counts(nn + 1, 0);
    for (int i = 0; i < n; ++i) {
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            int a = leaf_of[i], b = leaf_of[col[k]];
            while (a != b) {
                int la = nodes[a].level, lb = nodes[b].level;
                if (la >= lb) a = nodes[a].parent;
                if (lb >= la) b = nodes[b].parent;
            }
            lca[k] = a;
            counts[a + 1]++;
        }
    }
    for (int s = 0; s < nn; ++s) counts[s + 1] += counts[s];
    T->e_off.resize(nn + 1);
    for (int s = 0; s <= nn; ++s) T->e_off[s] = (int32_t)counts[s];
    T->e_row.resize(nnz);
    T->e_col.resize(nnz);
    T->e_idx.resize(nnz);
    std::vector<int64_t> fill(counts.begin(), counts.end() - 1);
    for (int i = 0; i < n; ++i) {
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            int s = lca[k];
            int64_t p = fill[s]++;
            if (!front_pos(i, s, &T->e_row[p]) || !front_pos(col[k], s, &T->e_col[p]))
                return set_error(NDHSS_ERR_INVALID_ARG,
                                 "build_tree: entry (%d,%d) outside its front; pattern not structurally symmetric?",
                                 i, col[k]);
            T->e_idx[p] = (int32_t)k;
        }
    }
    int depth = 0;
    for (auto& rec : nodes) depth = std::max(depth, rec.level);
    T->depth = depth;
    T->nnz = nnz;
    return NDHSS_OK;
}

}  // namespace ndhss
