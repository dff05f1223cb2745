// Forest of independent problems (the batched workload of many meshes):
// every problem's own nested-dissection tree (Def. 3.1, built by the same
// rule as ndhss_build_tree), joined side by side into one tree whose levels
// hold the nodes of all problems.  The matrix it describes is block diagonal,
// diag(A_0, ..., A_{S-1}), with problem s's DOFs at offset sum_{s' < s} n_s'
// and its CSR entries at offset sum_{s' < s} nnz_s'; node ids, DOF positions,
// B lists and entry indices are shifted accordingly, roots sit on level 0, so
// one level of the factorization and of the apply covers every problem.
// Host-only integer code.
#include "internal.h"

#include <algorithm>

namespace ndhss {

ndhss_status join_trees(const std::vector<Tree>& parts, Tree* T) {
    int64_t n = 0, nn = 0, nnz = 0, nb = 0;
    int depth = 0;
    for (const Tree& p : parts) {
        n += p.n;
        nn += p.nnodes;
        nnz += p.nnz;
        nb += (int64_t)p.blist.size();
        depth = std::max(depth, p.depth);
    }
    if (n > INT32_MAX || nn > INT32_MAX || nnz > INT32_MAX || nb > INT32_MAX)
        return set_error(NDHSS_ERR_INVALID_ARG, "build_tree_batched: the batch exceeds int32 sizes");
    T->n = (int32_t)n;
    T->nnodes = (int32_t)nn;
    T->nnz = nnz;
    T->depth = depth;
    T->node_info.clear();
    T->perm.clear();
    T->iperm.clear();
    T->blist.clear();
    T->emap.clear();
    T->e_row.clear();
    T->e_col.clear();
    T->e_idx.clear();
    T->coords.clear();
    T->e_off.assign(1, 0);
    T->node_info.reserve((size_t)nn * NODE_NF);
    T->perm.reserve(n);
    T->iperm.reserve(n);
    int32_t dof = 0, node = 0, boff = 0, eoff = 0;
    for (const Tree& p : parts) {
        for (int s = 0; s < p.nnodes; ++s) {
            int32_t ni[NODE_NF];
            for (int f = 0; f < NODE_NF; ++f) ni[f] = p.info(s, f);
            for (int f = 1; f <= 3; ++f)
                if (ni[f] >= 0) ni[f] += node;                  // parent, children
            ni[4] += dof;                                       // i_off
            ni[6] += boff;                                      // b_off
            T->node_info.insert(T->node_info.end(), ni, ni + NODE_NF);
            T->e_off.push_back(eoff + p.e_off[s + 1]);
        }
        for (int32_t v : p.perm) T->perm.push_back(v + dof);
        for (int32_t v : p.iperm) T->iperm.push_back(v + dof);
        for (int32_t v : p.blist) T->blist.push_back(v + dof);
        T->emap.insert(T->emap.end(), p.emap.begin(), p.emap.end());
        T->e_row.insert(T->e_row.end(), p.e_row.begin(), p.e_row.end());
        T->e_col.insert(T->e_col.end(), p.e_col.begin(), p.e_col.end());
        for (int32_t v : p.e_idx) T->e_idx.push_back(v + eoff);
        T->coords.insert(T->coords.end(), p.coords.begin(), p.coords.end());
        dof += p.n;
        node += p.nnodes;
        boff += (int32_t)p.blist.size();
        eoff += (int32_t)p.nnz;
    }
    return NDHSS_OK;
}

}  // namespace ndhss
