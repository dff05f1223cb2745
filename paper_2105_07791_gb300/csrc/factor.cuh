// Device-resident factorization P = L D R shared by the factor, apply and
// Krylov translation units.
#pragma once

#include <vector>

#include "common.cuh"

namespace ndhss {

// Storage of node sigma's front (m = m_i + m_b, column-major, ld = m) after
// elimination of its first m_i unknowns (Sec. 3.1, Eq. 3.2 - 3.5), with
// P the row interchanges chosen inside A_ii and sigma(j) the original row
// now at position j:
//
//      [ A_ii^{-1} P^T    |  R = -A_ii^{-1} A_ib ]      R: Eq. 3.3b
//      [ -L P^T           |  S                   ]      L: Eq. 3.3a, S: Eq. 3.5
//
// so (A_ii^{-1} y)_i = sum_j X(i, j) y_{sigma(j)} and
// (L y)_k = -sum_j BL(k, j) y_{sigma(j)}.
struct FactorData {
    int32_t vtype = 0, prec = 0;
    int32_t n = 0, nnodes = 0, depth = 0;
    size_t esize = 0;                         // bytes per stored front element
    std::vector<int32_t> node_info;           // copy of the tree's node table
    std::vector<int64_t> foff;                // front offset (elements) per node
    std::vector<std::vector<int32_t>> levels; // levels[l] = node ids on level l
    int64_t front_elems = 0;

    int32_t* d_node = nullptr;
    int64_t* d_foff = nullptr;
    int32_t* d_blist = nullptr;
    int32_t* d_perm = nullptr;
    int32_t* d_sigma = nullptr;               // [n], block of node s at i_off(s)
    int32_t* d_ipiv = nullptr;                // [n]
    void* d_front = nullptr;

    // apply work lists: pairs (node, first row) of 64-row tasks
    int32_t* d_tasks = nullptr;
    std::vector<int64_t> up_off, up_cnt;      // per level
    std::vector<int64_t> dn_off, dn_cnt;      // per level
    int64_t diag_off = 0, diag_cnt = 0;
    int32_t max_mi = 0, max_mb = 0;

    double factor_ms = 0.0;
    int64_t launches = 0;
    double class_ms[8] = {0};
    int64_t class_launches[8] = {0};
    double update_flops = 0.0;
    int64_t apply_bytes = 0;
    int64_t dev_bytes = 0;

    int32_t info(int s, int f) const { return node_info[(size_t)s * NODE_NF + f]; }
    int32_t m_i(int s) const { return info(s, 5); }
    int32_t m_b(int s) const { return info(s, 7); }
};

constexpr int APPLY_ROWS = 64;   // rows per apply task

ndhss_status apply_device(const FactorData& F, int32_t nrhs, const void* d_x, int64_t ldx,
                          void* d_y, int64_t ldy, void* d_work, cudaStream_t st);
size_t apply_work_bytes(const FactorData& F);

}  // namespace ndhss

struct ndhss_factorization {
    ndhss::FactorData f;
};
