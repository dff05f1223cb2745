// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cstdio>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/ndhss.h"

namespace ndhss {

constexpr int NODE_NF = 14;   // level, parent, child0, child1, i_off, m_i, b_off, m_b, x0, x1, y0, y1, axis, cut

struct Tree {
    int32_t n = 0, nnodes = 0, depth = 0;
    int64_t nnz = 0;
    std::vector<int32_t> node_info;   // [nnodes * NODE_NF]
    std::vector<int32_t> perm, iperm, blist, emap, e_off, e_row, e_col, e_idx;
    std::vector<int32_t> coords;      // [n * 2] lattice coordinates (original numbering)

    int32_t info(int s, int f) const { return node_info[(size_t)s * NODE_NF + f]; }
    int32_t level(int s) const { return info(s, 0); }
    int32_t parent(int s) const { return info(s, 1); }
    int32_t child(int s, int c) const { return info(s, 2 + c); }
    int32_t i_off(int s) const { return info(s, 4); }
    int32_t m_i(int s) const { return info(s, 5); }
    int32_t b_off(int s) const { return info(s, 6); }
    int32_t m_b(int s) const { return info(s, 7); }
};

// Records a formatted message for ndhss_last_error() and returns `code`.
ndhss_status set_error(ndhss_status code, const char* fmt, ...);
void clear_error();
void note_launches(int64_t k);

// Runs an entry point's body so that no C++ exception crosses the C ABI: a
// failed host allocation becomes NDHSS_ERR_OOM, any other exception
// NDHSS_ERR_INTERNAL (with its message).  Memory that the interrupted call
// held is not reclaimed on that path.
template <typename Fn>
ndhss_status guarded(const char* who, Fn&& fn) noexcept {
    try {
        return fn();
    } catch (const std::bad_alloc&) {
        return set_error(NDHSS_ERR_OOM, "%s: host allocation failed", who);
    } catch (const std::exception& e) {
        return set_error(NDHSS_ERR_INTERNAL, "%s: %s", who, e.what());
    } catch (...) {
        return set_error(NDHSS_ERR_INTERNAL, "%s: unexpected exception", who);
    }
}

ndhss_status build_tree_impl(int32_t n, const int32_t* coords, const int32_t* rowptr,
                             const int32_t* col, int32_t leaf_size, Tree* T);
// The forest of independent problems' trees (batch_tree.cpp).
ndhss_status join_trees(const std::vector<Tree>& parts, Tree* T);

}  // namespace ndhss

struct ndhss_tree {
    ndhss::Tree t;
};
