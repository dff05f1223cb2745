// C ABI glue: version, error reporting and the tree handle.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <new>

#include "internal.h"

namespace ndhss {

static thread_local char g_err[1024] = "";

ndhss_status set_error(ndhss_status code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = '\0'; }

static std::atomic<int64_t> g_launches{0};

void note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

}  // namespace ndhss

extern "C" {

const char* ndhss_version(void) { return "ndhss 0.1 (sm_103a)"; }

const char* ndhss_last_error(void) { return ndhss::g_err; }

int64_t ndhss_kernel_launches(void) { return ndhss::g_launches.load(); }

ndhss_status ndhss_build_tree(int32_t n, const int32_t* coords, const int32_t* rowptr, const int32_t* col,
                              int32_t leaf_size, ndhss_tree** out) {
    ndhss::clear_error();
    if (!out) return ndhss::set_error(NDHSS_ERR_INVALID_ARG, "ndhss_build_tree: out is NULL");
    *out = nullptr;
    auto* t = new (std::nothrow) ndhss_tree();
    if (!t) return ndhss::set_error(NDHSS_ERR_OOM, "ndhss_build_tree: host allocation failed");
    ndhss_status rc;
    try {
        rc = ndhss::build_tree_impl(n, coords, rowptr, col, leaf_size, &t->t);
    } catch (const std::bad_alloc&) {
        rc = ndhss::set_error(NDHSS_ERR_OOM, "ndhss_build_tree: host allocation failed");
    } catch (...) {
        rc = ndhss::set_error(NDHSS_ERR_INTERNAL, "ndhss_build_tree: unexpected exception");
    }
    if (rc != NDHSS_OK) {
        delete t;
        return rc;
    }
    *out = t;
    return NDHSS_OK;
}

ndhss_status ndhss_build_tree_batched(int32_t nsys, const int32_t* n, const int32_t* const* coords,
                                      const int32_t* const* rowptr, const int32_t* const* col, int32_t leaf_size,
                                      ndhss_tree** out) {
    ndhss::clear_error();
    if (!out) return ndhss::set_error(NDHSS_ERR_INVALID_ARG, "ndhss_build_tree_batched: out is NULL");
    *out = nullptr;
    if (nsys < 1 || !n || !coords || !rowptr || !col)
        return ndhss::set_error(NDHSS_ERR_INVALID_ARG, "ndhss_build_tree_batched: need nsys >= 1 and the four arrays");
    auto* t = new (std::nothrow) ndhss_tree();
    if (!t) return ndhss::set_error(NDHSS_ERR_OOM, "ndhss_build_tree_batched: host allocation failed");
    ndhss_status rc = NDHSS_OK;
    try {
        std::vector<ndhss::Tree> parts(nsys);
        for (int32_t s = 0; s < nsys && rc == NDHSS_OK; ++s) {
            rc = ndhss::build_tree_impl(n[s], coords[s], rowptr[s], col[s], leaf_size, &parts[s]);
            if (rc != NDHSS_OK) {
                const std::string msg = ndhss_last_error();
                rc = ndhss::set_error(rc, "ndhss_build_tree_batched: problem %d: %s", s, msg.c_str());
            }
        }
        if (rc == NDHSS_OK) rc = ndhss::join_trees(parts, &t->t);
    } catch (const std::bad_alloc&) {
        rc = ndhss::set_error(NDHSS_ERR_OOM, "ndhss_build_tree_batched: host allocation failed");
    } catch (...) {
        rc = ndhss::set_error(NDHSS_ERR_INTERNAL, "ndhss_build_tree_batched: unexpected exception");
    }
    if (rc != NDHSS_OK) {
        delete t;
        return rc;
    }
    *out = t;
    return NDHSS_OK;
}

ndhss_status ndhss_tree_sizes(const ndhss_tree* t, int32_t* nnodes, int32_t* depth, int64_t* nnz, int64_t* sum_mb) {
    ndhss::clear_error();
    if (!t) return ndhss::set_error(NDHSS_ERR_INVALID_ARG, "ndhss_tree_sizes: NULL tree");
    if (nnodes) *nnodes = t->t.nnodes;
    if (depth) *depth = t->t.depth;
    if (nnz) *nnz = t->t.nnz;
    if (sum_mb) *sum_mb = (int64_t)t->t.blist.size();
    return NDHSS_OK;
}

ndhss_status ndhss_tree_export(const ndhss_tree* th, int32_t* perm, int32_t* node_info, int32_t* blist, int32_t* emap,
                               int32_t* e_off, int32_t* e_row, int32_t* e_col, int32_t* e_idx) {
    ndhss::clear_error();
    if (!th) return ndhss::set_error(NDHSS_ERR_INVALID_ARG, "ndhss_tree_export: NULL tree");
    const auto& t = th->t;
    auto cp = [](int32_t* dst, const std::vector<int32_t>& v) {
        if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(int32_t));
    };
    cp(perm, t.perm);
    cp(node_info, t.node_info);
    cp(blist, t.blist);
    cp(emap, t.emap);
    cp(e_off, t.e_off);
    cp(e_row, t.e_row);
    cp(e_col, t.e_col);
    cp(e_idx, t.e_idx);
    return NDHSS_OK;
}

void ndhss_tree_destroy(ndhss_tree* t) { delete t; }

}  // extern "C"
