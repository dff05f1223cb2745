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
    std::vector<int32_t> blist_h;             // copy of the tree's B lists (new numbering)
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

    int32_t max_mi = 0, max_mb = 0;

    // task queue of the apply (apply.cu): entries (flags | kind | node, a, b),
    // its dependency groups (level schedule), per-node completion requirements
    // [6][nnodes], slots of the diagonal partial products, and a sticky error
    // word set when a bounded wait of the persistent kernel gives up
    int32_t* d_sched = nullptr;                 // [QW * sched_n], 16-byte aligned entries
    int64_t sched_n = 0;
    std::vector<int64_t> sched_groups;
    int32_t sched_ngather = 0;
    int32_t sched_grid = 0;
    int32_t sched_vlen = 0;
    int32_t* d_need = nullptr;
    int32_t* d_wdesc = nullptr;               // warp-node descriptors (8 ints per node)
    int32_t* d_sublist = nullptr;             // bottom subtrees: node lists by level
    int32_t* d_sched_dep = nullptr;           // per task: counter words, count | requirements (2 x int4)
    int32_t sched_sub_level = 0;              // first level handled by subtree tasks
    int32_t sched_warp_level = 0;             // first level handled a warp per node
    int64_t dpart_total = 0;
    int32_t* d_apply_err = nullptr;

    // compressed tier (Alg. 3.4 above the switching level): low-rank R ~ X R(J, :)
    // per node: X (m_i x k, ld m_i) followed by R(J, :)^T (m_b x k, ld m_b), in
    // device buffers of the compression rounds; lr_pending queues the fronts
    // whose R waits for the batch at the end of the factorization
    int32_t L_hss = -1;                       // levels <= L_hss compress S; < L_hss also R
    std::vector<void*> lr_bufs;
    // side streams of the row-ID launches for a caller that owns its own (a
    // second host thread); null: the library's per-device pool
    cudaStream_t side_streams[4] = {};
    std::vector<int32_t> lr_pending;

    // multi right-hand-side apply (multi.cu): the (node, first row) of every
    // 64-row tile, up-sweep tiles of all levels then down-sweep tiles, and
    // each level's range in both
    int2* d_mjobs = nullptr;
    std::vector<int64_t> mj_up_off, mj_dn_off;
    // low-rank nodes of the multi apply: (node, first row, T offset) tiles
    // per level of the four products t = X^T u(I), u(B) += RJt t,
    // t = RJt^T z(B), z(I) += X t; T scratch elements (k x 32 per node)
    int4* d_mlr = nullptr;
    std::vector<int64_t> ml_off[4];
    int64_t ml_t_total = 0;
    std::vector<uint64_t> lr_ptr;             // per node, 0 = dense R
    std::vector<int32_t> lr_k;
    uint64_t* d_lr_ptr = nullptr;
    int32_t* d_lr_k = nullptr;
    int32_t* d_lr_list = nullptr;             // low-rank nodes grouped by level
    std::vector<int64_t> lr_off_l, lr_cnt;    // per level
    // each low-rank node's slot for the apply's per-chunk partial products
    // (ceil(max(m_i, m_b) / LR_CHUNK) x k values)
    std::vector<int64_t> lr_toff;
    int64_t lr_t_total = 0;
    int32_t kmax = 0;
    int32_t hss_rounds_max = 0;

    // ULV of HSS(A_ii) strictly above the switching level (opts.ulv): one
    // record per HSS node of each such front; the apply's diagonal step of
    // those fronts is the ULV solve (ulv.cu, apply.cu)
    struct UlvRec {
        int32_t s;                  // tree node
        int32_t lo, hi;             // leaf: rows of the front's HSS order; else -1
        int32_t m, k, ne, kt;       // block, basis width, eliminated, remaining
        int32_t ka, kb;             // inner: children's basis widths
        int32_t parent, c1, c2;     // records (-1 = none)
        int32_t level, leaf, root;
        uint64_t Mup, W, Mm, E, Dinv;   // device addresses of the solve data
    };
    bool ulv = false;
    std::vector<UlvRec> ulv_recs;
    std::vector<int32_t> ulv_root_of;       // per tree node: its root record, -1 = dense A_ii^{-1}
    std::vector<int64_t> ulv_ord_off;       // per tree node: offset of its HSS order in ulv_ord
    std::vector<int32_t> ulv_ord;           // HSS order of I^s (position -> index in I^s)
    std::vector<void*> ulv_bufs;
    int32_t* d_ulv_ord = nullptr;
    void* d_ulvdev = nullptr;               // device records of the apply (apply.cu)
    int64_t ulv_scratch = 0;                // apply scratch elements of the ULV vectors
    int64_t ulv_bytes = 0;                  // solve data streamed per apply
    double hss_ms = 0.0;

    double factor_ms = 0.0;
    int64_t launches = 0;
    double class_ms[8] = {0};
    int64_t class_launches[8] = {0};
    double update_flops = 0.0;
    double tc_flops = 0.0;                    // real flops of the tensor-core front products
    double host_setup_ms = 0.0;               // host time from the call's entry to the first launch
    double host_tail_ms = 0.0;                // host time from the last kernel's completion to the return
    int64_t apply_bytes = 0;
    int64_t dev_bytes = 0;

    int32_t info(int s, int f) const { return node_info[(size_t)s * NODE_NF + f]; }
    int32_t m_i(int s) const { return info(s, 5); }
    int32_t m_b(int s) const { return info(s, 7); }
};

constexpr int APPLY_ROWS = 64;   // rows per apply task
constexpr int LR_CHUNK = 256;    // input rows per low-rank dot task

// Compress the Schur complements (and, strictly above the switching level,
// the Gauss transforms R) of the fronts on tree level `level`, which have
// just been eliminated densely.  Defined in hss.cu.
ndhss_status hss_compress_level(FactorData& F, const Tree& t, int level, const ndhss_factor_opts& o,
                                cudaStream_t st);
// Low-rank compression of the Gauss transforms R queued by hss_compress_level,
// every level in one batch.  Defined in hss.cu.
ndhss_status hss_lowrank_pending(FactorData& F, const ndhss_factor_opts& o, cudaStream_t st);
// Compress the interior blocks (already gathered in HSS order into aii,
// node s's block at aii_off[s], ld m_i) of the ULV fronts of tree level
// `level` and ULV-factor them.  Defined in hss.cu.
ndhss_status hss_ulv_level(FactorData& F, const Tree& t, int level, void* aii, const std::vector<int64_t>& aii_off,
                           const ndhss_factor_opts& o, cudaStream_t st);

// Outer pivot block of the two-level Gauss-Jordan sweep on the tensor cores.
constexpr int TC_KB2 = 128;
// Whether a level whose largest interior block has mi_max unknowns takes the
// two-level sweep with tensor-core block exchanges; tcgemm.cu.
bool tc_front_path(const FactorData& F, int64_t mi_max);
// The exchange of the outer pivot block starting at pivot k0 (its slab of
// columns [k0, k0 + TC_KB2) already swept, the row interchanges applied to
// every column) on every other column of the fronts of `nodes`, as one
// tcgen05 GEMM with K = the block's width; tcgemm.cu.
ndhss_status tc_block_exchange(FactorData& F, const std::vector<int>& nodes, int k0, DevStatus* d_status,
                               cudaStream_t st);

// Input and output of one apply chosen on the device (by the kernel before
// it on the stream): the apply kernels read x and y here at their start and
// return at once while *skip is nonzero.
struct ApplyInd {
    const void* x;
    void* y;
    const int32_t* skip;
};

ndhss_status apply_device(const FactorData& F, int32_t nrhs, const void* d_x, int64_t ldx,
                          void* d_y, int64_t ldy, void* d_work, cudaStream_t st, const ApplyInd* ind = nullptr);
size_t apply_work_bytes(const FactorData& F);
// Builds and uploads the dataflow queue once the factor (and its low-rank
// tier) is complete; defined in apply.cu.
ndhss_status build_apply_schedule(FactorData& F, cudaStream_t st);
// Low-rank R of the given (final) fronts on stream st: results to F.lr_ptr /
// F.lr_k (one element per front), device storage and counters to acc, the
// largest rank to *kmax.  Defined in hss.cu.
ndhss_status hss_lowrank_fronts(FactorData& F, const std::vector<int32_t>& fronts, FactorData& acc, int* kmax,
                                const ndhss_factor_opts& o, cudaStream_t st);
// The tile lists of the multi right-hand-side apply.  Defined in multi.cu.
ndhss_status build_multi_plan(FactorData& F, cudaStream_t st);
// NDHSS_ERR_TIMEOUT if an earlier apply of this factorization gave up a wait.
ndhss_status apply_check_error(const FactorData& F, const char* who);

}  // namespace ndhss

struct ndhss_factorization {
    ndhss::FactorData f;
};
