/*
 * ndhss.h -- C ABI of a GB300 (sm_103a) nested-dissection preconditioner
 * with dense and HSS-compressed fronts (Bonev & Hesthaven, "A hierarchical
 * preconditioner for wave problems in quasilinear complexity").
 *
 * The library solves A x = b for a sparse Galerkin matrix A (Sec. 1,
 * Eq. 1.1) with GMRES on P^{-1} A x = P^{-1} b (Eq. 1.2), where
 * P = L D R (Eq. 3.1) is built front by front over a box nested dissection.
 *
 * Conventions that hold for every entry point:
 *  - All functions return an ndhss_status; on failure ndhss_last_error()
 *    returns a thread-local message (with node / level where known).  No
 *    function aborts, throws across the ABI or traps the GPU.
 *  - "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *    device memory of the current device.  The caller owns every buffer it
 *    passes; the library never keeps a caller pointer after returning.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *    Device work is ordered on it.  Functions that return host-side results
 *    (ndhss_factor, ndhss_gmres, ndhss_factor_get_block) synchronise it.
 *  - Matrices are CSR with int32 row pointers and column indices in the
 *    ORIGINAL numbering, values float64 (NDHSS_R64) or interleaved
 *    complex128 (NDHSS_C128).  A must be structurally symmetric.
 *  - Dense blocks are column-major.  Complex numbers are interleaved
 *    (re, im) pairs.
 *  - Opaque handles are owned by the library and released with the
 *    matching _destroy function.
 */
#ifndef NDHSS_H
#define NDHSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NDHSS_OK = 0,
    NDHSS_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, inconsistent input        */
    NDHSS_ERR_OOM = 2,           /* device or host allocation failed                    */
    NDHSS_ERR_SINGULAR = 3,      /* exact zero pivot in some A_ii (node in message)     */
    NDHSS_ERR_RANK_CAP = 4,      /* HSS compression hit rank_cap before eps_hss         */
    NDHSS_ERR_NOT_CONVERGED = 5, /* GMRES stopped at maxit above tolerance (x is valid) */
    NDHSS_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                       */
    NDHSS_ERR_CUDA = 7,          /* a CUDA runtime call failed (message has the code)   */
    NDHSS_ERR_INTERNAL = 8
} ndhss_status;

typedef enum { NDHSS_R64 = 0, NDHSS_C128 = 1 } ndhss_vtype;

/* Factor storage / arithmetic.  GMRES vectors, the sparse product and the
 * true residual are always float64 (complex128). */
typedef enum {
    NDHSS_FP64 = 0,      /* fronts in float64 / complex128, FP64 arithmetic           */
    NDHSS_FP32 = 1,      /* fronts in float32 / complex64; R, L, S of the larger fronts
                            on the TF32 tensor cores with each operand split in two
                            rounded TF32 parts (hi*hi + hi*lo + lo*hi, FP32
                            accumulation: FP32-accurate products); the rest FP32  */
    NDHSS_FP32_TF32 = 2, /* as FP32 with one rounded TF32 part per operand          */
    NDHSS_FP32_BF16 = 3  /* as FP32 with two rounded BF16 parts per operand
                            (tcgen05 kind::f16, FP32 accumulation, ~16 bits)         */
} ndhss_prec;

typedef struct ndhss_tree ndhss_tree;
typedef struct ndhss_factorization ndhss_factorization;

typedef struct {
    int32_t prec;               /* ndhss_prec                                          */
    int32_t hss_levels;         /* compress fronts on levels <= depth - hss_levels
                                   (4 = "4 levels above the lowest", Sec. 4);
                                   < 0 disables compression (exact factorization)     */
    double eps_hss;             /* relative HSS tolerance (Eq. 2.7), e.g. 1e-6        */
    int32_t beta;               /* HSS leaf block size (Eq. 2.1), e.g. 64              */
    int32_t k0;                 /* initial rank guess of Alg. A.1, e.g. 32             */
    int32_t r;                  /* rank step / estimator samples of Alg. A.1, e.g. 16  */
    int32_t rank_cap;           /* largest HSS rank allowed, e.g. 512                  */
    int32_t panel;              /* pivot block width of the front kernels, 0 = auto    */
    uint64_t seed;              /* random sampling seed                                */
    int32_t timing;             /* 1: time every kernel class with CUDA events         */
    int32_t ulv;                /* 1: A_ii of the fronts strictly above the switching
                                   level in HSS form (Alg. A.1, ordered along the cut)
                                   with a ULV factorization; the apply's diagonal step
                                   of those fronts is the ULV solve.  0: A_ii^{-1}
                                   formed densely at every level                      */
} ndhss_factor_opts;

typedef struct {
    int32_t restart;            /* Krylov basis length per cycle, e.g. 30              */
    int32_t maxit;              /* total Arnoldi steps allowed, e.g. 300               */
    double tol;                 /* relative residual target, e.g. 1e-8                 */
    int32_t timing;             /* 1: time every apply / SpMV with CUDA events         */
    int32_t conj_transpose;     /* 1: solve A^H x = b on the same factor (the adjoint
                                   solve; A complex symmetric, so x = conj(A^{-1}
                                   conj(b)): b is conjugated into scratch, the solve
                                   runs as usual and x is conjugated on the device;
                                   stats describe ||b - A^H x||).  No effect for real
                                   A.  ndhss_gmres only; 0 otherwise                  */
    double inner;               /* a cycle ends at ||P^{-1} r|| <= inner tol ||P^{-1} b||;
                                   0.1 = one decade below tol, as Sec. 4 stops at 1e-9 */
    double cycle_rtol;          /* a cycle also ends once its residual estimate fell by
                                   this factor (what one reduced-precision apply can
                                   resolve); < 0 = automatic: 1e-3 for FP32 fronts
                                   (a cycle then takes about one Arnoldi step and the
                                   float64 restarts refine), 0 (off) for FP64 fronts.  After a cycle that did
                                   not halve the true residual, later cycles of that
                                   solve end only once their estimate fell by the
                                   reduction the true residual still needs
                                   (0.1 tol / relres, relative to the cycle start)   */
} ndhss_gmres_opts;

typedef struct {
    int32_t iters;              /* Arnoldi steps (products with P^{-1} A)              */
    int32_t cycles;             /* restart cycles                                      */
    int32_t converged;          /* 1 when ||b - A x|| / ||b|| <= tol                   */
    int32_t pad;
    double true_relres;         /* final float64 ||b - A x|| / ||b||                   */
    double precond_relres;      /* last ||P^{-1}(b - A x)|| / ||P^{-1} b|| estimate    */
    int32_t napply, nspmv;      /* preconditioner applies / sparse products issued     */
    double apply_ms, spmv_ms;   /* their summed device time (only when timing = 1)     */
} ndhss_gmres_stats;

typedef struct {
    int64_t n;
    int32_t nnodes, depth;
    int64_t front_elems;        /* sum over nodes of m^2 (dense front storage)        */
    int64_t apply_bytes;        /* bytes of factor data one apply reads                */
    int64_t factor_bytes;       /* device bytes held by the factor                     */
    double factor_ms;           /* device time of the last ndhss_factor (CUDA events)  */
    int32_t kmax;               /* largest rank of any compressed block (0 if none)    */
    int32_t prec;
    int64_t launches;           /* kernels launched by the last ndhss_factor           */
    /* per kernel class (only when opts.timing = 1): summed device ms and launches;
       classes 0 assemble, 1 scatter, 2 panel, 3 prep, 4 update, 5 finalize,
       6 compression (S by Alg. A.1, R by a randomized row ID), 7 tensor-core
       products R, L, S of the larger fronts (operand packing and tcgen05 GEMMs)     */
    double class_ms[8];
    int64_t class_launches[8];
    double update_flops;        /* real flops of the Gauss-Jordan rank-kb updates      */
    double tc_flops;            /* real flops of the tensor-core products R, L, S
                                   (8 per complex multiply-add), counted once per
                                   product whatever the operand split              */
    double host_setup_ms;       /* host time from the call's entry to its first launch
                                   (table uploads, allocations)                     */
    double host_tail_ms;        /* host time from the last factor kernel's completion
                                   to the return (apply schedule and multi-apply plan) */
} ndhss_factor_stats;

/* Library version string (static storage). */
const char* ndhss_version(void);

/* Message of the last failed call on this thread (static per-thread storage). */
const char* ndhss_last_error(void);

/* Number of CUDA kernels the library has launched in this process so far
 * (monotonic; for accounting of device work, e.g. per timed region). */
int64_t ndhss_kernel_launches(void);

/* Measurement aid, no counterpart in the paper: the sustained FMA rate of the
 * current device's CUDA cores in TFLOP/s (two flops per FMA), which = 0 for
 * FP64, 1 for FP32: a kernel of eight independent FMA chains per thread, eight
 * 256-thread CTAs per SM, timed with CUDA events on `stream` (0 = default),
 * best of three launches after a warm-up (tens of ms).  It is the denominator
 * of the rooflines of the kernels bound by plain arithmetic.  *tflops is
 * written on success.  Errors: NDHSS_ERR_INVALID_ARG (another `which`, null
 * pointer), NDHSS_ERR_CUDA (allocation or launch failure). */
ndhss_status ndhss_measure_fma_peak(int32_t which, void* stream, double* tflops);

/*
 * ndhss_build_tree -- box nested dissection and elimination tree
 * (Def. 3.1; boxes of Fig. 3; Sec. 3.1 for I^sigma and B^sigma; Sec. 3.3 and
 * Fig. 4 for the numbering inside the fronts).  Host only, integer only,
 * deterministic.
 *   n          number of DOFs (>= 1)
 *   coords     host int32 [n][2], integer lattice coordinate of every DOF
 *              (DOFs of one DG element share one coordinate)
 *   rowptr,col host int32 CSR pattern of A (n+1, nnz); explicit zeros count
 *   leaf_size  a box with at most leaf_size DOFs is a leaf (e.g. 64)
 *   out        receives a new tree handle
 * Inputs are copied.  Returns INVALID_ARG for bad sizes or indices.
 */
ndhss_status ndhss_build_tree(int32_t n, const int32_t* coords, const int32_t* rowptr,
                              const int32_t* col, int32_t leaf_size, ndhss_tree** out);

/*
 * ndhss_build_tree_batched -- many independent problems as one forest (the
 * batched workload: many meshes of uneven size, Sec. 3.1's tree per mesh).
 * Problem s (0 <= s < nsys) is given exactly as to ndhss_build_tree
 * (n[s], coords[s], rowptr[s], col[s]; host arrays); its tree is built by the
 * same rule, and the trees are joined side by side: node ids, DOF positions,
 * B lists and entry indices shifted, every root on level 0, depth = the
 * deepest problem's.  The tree describes the block-diagonal matrix
 * diag(A_0, ..., A_{nsys-1}): problem s's DOFs occupy rows
 * [sum_{s'<s} n[s'], sum_{s'<=s} n[s']) and its CSR entries follow those of
 * the problems before it, so ndhss_factor / ndhss_apply / ndhss_gmres_batched
 * take the problems' CSR arrays concatenated (rowptr shifted by the entry
 * offset, col by the DOF offset, values in problem order).  One level of the
 * factorization then eliminates the fronts of all problems together.
 * Inputs are copied.  INVALID_ARG names the failing problem.
 */
ndhss_status ndhss_build_tree_batched(int32_t nsys, const int32_t* n, const int32_t* const* coords,
                                      const int32_t* const* rowptr, const int32_t* const* col,
                                      int32_t leaf_size, ndhss_tree** out);

/* ndhss_tree_sizes -- sizes of the arrays ndhss_tree_export fills: node
 * count, tree depth (levels 0 .. depth), number of CSR entries and the summed
 * length of all B^sigma lists (any output pointer may be NULL).  Host only.
 * INVALID_ARG when t is NULL. */
ndhss_status ndhss_tree_sizes(const ndhss_tree* t, int32_t* nnodes, int32_t* depth,
                              int64_t* nnz, int64_t* sum_mb);

/*
 * ndhss_tree_export -- copy the tree into caller-owned host arrays, for
 * inspection and bit-exact comparison (any pointer may be NULL to skip):
 *   perm      int32 [n]           new -> old numbering (I^sigma in post-order)
 *   node_info int32 [nnodes][14]  level, parent, child0, child1, i_off, m_i,
 *                                 b_off, m_b, x0, x1, y0, y1, axis, cut
 *   blist     int32 [sum_mb]      B^sigma in new numbering, node after node
 *   emap      int32 [sum_mb]      position of each B^kappa row in the parent front
 *   e_off     int32 [nnodes+1]    entry ranges per node
 *   e_row, e_col, e_idx int32 [nnz]  front-local row/column and CSR position of
 *                                 every entry of A, grouped by the node whose
 *                                 front receives it (Eq. 3.2 / Eq. 3.4)
 */
ndhss_status ndhss_tree_export(const ndhss_tree* t, int32_t* perm, int32_t* node_info,
                               int32_t* blist, int32_t* emap, int32_t* e_off, int32_t* e_row,
                               int32_t* e_col, int32_t* e_idx);

void ndhss_tree_destroy(ndhss_tree* t);

/*
 * ndhss_factor -- approximate factorization P = L D R (Alg. 3.4): fronts
 * assembled bottom-up level by level (Eq. 3.2, Eq. 3.4), interior blocks
 * eliminated with partial pivoting restricted to I^sigma, giving
 * (A_ii)^{-1}, R = -(A_ii)^{-1} A_ib (Eq. 3.3b), L = -A_bi (A_ii)^{-1}
 * (Eq. 3.3a) and the Schur complement S (Eq. 3.5) passed to the parent.
 * With opts.hss_levels >= 0, on levels <= L_HSS = depth - hss_levels the
 * Schur complement is compressed by randomized adaptive HSS compression
 * (Alg. A.1, cluster tree of Fig. 4, tolerance eps_hss, Philox samples from
 * opts.seed) and the parent assembles the compressed S; strictly above L_HSS
 * R is stored as a row interpolative decomposition R ~ X R(J, :) found by
 * randomized range finding (Sec. 3.4) and L = R^T is used (A symmetric).
 *   t          tree from ndhss_build_tree (not modified, must outlive nothing)
 *   vtype      value type of A
 *   d_rowptr, d_col, d_vals  device CSR of A in the original numbering; only
 *              read during the call
 *   opts       factor options (NULL = FP64, no compression)
 *   stream     stream for all device work; synchronised before returning
 *              (with compression, the low-rank R is compressed on a stream
 *              and host thread of the library's own, beside the root level's
 *              elimination; both are joined back to `stream` and ended
 *              before the call returns)
 *   out        receives a new factor handle holding device memory
 * Errors: SINGULAR (node reported), OOM, CUDA, INVALID_ARG.
 */
ndhss_status ndhss_factor(const ndhss_tree* t, int32_t vtype, const int32_t* d_rowptr,
                          const int32_t* d_col, const void* d_vals, const ndhss_factor_opts* opts,
                          void* stream, ndhss_factorization** out);

/* ndhss_factor_stats_get -- copy the factor's sizes, ranks and (with
 * opts.timing = 1) per-class device times into caller-owned *st.  Host only,
 * no device work.  INVALID_ARG when f or st is NULL. */
ndhss_status ndhss_factor_stats_get(const ndhss_factorization* f, ndhss_factor_stats* st);

/*
 * ndhss_factor_get_block -- copy one factor block of node `node` to host
 * memory as float64/complex128 column-major with leading dimension ld:
 *   which 0: (A_ii)^{-1}   m_i x m_i        which 1: R   m_i x m_b (Eq. 3.3b)
 *   which 2: L   m_b x m_i (Eq. 3.3a)       which 3: S   m_b x m_b (Eq. 3.5)
 * Compressed nodes return the stored approximations: S as handed to the
 * parent (its HSS reconstruction), R = X R(J, :) and L = R^T.
 * Synchronises the factor's stream.  INVALID_ARG for a bad node, block or ld.
 */
ndhss_status ndhss_factor_get_block(const ndhss_factorization* f, int32_t node, int32_t which,
                                    void* host_out, int64_t ld);

/*
 * ndhss_factor_destroy -- release a factorization (NULL is ignored).  Waits
 * for all work on the device first, since any stream may still read it.
 * Device memory of the library (factor storage and per-call work space)
 * comes from one stream-ordered pool per device that keeps freed memory
 * cached for the next call rather than returning it to the driver; it is
 * released when the process exits.
 */
void ndhss_factor_destroy(ndhss_factorization* f);

/*
 * ndhss_apply -- y = P^{-1} x by Algorithm 3.1: bottom-up b(B) += L b(I),
 * the block-diagonal solve b(I) <- (A_ii)^{-1} b(I) at all nodes at once,
 * top-down b(I) += R b(B).
 *   nrhs      number of right-hand sides (columns)
 *   x, y      float64/complex128 (per the factor's vtype) n x nrhs,
 *             column-major with leading dimensions ldx, ldy >= n, ORIGINAL
 *             numbering; device or host pointers (host buffers are staged
 *             through device memory inside the call).  x and y may alias.
 * Stream-ordered; synchronises only when x or y is host memory.
 * Each right-hand side is one persistent kernel launch working through a
 * queue of row tasks in dependency order (plus one memset of its control
 * words).  Every wait inside that kernel is bounded (2 s); when one gives
 * up, the kernel returns early, y is undefined and the factorization keeps
 * an error mark: this call (if it synchronises), ndhss_gmres and every later
 * ndhss_apply that synchronises then return NDHSS_ERR_TIMEOUT, and later
 * applies of that factorization return at once.  Destroy it and factor again.
 * Setting the environment variable NDHSS_APPLY_SCHEDULE=levels selects one
 * launch per tree level and phase instead (same arithmetic, bit-identical
 * result; kept as a cross-check).
 */
ndhss_status ndhss_apply(const ndhss_factorization* f, int32_t nrhs, const void* x, int64_t ldx,
                         void* y, int64_t ldy, void* stream);

/*
 * ndhss_apply_noalloc -- the result of ndhss_apply for one right-hand side,
 * from a call that allocates no memory at all.  For callers that cannot
 * allocate device memory at the moment they need P^{-1}: a solver loop in a
 * process whose device memory is reserved up front by another allocator (a
 * framework's caching allocator, a fixed memory budget), or code under a
 * no-allocation-after-setup rule, where an allocation could fail or stall.
 * The paper has no counterpart; this is an interface convenience.
 *   f          factor from ndhss_factor
 *   d_x, d_y   DEVICE pointers, n float64/complex128 values (original
 *              numbering); host pointers are rejected with INVALID_ARG
 *   stream     stream the kernels are ordered on
 * The work area (two vectors of n elements of the factor's type, the
 * low-rank nodes' partial products for each sweep, the diagonal partial
 * products, and 32-bit control words: 4 + 6 per tree node + 2 per ULV
 * record) lives in one static device array of 16 MiB that every GPU loading
 * the library holds until the process exits; problems needing more (about
 * n > 520000 for complex128 fronts, n > 1000000 for complex64 or float64
 * fronts, less with compressed factors) get INVALID_ARG.
 * The first call on a device looks up that array's device address (once per
 * device, with that device current, and again if the device's context was
 * replaced, e.g. after a device reset): make that first call before any
 * stream capture.  All calls share the array and each overwrites what it
 * reads before reading it, so nothing needs clearing; calls that overlap on
 * the GPU (other streams, other threads) race on it and must be serialised.
 * The call never synchronises: if a bounded wait of the apply kernel gives
 * up inside it, y is undefined, the call has already returned NDHSS_OK, and
 * the factorization's error mark surfaces at the next synchronising call on
 * it (ndhss_gmres, or ndhss_apply with a host buffer), which returns
 * NDHSS_ERR_TIMEOUT.
 */
ndhss_status ndhss_apply_noalloc(const ndhss_factorization* f, const void* d_x, void* d_y, void* stream);

/*
 * ndhss_elem_qform -- per group g of elements (elements goff[g] .. goff[g+1]-1):
 *     q[g] = sum_e sum_{a,b} conj(lam[idx[e][a]]) M_e[a][b] x[idx[e][b]]
 * the quadratic forms of the adjoint-state gradient of a misfit with respect
 * to piecewise-constant coefficients (dJ/dm_j = -Re(lam^H dA/dm_j x) with
 * dA/dm_j assembled from the element matrices of block j; Helmholtz model of
 * Sec. 4, Eq. 4.2; the paper itself has no adjoint).  No counterpart in the
 * paper otherwise.
 *   ngroups    number of groups (output length)
 *   d_goff     device int32 [ngroups + 1], element offsets of each group
 *              (elements sorted by group)
 *   nloc       DOFs per element
 *   d_idx      device int32 [n_elem x nloc], row-major: the elements' DOFs
 *   d_mats     device float64 [n_elem x nloc x nloc], row-major real element
 *              matrices
 *   d_lam, d_x device complex128 vectors indexed by DOF
 *   d_q        device complex128 [ngroups], overwritten
 * Stream-ordered; deterministic (fixed summation order).  INVALID_ARG for
 * NULL pointers, ngroups < 0 or nloc < 1.
 */
ndhss_status ndhss_elem_qform(int32_t ngroups, const int32_t* d_goff, int32_t nloc, const int32_t* d_idx,
                              const double* d_mats, const void* d_lam, const void* d_x, void* d_q, void* stream);

/*
 * ndhss_testing_stall_apply -- failure-detection hook for tests (no
 * counterpart in the paper).  Raises the completion requirement of the
 * root's diagonal step by one, a count that no task will ever reach, so the
 * down-sweep tasks of the next apply wait until their bound runs out.  That
 * apply then ends early with the factorization marked as failed (see
 * ndhss_apply).  Synchronous.  INVALID_ARG for NULL or a factorization
 * without a dataflow queue.
 */
ndhss_status ndhss_testing_stall_apply(ndhss_factorization* f);

/*
 * ndhss_spmv -- y = A x for a CSR matrix in float64 / complex128 (the
 * matrix-vector product x -> A x of Sec. 2.3 and of every Krylov step).
 * All pointers are device pointers; n rows; stream-ordered.
 */
ndhss_status ndhss_spmv(int32_t n, int32_t vtype, const int32_t* d_rowptr, const int32_t* d_col,
                        const void* d_vals, const void* d_x, void* d_y, void* stream);

/*
 * ndhss_gmres -- solve A x = b with restarted GMRES on P^{-1} A x = P^{-1} b
 * (Eq. 1.2, Sec. 4): x0 = 0, Arnoldi by classical Gram-Schmidt applied
 * twice in float64, complex Givens rotations, a cycle ends when
 * ||P^{-1} r|| <= inner tol ||P^{-1} b|| or after `restart` steps; a solve is
 * converged only when the float64 true residual ||b - A x|| / ||b|| <= tol,
 * checked after every cycle (restarts act as iterative refinement).
 *   f         factor (the preconditioner)
 *   d_rowptr, d_col, d_vals  device CSR of A (original numbering, vtype of f)
 *   nrhs      right-hand sides, solved one after another
 *   b, x      n x nrhs column-major (ldb, ldx >= n), device or host pointers
 *   opts      NULL = restart 30, maxit 300, tol 1e-8, inner 0.1, cycle_rtol auto,
 *             conj_transpose 0 (1: the adjoint system A^H x = b, Sec. 4's
 *             gradient by the adjoint state)
 *   stats     host array of nrhs entries (may be NULL)
 * Returns NOT_CONVERGED if any right-hand side missed tol (x still written).
 * Synchronises the stream once per Arnoldi step (to read the residual).
 */
ndhss_status ndhss_gmres(const ndhss_factorization* f, const int32_t* d_rowptr, const int32_t* d_col,
                         const void* d_vals, int32_t nrhs, const void* b, int64_t ldb, void* x,
                         int64_t ldx, const ndhss_gmres_opts* opts, ndhss_gmres_stats* stats,
                         void* stream);

/*
 * ndhss_apply_multi -- y = P^{-1} x for up to 32 right-hand sides at once
 * (Alg. 3.1 with one pass over the factor for all of them): per level,
 * deepest first, z(I^s) = A_ii^{-1} P^T y(I^s) and y(B^s) -= L P^T y(I^s) for
 * every node of the level as 64-row x 32-column tiles; then per level from
 * the roots, z(I^s) += R z(B^s).  Nodes with compressed Gauss transforms
 * (R ~ X R(J,:), L = R^T above the switching level) take the low-rank
 * products t = X^T y(I^s), y(B^s) += R(J,:)^T t on the way up and
 * t = R(J,:) z(B^s), z(I^s) += X t on the way down, 32 columns at a time.  A
 * factorization with a ULV diagonal gives INVALID_ARG (ndhss_apply handles it).
 *   nrhs       0..32 right-hand sides
 *   d_x, d_y   device float64 / complex128 (per the factor's vtype) arrays of
 *              n rows, interleaved: element (row, c) at row * ld + c,
 *              ldx, ldy >= nrhs; original numbering
 * Works in the factor's precision (one conversion at entry and exit); uses
 * 2 n x 32 front-type elements of pooled scratch plus k x 32 per low-rank
 * node; synchronises the stream.
 */
ndhss_status ndhss_apply_multi(const ndhss_factorization* f, int32_t nrhs, const void* d_x, int64_t ldx,
                               void* d_y, int64_t ldy, void* stream);

/*
 * ndhss_gmres_batched -- restarted GMRES (as ndhss_gmres: x0 = 0, classical
 * Gram-Schmidt twice in float64, complex Givens rotations, true-residual
 * restarts, the same stopping rules) for nsys independent problems x nrhs
 * right-hand sides at once, in lockstep: every Arnoldi step is one sparse
 * product of 32 interleaved columns, one ndhss_apply_multi and segmented
 * reductions per problem, so a pass over A and over the factor serves all
 * nsys * nrhs systems.  A system that meets its tolerance stops changing
 * while the others go on.  f is the factorization of the batch's forest
 * (ndhss_build_tree_batched), dense or compressed fronts (no ULV diagonal).
 *   d_rowptr, d_col, d_vals  device CSR of the block-diagonal batch matrix
 *   nsys       problems; sys_off host int64 [nsys + 1], problem s owns rows
 *              [sys_off[s], sys_off[s+1]), sys_off[0] = 0, sys_off[nsys] = n
 *   nrhs       right-hand sides per problem, 0..32
 *   d_b, d_x   device n x nrhs column-major (ldb, ldx >= n); column c of
 *              problem s's rows is system (s, c)
 *   opts       as ndhss_gmres (restart <= 31)
 *   stats      host array [nsys * nrhs] (system (s, c) at s * nrhs + c), or NULL
 * Memory: (restart + 5) n x 32 vectors of float64 / complex128 from the
 * library's pool.  Synchronises once per Arnoldi step.  NOT_CONVERGED if any
 * system missed tol (x still written).
 */
ndhss_status ndhss_gmres_batched(const ndhss_factorization* f, const int32_t* d_rowptr, const int32_t* d_col,
                                 const void* d_vals, int32_t nsys, const int64_t* sys_off, int32_t nrhs,
                                 const void* d_b, int64_t ldb, void* d_x, int64_t ldx,
                                 const ndhss_gmres_opts* opts, ndhss_gmres_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NDHSS_H */
