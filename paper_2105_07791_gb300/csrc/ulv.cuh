// ULV factorization of HSS(A_ii) (the assembled interior block of a front
// strictly above the switching level, in the order along the node's cut):
// device job description shared by the compression (hss.cu, which builds the
// jobs from its HSS generators) and the factorization kernel (ulv.cu).
#pragma once

#include "common.cuh"

namespace ndhss {

// One HSS node of one front.  Sizes: the node's current block is m x m with
// row and column bases of width k; ne = m - kt unknowns are eliminated and
// kt = min(m, k) remain for the parent.  Children are jobs of the previous
// (deeper) launch; a root job inverts its merged block instead.
template <typename T>
struct UlvJob {
    int m, k, ne, kt;
    int leaf, root;
    int ka, kb;                 // inner: children's basis widths (B12 is ka x kb)
    int c1, c2;                 // inner: child jobs (indices into the same job array family)
    const T* D0;                // leaf: its diagonal block of A_ii (ld ldd0)
    int64_t ldd0;
    const T* X;                 // leaf: basis U = V (m x k, ld ldx); inner: transfer E ((ka+kb) x k)
    int64_t ldx;
    const T* B12;               // inner: ka x kb (ld ka); B21: kb x ka (ld kb)
    const T* B21;
    // persistent solve data (apply)
    T* Mup;                     // (m + k) x m: rows [y1 (ne); r^ (kt); G (k)]
    T* W;                       // m x m
    T* Mm;                      // inner: m x (ka + kb)
    T* E;                       // inner non-root: (ka + kb) x k
    T* Dinv;                    // root: m x m
    // handed to the parent (scratch): D^ (kt x kt), U^, V^ (kt x k)
    T* Dh;
    T* Uh;
    T* Vh;
    // work space of this job (scratch)
    T* w;                       // >= ulv_work_elems(m, k, ne)
    int* status;                // set to 1 when a pivot of the root inverse vanishes
};

// Scratch elements one job needs (see ulv_factor_kernel).
__host__ __device__ inline int64_t ulv_work_elems(int m, int k, int ne) {
    return 4 * (int64_t)m * m + 2 * (int64_t)m * k + (int64_t)m * ne + (int64_t)k * m + (int64_t)ne * ne +
           (int64_t)ne * m + 2 * (int64_t)m + 64;
}

template <typename T>
ndhss_status ulv_launch_level(const UlvJob<T>* d_jobs, const UlvJob<T>* d_all, int count, cudaStream_t st);

}  // namespace ndhss
