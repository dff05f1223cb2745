// Quadratic forms summed by groups of elements, for the adjoint-state
// gradient of a misfit with respect to piecewise-constant coefficients of
// the Helmholtz model (Sec. 4, Eq. 4.2):  dJ/dm_j = -Re(lambda^H dA/dm_j x)
// with dA/dm_j assembled from the element (or boundary-edge) matrices of
// block j.  One warp per group, lanes strided over the group's elements,
// then a fixed shuffle tree: the sum does not depend on scheduling.
#include "common.cuh"

namespace ndhss {
namespace {

__global__ void elem_qform_kernel(int ngroups, const int32_t* __restrict__ goff, int nloc, const int32_t* __restrict__ idx,
                                  const double* __restrict__ mats, const c128* __restrict__ lam,
                                  const c128* __restrict__ x, c128* __restrict__ q) {
    const int g = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= ngroups) return;
    c128 acc = {0.0, 0.0};
    for (int e = goff[g] + lane; e < goff[g + 1]; e += 32) {
        const int32_t* id = idx + (int64_t)e * nloc;
        const double* M = mats + (int64_t)e * nloc * nloc;
        for (int a = 0; a < nloc; ++a) {
            c128 t = {0.0, 0.0};
            for (int b = 0; b < nloc; ++b) {
                const c128 xv = x[id[b]];
                t.x = fma(M[a * nloc + b], xv.x, t.x);
                t.y = fma(M[a * nloc + b], xv.y, t.y);
            }
            const c128 l = conjv(lam[id[a]]);
            acc = fmac(l, t, acc);
        }
    }
    for (int o = 16; o; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) q[g] = acc;
}

}  // namespace
}  // namespace ndhss

extern "C" ndhss_status ndhss_elem_qform(int32_t ngroups, const int32_t* d_goff, int32_t nloc, const int32_t* d_idx,
                                         const double* d_mats, const void* d_lam, const void* d_x, void* d_q,
                                         void* stream) {
    return ::ndhss::guarded("ndhss_elem_qform", [&]() -> ndhss_status {
        using namespace ndhss;
        clear_error();
        if (ngroups < 0 || nloc < 1 || !d_goff || !d_idx || !d_mats || !d_lam || !d_x || !d_q)
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_elem_qform: bad argument");
        if (ngroups == 0) return NDHSS_OK;
        const int threads = 256;
        const unsigned blocks = (unsigned)(((int64_t)ngroups * 32 + threads - 1) / threads);
        elem_qform_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
            ngroups, d_goff, nloc, d_idx, d_mats, static_cast<const c128*>(d_lam), static_cast<const c128*>(d_x),
            static_cast<c128*>(d_q));
        NDHSS_LAUNCH_CHECK("elem_qform_kernel");
        return NDHSS_OK;
    });
}
