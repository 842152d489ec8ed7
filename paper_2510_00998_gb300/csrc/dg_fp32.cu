// Instantiation of the DG-level kernels for float arithmetic.
#include "dg_kernels.cuh"

namespace dgmg {

template <>
cudaError_t launch_project<float>(int dim, int q, const DGConst<float> &c, int cpb, float *u, const float *e0,
                                 float *tr, cudaStream_t s) {
    return launch_project_impl<float>(dim, q, c, cpb, u, e0, tr, s);
}

template <>
cudaError_t launch_smooth<float>(int dim, int q, const DGConst<float> &c, int cpb, int exact, float *u,
                                const float *b,
                                const float *kappa, const float *fd, const float *linv, const float *tr_in, float *tr_out,
                                cudaStream_t s) {
    return launch_smooth_impl<float>(dim, q, c, cpb, exact, u, b, kappa, fd, linv, tr_in, tr_out, s);
}

template <>
cudaError_t launch_residual<float>(int dim, int q, const DGConst<float> &c, int cpb, int mode, const float *u,
                                  const float *b, const float *kappa, const float *tr, float *r, float *corners,
                                  const float *fd, cudaStream_t s) {
    return launch_residual_impl<float>(dim, q, c, cpb, mode, u, b, kappa, tr, r, corners, fd, s);
}

template <>
cudaError_t launch_project_batch<float>(int dim, int q, const BatchDG<float> *D, const BlockMap *map, int nblocks, int cpb,
                                     float *u, int with_e0, cudaStream_t s) {
    return launch_project_batch_impl<float>(dim, q, D, map, nblocks, cpb, u, with_e0, s);
}
template <>
cudaError_t launch_smooth_batch<float>(int dim, int q, const BatchDG<float> *D, const BlockMap *map, int nblocks, int cpb,
                                    int exact, float *u, const float *b, int cur, cudaStream_t s) {
    return launch_smooth_batch_impl<float>(dim, q, D, map, nblocks, cpb, exact, u, b, cur, s);
}
template <>
cudaError_t launch_residual_batch<float>(int dim, int q, const BatchDG<float> *D, const BlockMap *map, int nblocks,
                                      int cpb, int mode, const float *u, const float *b, float *r, int cur,
                                      cudaStream_t s) {
    return launch_residual_batch_impl<float>(dim, q, D, map, nblocks, cpb, mode, u, b, r, cur, s);
}
template <>
cudaError_t launch_zero_traces_batch<float>(int dim, int q, const BatchDG<float> *D, int count, cudaStream_t s) {
    return launch_zero_traces_batch_impl<float>(dim, q, D, count, s);
}

template <>
cudaError_t launch_dg_transfer<float>(int dim, int qf, bool prolong, int64_t ncell, const DGInterp<float> &P,
                                   const float *in, float *out, cudaStream_t s) {
    return launch_dg_transfer_impl<float>(dim, qf, prolong, ncell, P, in, out, s);
}

cudaError_t wait_timeouts_fp32(unsigned long long *count) { return read_wait_timeouts(count); }
cudaError_t wait_timeouts_addr_fp32(unsigned long long **ptr) {
    return cudaGetSymbolAddress((void **)ptr, g_wait_timeouts);
}

}  // namespace dgmg
