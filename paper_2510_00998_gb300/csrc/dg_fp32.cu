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
                                  cudaStream_t s) {
    return launch_residual_impl<float>(dim, q, c, cpb, mode, u, b, kappa, tr, r, corners, s);
}

cudaError_t wait_timeouts_fp32(unsigned long long *count) { return read_wait_timeouts(count); }

}  // namespace dgmg
