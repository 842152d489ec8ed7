// Instantiation of the DG-level kernels for double arithmetic.
#include "dg_kernels.cuh"

namespace dgmg {

template <>
cudaError_t launch_project<double>(int dim, int q, const DGConst<double> &c, int cpb, double *u, const double *e0,
                                 double *tr, cudaStream_t s) {
    return launch_project_impl<double>(dim, q, c, cpb, u, e0, tr, s);
}

template <>
cudaError_t launch_smooth<double>(int dim, int q, const DGConst<double> &c, int cpb, int exact, double *u,
                                const double *b,
                                const double *kappa, const double *fd, const double *linv, const double *tr_in, double *tr_out,
                                cudaStream_t s) {
    return launch_smooth_impl<double>(dim, q, c, cpb, exact, u, b, kappa, fd, linv, tr_in, tr_out, s);
}

template <>
cudaError_t launch_residual<double>(int dim, int q, const DGConst<double> &c, int cpb, int mode, const double *u,
                                  const double *b, const double *kappa, const double *tr, double *r, double *corners,
                                  cudaStream_t s) {
    return launch_residual_impl<double>(dim, q, c, cpb, mode, u, b, kappa, tr, r, corners, s);
}

cudaError_t wait_timeouts_fp64(unsigned long long *count) { return read_wait_timeouts(count); }

}  // namespace dgmg
