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
                                  const double *fd, cudaStream_t s) {
    return launch_residual_impl<double>(dim, q, c, cpb, mode, u, b, kappa, tr, r, corners, fd, s);
}

template <>
cudaError_t launch_project_batch<double>(int dim, int q, const BatchDG<double> *D, const BlockMap *map, int nblocks, int cpb,
                                     double *u, int with_e0, cudaStream_t s) {
    return launch_project_batch_impl<double>(dim, q, D, map, nblocks, cpb, u, with_e0, s);
}
template <>
cudaError_t launch_smooth_batch<double>(int dim, int q, const BatchDG<double> *D, const BlockMap *map, int nblocks, int cpb,
                                    int exact, double *u, const double *b, int cur, cudaStream_t s) {
    return launch_smooth_batch_impl<double>(dim, q, D, map, nblocks, cpb, exact, u, b, cur, s);
}
template <>
cudaError_t launch_residual_batch<double>(int dim, int q, const BatchDG<double> *D, const BlockMap *map, int nblocks,
                                      int cpb, int mode, const double *u, const double *b, double *r, int cur,
                                      cudaStream_t s) {
    return launch_residual_batch_impl<double>(dim, q, D, map, nblocks, cpb, mode, u, b, r, cur, s);
}
template <>
cudaError_t launch_zero_traces_batch<double>(int dim, int q, const BatchDG<double> *D, int count, cudaStream_t s) {
    return launch_zero_traces_batch_impl<double>(dim, q, D, count, s);
}

template <>
cudaError_t launch_dg_transfer<double>(int dim, int qf, bool prolong, int64_t ncell, const DGInterp<double> &P,
                                   const double *in, double *out, cudaStream_t s) {
    return launch_dg_transfer_impl<double>(dim, qf, prolong, ncell, P, in, out, s);
}

cudaError_t wait_timeouts_fp64(unsigned long long *count) { return read_wait_timeouts(count); }
cudaError_t wait_timeouts_addr_fp64(unsigned long long **ptr) {
    return cudaGetSymbolAddress((void **)ptr, g_wait_timeouts);
}

}  // namespace dgmg
