// Internal declarations of libdgmg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "dgmg.h"

namespace dgmg {

constexpr int QMAX = 7;     // p <= 6
constexpr int PMAX = QMAX - 1;

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define DG_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ::dgmg::cuda_fail(e_, #call); \
    } while (0)

// Values stored per cell face in a trace buffer: the value and the normal
// derivative at the q^(d-1) face nodes, padded so that every face of every cell
// starts on a 16-byte boundary (a bulk copy moves one face). Only FP32 with an
// odd number of face nodes pads (2 values per face for q = 5 in 3D).
template <typename T>
__host__ __device__ constexpr int trace_face_stride(int nf) {
    return (2 * nf * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);
}

// Process-wide count of kernels launched by the library (dgmg_kernel_launches).
extern std::atomic<long long> g_kernel_launches;
inline void count_launches(int k) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }
// Bounded waits that ran out in the kernels of the float / double translation unit.
cudaError_t wait_timeouts_fp32(unsigned long long *count);
cudaError_t wait_timeouts_fp64(unsigned long long *count);
cudaError_t wait_timeouts_volume(unsigned long long *count);
// device addresses of the same counters on the current device (for
// stream-ordered snapshots)
cudaError_t wait_timeouts_addr_fp32(unsigned long long **ptr);
cudaError_t wait_timeouts_addr_fp64(unsigned long long **ptr);

// ------------------------------------------------------- reference element
// 1D Lagrange element of degree p on [-1,1] with GLL (Sec. 2.2) or GL
// (Sec. 6.4) nodes, computed on the host in double precision.
struct RefElem1D {
    int p = 0, q = 0;
    int basis = DGMG_BASIS_GLL;
    std::vector<double> nodes;            // q nodes, ascending
    std::vector<double> M, K;             // q x q exact mass / stiffness on [-1,1], row-major
    std::vector<double> e0, ep;           // l_j(-1), l_j(+1): unit vectors for GLL, dense for GL
    std::vector<double> d0, dp;           // l_j'(-1), l_j'(+1)
};
RefElem1D make_refelem(int p, int basis = DGMG_BASIS_GLL);
void gauss_legendre(int m, std::vector<double> &x, std::vector<double> &w);
// values and derivatives of the Lagrange basis on `nodes` at x
void lagrange_at(const std::vector<double> &nodes, double x, double *val, double *der);

// lower Cholesky factor inverse of the SPD q x q matrix M (row-major)
bool cholesky_inverse_lower(int q, const double *M, double *Linv);

// Input of the per-cell fast-diagonalisation factor kernel for one DG space
// (the h-scaled 1D data per axis; see factors.cu).
struct FDInput {
    int dim, q, interior_only;
    int n[3];
    double Kh[3][QMAX * QMAX];      // stiffness
    double Linv[3][QMAX * QMAX];    // inverse of the lower Cholesky factor of the mass
    double d0[3][QMAX], dp[3][QMAX];
    double e0[QMAX], ep[QMAX];
    double gam[3];
};
// fd[cell][axis] = [S (q x q) | lambda (q)] for every cell (FP64 arithmetic,
// output in T); kappa: per-cell FP64 on the device
template <typename T>
cudaError_t launch_fd_factors(const FDInput &in, const double *kappa, int64_t ncell, T *fd, cudaStream_t s);
// The h-scaled 1D masses of the axes (FP64), by value.
struct MassTables {
    double M[3][QMAX * QMAX];
};
// fdr[cell][axis] = [S^T M_a (q x q) | lambda (q)] from fd[cell][axis] = [S | lambda]:
// the factors the one-thread-per-cell residual applies A_KK u with
template <typename TI, typename TO>
cudaError_t launch_residual_factors(int dim, int q, int64_t ncell, const TI *fd, const MassTables &m, TO *fdr,
                                    cudaStream_t s);
// kfac[cell][2 axis + side] = 2 kappa_K kappa_N / (kappa_K + kappa_N) across each
// interior face (0 on the boundary), from the FP64 kappa
template <typename T>
cudaError_t launch_facet_coefficients(int dim, const int *n, int64_t ncell, const double *kappa, T *kfac,
                                      cudaStream_t s);
// linv[cell][node] = omega / (sum of the cell's eigenvalues at the node): the
// smoother's damping folded into the table
cudaError_t launch_inverse_eigen_sums(int dim, int q, int64_t ncell, const double *fd, double omega,
                                      double *linv, cudaStream_t s);

// ------------------------------------------------------------ kernels API
// Constant data of one DG level, passed to kernels by value.
template <typename T>
struct DGConst {
    int n[3];
    int64_t ncell;
    T M[3][QMAX * QMAX];
    T K[3][QMAX * QMAX];
    T d0[3][QMAX];
    T dp[3][QMAX];
    T gamma[3];
    T hat[2][QMAX];
    T omega;
    // GL basis (gl != 0): the end values l_j(-1), l_j(+1) of the 1D basis,
    // which then are dense; with GLL (gl == 0) they are the unit vectors of
    // the end nodes and the kernels index those nodes directly
    int gl;
    T v0[QMAX], vp[QMAX];
    // the 1D mass of axis a as diag(mw[a]) - mu[a] mu[a]^T: with GLL nodes the
    // exact mass is the lumped GLL-quadrature mass plus a rank-one term (the rule
    // is exact to degree 2p - 1; for the degree-2p products l_i l_j its error
    // is a multiple of the product of their leading coefficients); with GL nodes
    // the mass is diagonal and mu = 0
    T mw[3][QMAX], mu[3][QMAX];
    // facet coefficients kfac[cell][face = 2 axis + side]: the harmonic mean of
    // the cell's and the neighbour's kappa on an interior face, 0 on a boundary
    // face (formed once per level, updated with kappa)
    const T *kfac;
};

// Q1 level description for the CG kernels.
template <typename T>
struct CGLevelDev {
    int m[3];              // interior vertices per axis
    int64_t nv;
    const T *st;           // [3^d][nv] stencil, offset (sx+1) + 3 (sy+1) + 9 (sz+1)
    // transfer to the next coarser level (per axis tables); null on the coarsest
    const int *pl_lo[3];   // fine vertex -> lower coarse parent (-1 if none)
    const int *pl_hi[3];   // fine vertex -> upper coarse parent (-1 if none)
    const T *pl_wlo[3], *pl_whi[3];
    const int *rs_start[3];  // coarse vertex -> first fine child
    const int *rs_cnt[3];    // number of fine children (<= 2f-1)
    const T *rs_w[3];        // [nc][5] weights
    int mc[3];               // interior vertices per axis of the coarser level
};

// Interpolation from DG degree q_c - 1 = q_f - 2 to degree q_f - 1 on the same
// cell: I[i_f][j_c] = l_j^c(x_i^f), row-major q_f x q_c (gradual p-hierarchy).
template <typename T>
struct DGInterp {
    T I[QMAX * QMAX];
};
// prolong: out += (I (x) I (x) I) in (coarse -> fine); else out = (I^T (x) ...) in.
// qf: nodes per axis of the finer level (3..7).
template <typename T>
cudaError_t launch_dg_transfer(int dim, int qf, bool prolong, int64_t ncell, const DGInterp<T> &P, const T *in,
                               T *out, cudaStream_t s);

// ---- batched launches: many independent instances of one degree share a launch
// Per instance (DG level): its constants (mesh, h-scaled 1D matrices), its first
// cell in the group's concatenated vectors (a multiple of 32 cells, so every
// instance's slice keeps the vectors' 16-byte alignment), and its own arrays.
template <typename T>
struct BatchDG {
    DGConst<T> c;
    int64_t off;
    const T *kappa, *fd, *linv;
    const T *fdr;         // the residual's factors [S^T M | lambda] (null: operator-only level)
    T *tr[2];
    T *corners;
    const T *e0;          // the instance's Q1 level-0 correction (p-prolongation source)
};
// CTA -> (instance, first cell of the CTA within the instance)
struct BlockMap {
    int inst, cell0;
};
// Per (instance, Q1 level): the level, its vectors, the next coarser level's
// right-hand side and correction, the dense inverse on the coarsest level, and
// (level 0) the DG mesh and cell corner sums of the p-restriction.
template <typename T>
struct BatchCG {
    CGLevelDev<T> L;
    T *u[2], *b, *r;
    T *b_next;
    const T *e_next;
    const double *Ainv;
    int n[3];
    const T *corners;
};
// The Q1 h-cycle of one problem as one cooperative launch: every level's
// operator and transfer tables, its vectors, the coarsest inverse.
constexpr int Q1_MAXLEV = 24;
// threads per block of the cooperative cycle: 256, or (FP32, wide) 512: one
// block per SM, more loads of the vertex loops in flight, fewer barrier
// arrivals, and 512 threads for the levels run in block 0. A 512-thread block
// holds a whole SM's registers, so its cooperative launch waits for empty SMs
// where other solves share the GPU (the solve server keeps 256); in FP64 the
// 512-thread kernel spills.
constexpr int Q1_TPB = 256, Q1_TPB_WIDE = 512;
template <typename T>
struct Q1Plan {
    int nlev, nu_pre, nu_post;
    int local_from;        // levels >= this one run in one block (nlev: none)
    T omega;
    int64_t ncoarse;
    const double *Ainv;
    CGLevelDev<T> L[Q1_MAXLEV];
    T *u0[Q1_MAXLEV], *u1[Q1_MAXLEV], *b[Q1_MAXLEV], *r[Q1_MAXLEV];
};
// e on level 0 (u0 or u1 of level 0, by the parity of nu_pre + nu_post) from b
// on level 0; bar: the plan's own arrival counter (zero before its first
// launch; every launch on it with the same number of blocks)
template <typename T>
cudaError_t launch_q1_cycle(int dim, const Q1Plan<T> *plan, unsigned long long *bar, int blocks, bool wide,
                            cudaStream_t s);
// the most blocks of the cooperative launch (one per SM), 0 if it cannot run
template <typename T>
int q1_cycle_max_blocks(int dim, bool wide);
cudaError_t q1_barrier_timeouts(unsigned long long *count);
cudaError_t q1_barrier_timeouts_addr(unsigned long long **ptr);
// Set once a grid-barrier wait of the one-launch Q1 cycle ran out anywhere in
// the process: that kernel then returns without work on its device, so every
// context takes the launch per step from then on (and recaptures its graphs).
extern std::atomic<int> g_q1_one_launch_off;

// CTA -> (descriptor, first vertex (or row) of the CTA)
struct VertMap {
    int desc, v0;
};
constexpr int BATCH_VERTS = 256;   // vertices (rows) per CTA of the batched Q1 kernels

// CTAs of a persistent batched launch of kernel `fn` (threads per CTA, dynamic
// shared memory) over `items` work items: as many as stay resident on the
// current device at once, at most `items` (cached per kernel and shared-memory
// size; a process drives devices of one kind).
unsigned persistent_grid(const void *fn, int threads, size_t smem, int64_t items);

// Launch wrappers (implemented per precision in dg_fp64.cu / dg_fp32.cu).
// All return cudaError_t of the launch.
template <typename T>
cudaError_t launch_project(int dim, int q, const DGConst<T> &c, int cpb, T *u, const T *e0,
                           T *tr, cudaStream_t s);
template <typename T>
cudaError_t launch_smooth(int dim, int q, const DGConst<T> &c, int cpb, int exact, T *u, const T *b,
                          const T *kappa, const T *fd, const T *linv, const T *tr_in, T *tr_out, cudaStream_t s);
// mode bits for launch_residual
// RES_DIRECT (batched FP32 one-thread-per-cell residual): A_KK u in the direct
// sum-factorised form instead of through the factors (the FP32 CG operator)
enum { RES_HAS_B = 1, RES_WRITE_R = 2, RES_CORNERS = 4, RES_NEGATE = 8, RES_DIRECT = 16 };
// fd: the level's fast-diagonalisation factors of the exact diagonal blocks, or
// null; with them (3D, q small enough, cpb <= 0) the one-thread-per-cell kernel
// runs, which forms A_KK u from the factors
template <typename T>
cudaError_t launch_residual(int dim, int q, const DGConst<T> &c, int cpb, int mode, const T *u,
                            const T *b, const T *kappa, const T *tr, T *r, T *corners, const T *fd,
                            cudaStream_t s);

template <typename T>
cudaError_t launch_project_batch(int dim, int q, const BatchDG<T> *D, const BlockMap *map, int nblocks, int cpb,
                                 T *u, int with_e0, cudaStream_t s);
// cpb 0: the one-thread-per-cell smoother (32 cells per CTA)
template <typename T>
cudaError_t launch_smooth_batch(int dim, int q, const BatchDG<T> *D, const BlockMap *map, int nblocks, int cpb,
                                int exact, T *u, const T *b, int cur, cudaStream_t s);
template <typename T>
cudaError_t launch_residual_batch(int dim, int q, const BatchDG<T> *D, const BlockMap *map, int nblocks, int cpb,
                                  int mode, const T *u, const T *b, T *r, int cur, cudaStream_t s);
// zero tr[0] of every instance (one CTA per instance)
template <typename T>
cudaError_t launch_zero_traces_batch(int dim, int q, const BatchDG<T> *D, int count, cudaStream_t s);

// CG kernels (cg.cu)
template <typename T>
cudaError_t launch_corner_gather(int dim, const int *n, const T *corners, T *b0, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_jacobi(int dim, const CGLevelDev<T> &L, const T *u_in, const T *b, T *u_out,
                             T omega, bool zero_guess, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_residual(int dim, const CGLevelDev<T> &L, const T *u, const T *b, T *r,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_h_restrict(int dim, const CGLevelDev<T> &L, const T *rf, T *rc, cudaStream_t s);
template <typename T>
cudaError_t launch_h_prolong(int dim, const CGLevelDev<T> &L, const T *ec, T *uf, cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_solve(int64_t nc, const double *Ainv, const T *r, T *e, cudaStream_t s);
// batched Q1 kernels: every CTA covers BATCH_VERTS vertices (rows) of one descriptor
template <typename T>
cudaError_t launch_corner_gather_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_jacobi_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, T omega,
                                   bool zero_guess, int cur, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_residual_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, int cur,
                                     cudaStream_t s);
// map over the vertices of the next coarser level
template <typename T>
cudaError_t launch_h_restrict_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, cudaStream_t s);
template <typename T>
cudaError_t launch_h_prolong_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, int cur,
                                   cudaStream_t s);
// e = u[0] = A_c^{-1} b on descriptors that are an instance's coarsest level
template <typename T>
cudaError_t launch_coarse_solve_batch(const BatchCG<T> *D, const VertMap *map, int nb, cudaStream_t s);

// BLAS-1 and helpers (blas.cu)
cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *partials,
                       double *out, cudaStream_t s);
cudaError_t launch_dot2(int64_t n, const double *x, const double *y, const double *z,
                        double *partials, double *out_xy, double *out_zy, cudaStream_t s);
cudaError_t launch_cast_d2f(int64_t n, const double *x, float *y, cudaStream_t s);
cudaError_t launch_cast_f2d(int64_t n, const float *x, double *y, cudaStream_t s);
cudaError_t launch_pcg_update_xr(int64_t n, double *x, double *r, const double *p,
                                 const double *q, const double *scal, cudaStream_t s);
cudaError_t launch_pcg_update_p(int64_t n, double *p, const double *z, const double *scal,
                                cudaStream_t s);
cudaError_t launch_sub(int64_t n, const double *a, const double *b, double *out, cudaStream_t s);
cudaError_t launch_copy_scalar(const double *src, double *dst, cudaStream_t s);
cudaError_t launch_dotf(int64_t n, const float *x, const float *y, double *partials, double *out,
                        cudaStream_t s);
cudaError_t launch_dot2f(int64_t n, const float *x, const float *y, const float *z, double *partials,
                         double *out_xy, double *out_zy, cudaStream_t s);
cudaError_t launch_update_xr_f(int64_t n, float *xs, float *r, float *rold, const float *p, const float *q,
                               const double *scal, cudaStream_t s);
// launch_update_xr_f and *out_rr = ||r||^2 of the updated r, in one pass over the vectors
cudaError_t launch_update_xr_dot_f(int64_t n, float *xs, float *r, float *rold, const float *p, const float *q,
                                   const double *scal, double *partials, double *out_rr, cudaStream_t s);
cudaError_t launch_update_p_f(int64_t n, float *p, const float *z, const double *scal, cudaStream_t s);
cudaError_t launch_accumulate_f2d(int64_t n, double *x, float *xs, cudaStream_t s);
cudaError_t launch_quad_points(int dim, int q, const int *n, int mq, const double *xq1,
                               double *xq, int64_t ncell, cudaStream_t s);
cudaError_t launch_load_vector(int dim, int q, int mq, int64_t ncell, const double *V,
                               const double *wq, const double *fq, double *b, cudaStream_t s);

// Residual + p-restriction with caller-chosen corner scratch (ctx.cu).
int64_t corner_scratch_count(const dgmg_ctx *C);
int residual_restrict_with_scratch(dgmg_ctx *C, const double *u, const double *b, const double *traces,
                                   double *r, double *rc, double *corner_scratch, cudaStream_t s);

constexpr int DOT_BLOCKS = 608;     // 4 x 152 SMs
constexpr int DOT_THREADS = 256;

}  // namespace dgmg
