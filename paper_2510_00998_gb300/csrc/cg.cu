// Kernels of the continuous Q1 levels of the hp hierarchy (paper Sec. 2.4 and
// Sec. 5.2): the vertex gather of the p-restriction, damped point Jacobi with
// the 3^d-point Galerkin stencils, residual, nested h-restriction and
// h-prolongation, and the dense coarsest solve.
#include "internal.h"

namespace dgmg {

namespace {

constexpr int TPB = 256;

template <int DIM>
__device__ __forceinline__ void vcoords(int64_t v, const int *m, int *c) {
    c[0] = (int)(v % m[0]);
    const int64_t r = v / m[0];
    if (DIM == 3) {
        c[1] = (int)(r % m[1]);
        c[2] = (int)(r / m[1]);
    } else {
        c[1] = (int)r;
    }
}

// b0[v] = sum over the 2^d cells around interior vertex v of the cell's corner
// partial sum for that vertex (fixed order: deterministic p-restriction).
template <int DIM, typename T>
__device__ __forceinline__ void corner_gather_at(int n0, int n1, int n2, const T *__restrict__ corners,
                                                 T *__restrict__ b0, int64_t v) {
    const int m[3] = {n0 - 1, n1 - 1, n2 - 1};
    const int64_t nv = DIM == 3 ? (int64_t)m[0] * m[1] * m[2] : (int64_t)m[0] * m[1];
    if (v >= nv) return;
    int c[3];
    vcoords<DIM>(v, m, c);
    T s = T(0);
#pragma unroll
    for (int a = 0; a < (1 << DIM); ++a) {
        // cell with lower corner (vertex - 1 + a) along each axis; the vertex is
        // that cell's corner (1 - a) along each axis
        const int cx = c[0] + (a & 1), cy = c[1] + ((a >> 1) & 1), cz = DIM == 3 ? c[2] + ((a >> 2) & 1) : 0;
        const int64_t cell = cx + (int64_t)n0 * (cy + (int64_t)n1 * cz);
        const int corner = (~a) & ((1 << DIM) - 1);
        s += corners[cell * (1 << DIM) + corner];
    }
    b0[v] = s;
}

template <int DIM, typename T>
__global__ void k_corner_gather(int n0, int n1, int n2, const T *__restrict__ corners, T *__restrict__ b0) {
    corner_gather_at<DIM, T>(n0, n1, n2, corners, b0, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <int DIM, typename T>
__device__ __forceinline__ T stencil_apply(const CGLevelDev<T> &L, int64_t v, const int *c,
                                           const T *__restrict__ u) {
    constexpr int NS = DIM == 3 ? 27 : 9;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const int sx = k % 3 - 1, sy = (k / 3) % 3 - 1, sz = DIM == 3 ? k / 9 - 1 : 0;
        const int x = c[0] + sx, y = c[1] + sy, z = DIM == 3 ? c[2] + sz : 0;
        if (x < 0 || x >= L.m[0] || y < 0 || y >= L.m[1]) continue;
        if (DIM == 3 && (z < 0 || z >= L.m[2])) continue;
        const int64_t w = x + (int64_t)L.m[0] * (y + (int64_t)L.m[1] * z);
        s += L.st[(int64_t)k * L.nv + v] * u[w];
    }
    return s;
}

template <int DIM, typename T>
__device__ __forceinline__ void cg_jacobi_at(const CGLevelDev<T> &L, const T *__restrict__ u_in,
                                             const T *__restrict__ b, T *__restrict__ u_out, T omega,
                                             int zero_guess, int64_t v) {
    constexpr int NS = DIM == 3 ? 27 : 9;
    if (v >= L.nv) return;
    const T diag = L.st[(int64_t)(NS / 2) * L.nv + v];
    if (zero_guess) {
        u_out[v] = omega * b[v] / diag;
        return;
    }
    int c[3] = {0, 0, 0};
    vcoords<DIM>(v, L.m, c);
    const T au = stencil_apply<DIM, T>(L, v, c, u_in);
    u_out[v] = u_in[v] + omega * (b[v] - au) / diag;
}

template <int DIM, typename T>
__global__ void k_cg_jacobi(CGLevelDev<T> L, const T *__restrict__ u_in, const T *__restrict__ b,
                            T *__restrict__ u_out, T omega, int zero_guess) {
    cg_jacobi_at<DIM, T>(L, u_in, b, u_out, omega, zero_guess, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <int DIM, typename T>
__device__ __forceinline__ void cg_residual_at(const CGLevelDev<T> &L, const T *__restrict__ u,
                                               const T *__restrict__ b, T *__restrict__ r, int64_t v) {
    if (v >= L.nv) return;
    int c[3] = {0, 0, 0};
    vcoords<DIM>(v, L.m, c);
    r[v] = b[v] - stencil_apply<DIM, T>(L, v, c, u);
}

template <int DIM, typename T>
__global__ void k_cg_residual(CGLevelDev<T> L, const T *__restrict__ u, const T *__restrict__ b,
                              T *__restrict__ r) {
    cg_residual_at<DIM, T>(L, u, b, r, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// rc[V] = sum_i P_h[i][V] rf[i]: per axis, the fine children of coarse vertex V.
template <int DIM, typename T>
__device__ __forceinline__ void h_restrict_at(const CGLevelDev<T> &L, const T *__restrict__ rf, T *__restrict__ rc,
                                              int64_t V) {
    const int64_t ncv = DIM == 3 ? (int64_t)L.mc[0] * L.mc[1] * L.mc[2] : (int64_t)L.mc[0] * L.mc[1];
    if (V >= ncv) return;
    int C[3] = {0, 0, 0};
    vcoords<DIM>(V, L.mc, C);
    const int sx = L.rs_start[0][C[0]], nx = L.rs_cnt[0][C[0]];
    const int sy = L.rs_start[1][C[1]], ny = L.rs_cnt[1][C[1]];
    const int sz = DIM == 3 ? L.rs_start[2][C[2]] : 0, nz = DIM == 3 ? L.rs_cnt[2][C[2]] : 1;
    T s = T(0);
    for (int k = 0; k < nz; ++k) {
        const T wz = DIM == 3 ? L.rs_w[2][C[2] * 5 + k] : T(1);
        for (int j = 0; j < ny; ++j) {
            const T wyz = wz * L.rs_w[1][C[1] * 5 + j];
            const int64_t row = (int64_t)L.m[0] * ((sy + j) + (int64_t)L.m[1] * (sz + k));
            for (int i = 0; i < nx; ++i) s += wyz * L.rs_w[0][C[0] * 5 + i] * rf[row + sx + i];
        }
    }
    rc[V] = s;
}

template <int DIM, typename T>
__global__ void k_h_restrict(CGLevelDev<T> L, const T *__restrict__ rf, T *__restrict__ rc) {
    h_restrict_at<DIM, T>(L, rf, rc, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// uf[i] += sum_V P_h[i][V] ec[V]: per axis, the (at most two) coarse parents.
template <int DIM, typename T>
__device__ __forceinline__ void h_prolong_at(const CGLevelDev<T> &L, const T *__restrict__ ec, T *__restrict__ uf,
                                             int64_t v) {
    if (v >= L.nv) return;
    int c[3] = {0, 0, 0};
    vcoords<DIM>(v, L.m, c);
    int px[2] = {L.pl_lo[0][c[0]], L.pl_hi[0][c[0]]};
    T wx[2] = {L.pl_wlo[0][c[0]], L.pl_whi[0][c[0]]};
    int py[2] = {L.pl_lo[1][c[1]], L.pl_hi[1][c[1]]};
    T wy[2] = {L.pl_wlo[1][c[1]], L.pl_whi[1][c[1]]};
    int pz[2] = {0, -1};
    T wz[2] = {T(1), T(0)};
    if (DIM == 3) {
        pz[0] = L.pl_lo[2][c[2]];
        pz[1] = L.pl_hi[2][c[2]];
        wz[0] = L.pl_wlo[2][c[2]];
        wz[1] = L.pl_whi[2][c[2]];
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (pz[k] < 0) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (py[j] < 0) continue;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (px[i] < 0) continue;
                s += wx[i] * wy[j] * wz[k] * ec[px[i] + (int64_t)L.mc[0] * (py[j] + (int64_t)L.mc[1] * pz[k])];
            }
        }
    }
    uf[v] += s;
}

template <int DIM, typename T>
__global__ void k_h_prolong(CGLevelDev<T> L, const T *__restrict__ ec, T *__restrict__ uf) {
    h_prolong_at<DIM, T>(L, ec, uf, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// e = A_c^{-1} r with the explicit FP64 inverse of the coarsest operator.
template <typename T>
__device__ __forceinline__ void coarse_row(int64_t nc, const double *__restrict__ Ainv, const T *__restrict__ r,
                                           T *__restrict__ e, int64_t i) {
    if (i >= nc) return;
    double s = 0.0;
    for (int64_t j = 0; j < nc; ++j) s += Ainv[i * nc + j] * (double)r[j];
    e[i] = (T)s;
}

template <typename T>
__global__ void k_coarse_solve(int64_t nc, const double *__restrict__ Ainv, const T *__restrict__ r,
                               T *__restrict__ e) {
    coarse_row<T>(nc, Ainv, r, e, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---- batched forms: CTA k covers vertices [v0, v0 + BATCH_VERTS) of descriptor
// map[k].desc (one level of one instance); all instances share the launch.
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_corner_gather_batch(const BatchCG<T> *__restrict__ D,
                                                                     const VertMap *__restrict__ map) {
    const VertMap m = map[blockIdx.x];
    const BatchCG<T> &d = D[m.desc];
    corner_gather_at<DIM, T>(d.n[0], d.n[1], d.n[2], d.corners, d.b, (int64_t)m.v0 + threadIdx.x);
}
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_cg_jacobi_batch(const BatchCG<T> *__restrict__ D,
                                                                 const VertMap *__restrict__ map, T omega,
                                                                 int zero_guess, int cur) {
    const VertMap m = map[blockIdx.x];
    const BatchCG<T> &d = D[m.desc];
    cg_jacobi_at<DIM, T>(d.L, d.u[cur], d.b, d.u[cur ^ 1], omega, zero_guess, (int64_t)m.v0 + threadIdx.x);
}
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_cg_residual_batch(const BatchCG<T> *__restrict__ D,
                                                                   const VertMap *__restrict__ map, int cur) {
    const VertMap m = map[blockIdx.x];
    const BatchCG<T> &d = D[m.desc];
    cg_residual_at<DIM, T>(d.L, d.u[cur], d.b, d.r, (int64_t)m.v0 + threadIdx.x);
}
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_h_restrict_batch(const BatchCG<T> *__restrict__ D,
                                                                  const VertMap *__restrict__ map) {
    const VertMap m = map[blockIdx.x];
    const BatchCG<T> &d = D[m.desc];
    h_restrict_at<DIM, T>(d.L, d.r, d.b_next, (int64_t)m.v0 + threadIdx.x);
}
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_h_prolong_batch(const BatchCG<T> *__restrict__ D,
                                                                 const VertMap *__restrict__ map, int cur) {
    const VertMap m = map[blockIdx.x];
    const BatchCG<T> &d = D[m.desc];
    h_prolong_at<DIM, T>(d.L, d.e_next, d.u[cur], (int64_t)m.v0 + threadIdx.x);
}
template <typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_coarse_solve_batch(const BatchCG<T> *__restrict__ D,
                                                                    const VertMap *__restrict__ map) {
    const VertMap m = map[blockIdx.x];
    const BatchCG<T> &d = D[m.desc];
    coarse_row<T>(d.L.nv, d.Ainv, d.b, d.u[0], (int64_t)m.v0 + threadIdx.x);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

}  // namespace

template <typename T>
cudaError_t launch_corner_gather(int dim, const int *n, const T *corners, T *b0, cudaStream_t s) {
    const int64_t nv = dim == 3 ? (int64_t)(n[0] - 1) * (n[1] - 1) * (n[2] - 1) : (int64_t)(n[0] - 1) * (n[1] - 1);
    if (nv <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_corner_gather<3, T><<<blocks_for(nv), TPB, 0, s>>>(n[0], n[1], n[2], corners, b0);
    else
        k_corner_gather<2, T><<<blocks_for(nv), TPB, 0, s>>>(n[0], n[1], 1, corners, b0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_jacobi(int dim, const CGLevelDev<T> &L, const T *u_in, const T *b, T *u_out, T omega,
                             bool zero_guess, cudaStream_t s) {
    if (L.nv <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_cg_jacobi<3, T><<<blocks_for(L.nv), TPB, 0, s>>>(L, u_in, b, u_out, omega, zero_guess ? 1 : 0);
    else
        k_cg_jacobi<2, T><<<blocks_for(L.nv), TPB, 0, s>>>(L, u_in, b, u_out, omega, zero_guess ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_residual(int dim, const CGLevelDev<T> &L, const T *u, const T *b, T *r, cudaStream_t s) {
    if (L.nv <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_cg_residual<3, T><<<blocks_for(L.nv), TPB, 0, s>>>(L, u, b, r);
    else
        k_cg_residual<2, T><<<blocks_for(L.nv), TPB, 0, s>>>(L, u, b, r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_h_restrict(int dim, const CGLevelDev<T> &L, const T *rf, T *rc, cudaStream_t s) {
    const int64_t ncv = dim == 3 ? (int64_t)L.mc[0] * L.mc[1] * L.mc[2] : (int64_t)L.mc[0] * L.mc[1];
    if (ncv <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_h_restrict<3, T><<<blocks_for(ncv), TPB, 0, s>>>(L, rf, rc);
    else
        k_h_restrict<2, T><<<blocks_for(ncv), TPB, 0, s>>>(L, rf, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_h_prolong(int dim, const CGLevelDev<T> &L, const T *ec, T *uf, cudaStream_t s) {
    if (L.nv <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_h_prolong<3, T><<<blocks_for(L.nv), TPB, 0, s>>>(L, ec, uf);
    else
        k_h_prolong<2, T><<<blocks_for(L.nv), TPB, 0, s>>>(L, ec, uf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(int64_t nc, const double *Ainv, const T *r, T *e, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    count_launches(1);
    k_coarse_solve<T><<<blocks_for(nc), TPB, 0, s>>>(nc, Ainv, r, e);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_corner_gather_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_corner_gather_batch<3, T><<<nb, BATCH_VERTS, 0, s>>>(D, map);
    else
        k_corner_gather_batch<2, T><<<nb, BATCH_VERTS, 0, s>>>(D, map);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_jacobi_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, T omega,
                                   bool zero_guess, int cur, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_cg_jacobi_batch<3, T><<<nb, BATCH_VERTS, 0, s>>>(D, map, omega, zero_guess ? 1 : 0, cur);
    else
        k_cg_jacobi_batch<2, T><<<nb, BATCH_VERTS, 0, s>>>(D, map, omega, zero_guess ? 1 : 0, cur);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_residual_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, int cur,
                                     cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_cg_residual_batch<3, T><<<nb, BATCH_VERTS, 0, s>>>(D, map, cur);
    else
        k_cg_residual_batch<2, T><<<nb, BATCH_VERTS, 0, s>>>(D, map, cur);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_h_restrict_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_h_restrict_batch<3, T><<<nb, BATCH_VERTS, 0, s>>>(D, map);
    else
        k_h_restrict_batch<2, T><<<nb, BATCH_VERTS, 0, s>>>(D, map);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_h_prolong_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, int cur,
                                   cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_h_prolong_batch<3, T><<<nb, BATCH_VERTS, 0, s>>>(D, map, cur);
    else
        k_h_prolong_batch<2, T><<<nb, BATCH_VERTS, 0, s>>>(D, map, cur);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve_batch(const BatchCG<T> *D, const VertMap *map, int nb, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    k_coarse_solve_batch<T><<<nb, BATCH_VERTS, 0, s>>>(D, map);
    return cudaGetLastError();
}

#define DGMG_CG_INST(T)                                                                                         \
    template cudaError_t launch_corner_gather<T>(int, const int *, const T *, T *, cudaStream_t);              \
    template cudaError_t launch_cg_jacobi<T>(int, const CGLevelDev<T> &, const T *, const T *, T *, T, bool,   \
                                             cudaStream_t);                                                    \
    template cudaError_t launch_cg_residual<T>(int, const CGLevelDev<T> &, const T *, const T *, T *,          \
                                               cudaStream_t);                                                  \
    template cudaError_t launch_h_restrict<T>(int, const CGLevelDev<T> &, const T *, T *, cudaStream_t);       \
    template cudaError_t launch_h_prolong<T>(int, const CGLevelDev<T> &, const T *, T *, cudaStream_t);        \
    template cudaError_t launch_coarse_solve<T>(int64_t, const double *, const T *, T *, cudaStream_t);        \
    template cudaError_t launch_corner_gather_batch<T>(int, const BatchCG<T> *, const VertMap *, int,           \
                                                       cudaStream_t);                                          \
    template cudaError_t launch_cg_jacobi_batch<T>(int, const BatchCG<T> *, const VertMap *, int, T, bool, int, \
                                                   cudaStream_t);                                              \
    template cudaError_t launch_cg_residual_batch<T>(int, const BatchCG<T> *, const VertMap *, int, int,         \
                                                     cudaStream_t);                                            \
    template cudaError_t launch_h_restrict_batch<T>(int, const BatchCG<T> *, const VertMap *, int, cudaStream_t); \
    template cudaError_t launch_h_prolong_batch<T>(int, const BatchCG<T> *, const VertMap *, int, int,          \
                                                   cudaStream_t);                                              \
    template cudaError_t launch_coarse_solve_batch<T>(const BatchCG<T> *, const VertMap *, int, cudaStream_t);

DGMG_CG_INST(double)
DGMG_CG_INST(float)

}  // namespace dgmg
