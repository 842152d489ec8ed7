// FP64 vector kernels of the outer conjugate-gradient loop: deterministic
// two-stage dot products (fixed grid, fixed reduction order), the CG updates
// with step lengths read from device memory, precision casts, and the
// right-hand-side quadrature (b_i = (f, phi_i)).
#include "internal.h"

namespace dgmg {

namespace {

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;   // valid in thread 0
}

__global__ void k_dot_partial(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                              double *__restrict__ partials) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += x[i] * y[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_dot2_partial(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                               const double *__restrict__ z, double *__restrict__ partials) {
    __shared__ double sh[32];
    double s = 0.0, t = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double yi = y[i];
        s += x[i] * yi;
        t += z[i] * yi;
    }
    s = block_sum(s, sh);
    __syncthreads();
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        partials[gridDim.x + blockIdx.x] = t;
    }
}

__global__ void k_reduce(int np, const double *__restrict__ partials, double *__restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += partials[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

// slots of the scalar array used by the CG kernels
__global__ void k_update_xr(int64_t n, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                            const double *__restrict__ q, const double *__restrict__ scal) {
    const double alpha = scal[0] / scal[1];   // rz / pq
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
    }
}

__global__ void k_update_p(int64_t n, double *__restrict__ p, const double *__restrict__ z,
                           const double *__restrict__ scal) {
    const double beta = scal[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

__global__ void k_sub(int64_t n, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

__global__ void k_d2f(int64_t n, const double *__restrict__ x, float *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

__global__ void k_f2d(int64_t n, const float *__restrict__ x, double *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

__global__ void k_copy_scalar(const double *src, double *dst) { *dst = *src; }

// FP32 vectors with FP64 accumulation (the inner loop of the mixed solver)
__global__ void k_dotf_partial(int64_t n, const float *__restrict__ x, const float *__restrict__ y,
                               double *__restrict__ partials) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)x[i] * (double)y[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_dot2f_partial(int64_t n, const float *__restrict__ x, const float *__restrict__ y,
                                const float *__restrict__ z, double *__restrict__ partials) {
    __shared__ double sh[32];
    double s = 0.0, t = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double yi = y[i];
        s += (double)x[i] * yi;
        t += (double)z[i] * yi;
    }
    s = block_sum(s, sh);
    __syncthreads();
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        partials[gridDim.x + blockIdx.x] = t;
    }
}

// xs += alpha p, r -= alpha q, rold = old r (when given), alpha = scal[0] / scal[1]
__global__ void k_update_xr_f(int64_t n, float *__restrict__ xs, float *__restrict__ r, float *__restrict__ rold,
                              const float *__restrict__ p, const float *__restrict__ q,
                              const double *__restrict__ scal) {
    const float alpha = (float)(scal[0] / scal[1]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float ri = r[i];
        if (rold) rold[i] = ri;
        xs[i] += alpha * p[i];
        r[i] = ri - alpha * q[i];
    }
}

__global__ void k_update_p_f(int64_t n, float *__restrict__ p, const float *__restrict__ z,
                             const double *__restrict__ scal) {
    const float beta = (float)scal[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

// x += xs (FP64 accumulation of the FP32 correction), xs = 0
__global__ void k_accumulate_f2d(int64_t n, double *__restrict__ x, float *__restrict__ xs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += (double)xs[i];
        xs[i] = 0.0f;
    }
}


// physical coordinates of the mq^d Gauss points of every cell
__global__ void k_quad_points(int dim, int n0, int n1, int n2, int mq, const double *__restrict__ xq1,
                              double *__restrict__ xq, int64_t ncell) {
    const int64_t npc = dim == 3 ? (int64_t)mq * mq * mq : (int64_t)mq * mq;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncell * npc) return;
    const int64_t cell = idx / npc;
    const int g = (int)(idx % npc);
    const int gi[3] = {g % mq, (g / mq) % mq, g / (mq * mq)};
    const int ci[3] = {(int)(cell % n0), (int)((cell / n0) % n1), (int)(cell / ((int64_t)n0 * n1))};
    const int n[3] = {n0, n1, n2};
    for (int a = 0; a < dim; ++a) xq[idx * dim + a] = (ci[a] + 0.5 * (xq1[gi[a]] + 1.0)) / n[a];
}

// b[cell][node] = sum_g w_g f_g phi_node(x_g) with phi = product of 1D Lagrange
// values V[i][g] (q x mq) and w = product of the 1D Gauss weights scaled to the cell.
__global__ void k_load_vector(int dim, int q, int mq, int64_t ncell, const double *__restrict__ V,
                              const double *__restrict__ wq, const double *__restrict__ fq, double *__restrict__ b) {
    const int nl = dim == 3 ? q * q * q : q * q;
    const int npc = dim == 3 ? mq * mq * mq : mq * mq;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncell * nl) return;
    const int64_t cell = idx / nl;
    const int node = (int)(idx % nl);
    const int a[3] = {node % q, (node / q) % q, node / (q * q)};
    const double *f = fq + cell * npc;
    double s = 0.0;
    for (int g = 0; g < npc; ++g) {
        const int gi[3] = {g % mq, (g / mq) % mq, g / (mq * mq)};
        double w = 1.0;
        for (int d = 0; d < dim; ++d) w *= wq[d * mq + gi[d]] * V[a[d] * mq + gi[d]];
        s += w * f[g];
    }
    b[idx] = s;
}

inline unsigned grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 4 * 152 * 4 ? (b > 0 ? b : 1) : 4 * 152 * 4);
}

}  // namespace

cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *partials, double *out, cudaStream_t s) {
    count_launches(2);
    k_dot_partial<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(n, x, y, partials);
    k_reduce<<<1, 512, 0, s>>>(DOT_BLOCKS, partials, out);
    return cudaGetLastError();
}

cudaError_t launch_dot2(int64_t n, const double *x, const double *y, const double *z, double *partials,
                        double *out_xy, double *out_zy, cudaStream_t s) {
    count_launches(3);
    k_dot2_partial<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(n, x, y, z, partials);
    k_reduce<<<1, 512, 0, s>>>(DOT_BLOCKS, partials, out_xy);
    k_reduce<<<1, 512, 0, s>>>(DOT_BLOCKS, partials + DOT_BLOCKS, out_zy);
    return cudaGetLastError();
}

cudaError_t launch_cast_d2f(int64_t n, const double *x, float *y, cudaStream_t s) {
    count_launches(1);
    k_d2f<<<grid_for(n), 256, 0, s>>>(n, x, y);
    return cudaGetLastError();
}

cudaError_t launch_cast_f2d(int64_t n, const float *x, double *y, cudaStream_t s) {
    count_launches(1);
    k_f2d<<<grid_for(n), 256, 0, s>>>(n, x, y);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update_xr(int64_t n, double *x, double *r, const double *p, const double *q,
                                 const double *scal, cudaStream_t s) {
    count_launches(1);
    k_update_xr<<<grid_for(n), 256, 0, s>>>(n, x, r, p, q, scal);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update_p(int64_t n, double *p, const double *z, const double *scal, cudaStream_t s) {
    count_launches(1);
    k_update_p<<<grid_for(n), 256, 0, s>>>(n, p, z, scal);
    return cudaGetLastError();
}

cudaError_t launch_sub(int64_t n, const double *a, const double *b, double *out, cudaStream_t s) {
    count_launches(1);
    k_sub<<<grid_for(n), 256, 0, s>>>(n, a, b, out);
    return cudaGetLastError();
}

cudaError_t launch_copy_scalar(const double *src, double *dst, cudaStream_t s) {
    count_launches(1);
    k_copy_scalar<<<1, 1, 0, s>>>(src, dst);
    return cudaGetLastError();
}

cudaError_t launch_quad_points(int dim, int q, const int *n, int mq, const double *xq1, double *xq, int64_t ncell,
                               cudaStream_t s) {
    (void)q;
    const int64_t npc = dim == 3 ? (int64_t)mq * mq * mq : (int64_t)mq * mq;
    const int64_t tot = ncell * npc;
    if (tot == 0) return cudaSuccess;
    count_launches(1);
    k_quad_points<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(dim, n[0], n[1], dim == 3 ? n[2] : 1, mq, xq1, xq,
                                                                 ncell);
    return cudaGetLastError();
}

cudaError_t launch_load_vector(int dim, int q, int mq, int64_t ncell, const double *V, const double *wq,
                               const double *fq, double *b, cudaStream_t s) {
    const int64_t nl = dim == 3 ? (int64_t)q * q * q : (int64_t)q * q;
    const int64_t tot = ncell * nl;
    if (tot == 0) return cudaSuccess;
    count_launches(1);
    k_load_vector<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(dim, q, mq, ncell, V, wq, fq, b);
    return cudaGetLastError();
}

cudaError_t launch_dotf(int64_t n, const float *x, const float *y, double *partials, double *out, cudaStream_t s) {
    count_launches(2);
    k_dotf_partial<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(n, x, y, partials);
    k_reduce<<<1, 512, 0, s>>>(DOT_BLOCKS, partials, out);
    return cudaGetLastError();
}

cudaError_t launch_dot2f(int64_t n, const float *x, const float *y, const float *z, double *partials,
                         double *out_xy, double *out_zy, cudaStream_t s) {
    count_launches(3);
    k_dot2f_partial<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(n, x, y, z, partials);
    k_reduce<<<1, 512, 0, s>>>(DOT_BLOCKS, partials, out_xy);
    k_reduce<<<1, 512, 0, s>>>(DOT_BLOCKS, partials + DOT_BLOCKS, out_zy);
    return cudaGetLastError();
}

cudaError_t launch_update_xr_f(int64_t n, float *xs, float *r, float *rold, const float *p, const float *q,
                               const double *scal, cudaStream_t s) {
    count_launches(1);
    k_update_xr_f<<<grid_for(n), 256, 0, s>>>(n, xs, r, rold, p, q, scal);
    return cudaGetLastError();
}

cudaError_t launch_update_p_f(int64_t n, float *p, const float *z, const double *scal, cudaStream_t s) {
    count_launches(1);
    k_update_p_f<<<grid_for(n), 256, 0, s>>>(n, p, z, scal);
    return cudaGetLastError();
}

cudaError_t launch_accumulate_f2d(int64_t n, double *x, float *xs, cudaStream_t s) {
    count_launches(1);
    k_accumulate_f2d<<<grid_for(n), 256, 0, s>>>(n, x, xs);
    return cudaGetLastError();
}

}  // namespace dgmg
