// FP64 vector kernels of the outer conjugate-gradient loop: deterministic
// two-stage dot products (fixed grid, fixed reduction order), the CG updates
// with step lengths read from device memory, precision casts, and the
// right-hand-side quadrature (b_i = (f, phi_i), the right-hand side of
// Eq. weak_form_IP). The CG loop uses one multigrid cycle as its preconditioner
// (P^-1 of Sec. 5.1 "Exit criterion").
#include <algorithm>

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

// The same with 16-byte loads, two per vector in flight per thread (x, y
// 16-byte aligned); the n % 2 tail goes to the last thread of the grid.
__global__ void __launch_bounds__(DOT_THREADS) k_dot_partial_v(int64_t n, const double *__restrict__ x,
                                                               const double *__restrict__ y,
                                                               double *__restrict__ partials) {
    __shared__ double sh[32];
    const double2 *x2 = reinterpret_cast<const double2 *>(x), *y2 = reinterpret_cast<const double2 *>(y);
    const int64_t n2 = n >> 1, stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    for (; i + stride < n2; i += 2 * stride) {
        const double2 a = x2[i], b = y2[i], c = x2[i + stride], d = y2[i + stride];
        s0 = fma(a.x, b.x, s0);
        s0 = fma(a.y, b.y, s0);
        s1 = fma(c.x, d.x, s1);
        s1 = fma(c.y, d.y, s1);
    }
    if (i < n2) {
        const double2 a = x2[i], b = y2[i];
        s0 = fma(a.x, b.x, s0);
        s0 = fma(a.y, b.y, s0);
    }
    if ((n & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) s1 = fma(x[n - 1], y[n - 1], s1);
    const double s = block_sum(s0 + s1, sh);
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
//
// Vectorised form: 16-byte loads, two float4 per vector in flight per thread;
// the four products of a float4 are summed in FP32 (fused multiply-adds) and
// each such group sum is accumulated in FP64. A group sum carries an error of
// a few FP32 ulps of its terms, the order of the FP32 rounding of the vector
// entries themselves. The n % 4 tail goes to the last thread of the grid.
__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}

// partials[block] = sum x.y; with z: partials[gridDim + block] = sum z.y
template <bool TWO>
__global__ void __launch_bounds__(DOT_THREADS) k_dotf_partial_v(int64_t n, const float *__restrict__ x,
                                                                const float *__restrict__ y,
                                                                const float *__restrict__ z,
                                                                double *__restrict__ partials) {
    __shared__ double sh[32];
    const float4 *x4 = reinterpret_cast<const float4 *>(x), *y4 = reinterpret_cast<const float4 *>(y);
    const float4 *z4 = reinterpret_cast<const float4 *>(z);
    const int64_t n4 = n >> 2, stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0, t = 0.0;
    for (; i + stride < n4; i += 2 * stride) {
        const float4 b0 = y4[i], b1 = y4[i + stride];
        const float4 a0 = x4[i], a1 = x4[i + stride];
        if (TWO) {
            const float4 c0 = z4[i], c1 = z4[i + stride];
            t += (double)dot4(c0, b0) + (double)dot4(c1, b1);
        }
        s += (double)dot4(a0, b0) + (double)dot4(a1, b1);
    }
    if (i < n4) {
        const float4 b0 = y4[i];
        s += (double)dot4(x4[i], b0);
        if (TWO) t += (double)dot4(z4[i], b0);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1)
        for (int64_t k = n4 << 2; k < n; ++k) {
            s += (double)x[k] * (double)y[k];
            if (TWO) t += (double)z[k] * (double)y[k];
        }
    s = block_sum(s, sh);
    if (TWO) {
        __syncthreads();
        t = block_sum(t, sh);
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        if (TWO) partials[gridDim.x + blockIdx.x] = t;
    }
}

// xs += alpha p, r -= alpha q, rold = old r, and partials[block] = sum of the
// new r squared (the CG update and the residual norm in one pass; 16-byte
// aligned vectors; group sums as in k_dotf_partial_v)
__global__ void __launch_bounds__(DOT_THREADS) k_update_xr_dot_f(int64_t n, float *__restrict__ xs,
                                                                 float *__restrict__ r, float *__restrict__ rold,
                                                                 const float *__restrict__ p,
                                                                 const float *__restrict__ q,
                                                                 const double *__restrict__ scal,
                                                                 double *__restrict__ partials) {
    __shared__ double sh[32];
    const float alpha = (float)(scal[0] / scal[1]);
    float4 *xs4 = reinterpret_cast<float4 *>(xs), *r4 = reinterpret_cast<float4 *>(r);
    float4 *ro4 = reinterpret_cast<float4 *>(rold);
    const float4 *p4 = reinterpret_cast<const float4 *>(p), *q4 = reinterpret_cast<const float4 *>(q);
    const int64_t n4 = n >> 2, stride = (int64_t)gridDim.x * blockDim.x;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 ri = r4[i], pi = p4[i], qi = q4[i];
        float4 xi = xs4[i];
        if (rold) ro4[i] = ri;
        xi.x = fmaf(alpha, pi.x, xi.x);
        xi.y = fmaf(alpha, pi.y, xi.y);
        xi.z = fmaf(alpha, pi.z, xi.z);
        xi.w = fmaf(alpha, pi.w, xi.w);
        float4 rn;
        rn.x = fmaf(-alpha, qi.x, ri.x);
        rn.y = fmaf(-alpha, qi.y, ri.y);
        rn.z = fmaf(-alpha, qi.z, ri.z);
        rn.w = fmaf(-alpha, qi.w, ri.w);
        xs4[i] = xi;
        r4[i] = rn;
        s += (double)dot4(rn, rn);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1)
        for (int64_t k = n4 << 2; k < n; ++k) {
            const float ri = r[k];
            if (rold) rold[k] = ri;
            xs[k] = fmaf(alpha, p[k], xs[k]);
            const float rn = fmaf(-alpha, q[k], ri);
            r[k] = rn;
            s += (double)rn * (double)rn;
        }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

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
// values V[i][g] (q x mq) and w = product of the 1D Gauss weights scaled to the
// cell, sum-factorised: one CTA per cell contracts the mq^d point values with
// W_a[i][g] = V[i][g] w_a[g] one axis at a time (x, then y, then z).
constexpr int LV_THREADS = 128;
constexpr int LV_MQ = QMAX + 1;     // Gauss points per axis of the load quadrature (p + 2)
__global__ void __launch_bounds__(LV_THREADS) k_load_vector(int dim, int q, int mq, int64_t ncell,
                                                            const double *__restrict__ V,
                                                            const double *__restrict__ wq,
                                                            const double *__restrict__ fq, double *__restrict__ b) {
    __shared__ double sW[3][QMAX * LV_MQ];
    __shared__ double sF[LV_MQ * LV_MQ * LV_MQ];
    __shared__ double s1[QMAX * LV_MQ * LV_MQ];
    __shared__ double s2[QMAX * QMAX * LV_MQ];
    const int64_t cell = blockIdx.x;
    const int t = threadIdx.x;
    const int npc = dim == 3 ? mq * mq * mq : mq * mq;
    for (int e = t; e < dim * q * mq; e += blockDim.x) {
        const int a = e / (q * mq), r = e - a * q * mq, g = r % mq;
        sW[a][r] = V[r] * wq[a * mq + g];
    }
    for (int e = t; e < npc; e += blockDim.x) sF[e] = fq[cell * npc + e];
    __syncthreads();
    // x: s1[i + q (g2 + mq g3)] = sum_g1 W_x[i][g1] f[g1 + mq (g2 + mq g3)]
    const int n1 = dim == 3 ? q * mq * mq : q * mq;
    for (int e = t; e < n1; e += blockDim.x) {
        const int i = e % q, rest = e / q;
        double s = 0.0;
        for (int g = 0; g < mq; ++g) s = fma(sW[0][i * mq + g], sF[g + mq * rest], s);
        s1[e] = s;
    }
    __syncthreads();
    const int nl = dim == 3 ? q * q * q : q * q;
    double *out = b + cell * nl;
    if (dim == 2) {
        // y: b[i + q j] = sum_g2 W_y[j][g2] s1[i + q g2]
        for (int e = t; e < nl; e += blockDim.x) {
            const int i = e % q, j = e / q;
            double s = 0.0;
            for (int g = 0; g < mq; ++g) s = fma(sW[1][j * mq + g], s1[i + q * g], s);
            out[e] = s;
        }
        return;
    }
    // y: s2[i + q (j + q g3)] = sum_g2 W_y[j][g2] s1[i + q (g2 + mq g3)]
    const int n2 = q * q * mq;
    for (int e = t; e < n2; e += blockDim.x) {
        const int i = e % q, j = (e / q) % q, g3 = e / (q * q);
        double s = 0.0;
        for (int g = 0; g < mq; ++g) s = fma(sW[1][j * mq + g], s1[i + q * (g + mq * g3)], s);
        s2[e] = s;
    }
    __syncthreads();
    // z: b[i + q (j + q k)] = sum_g3 W_z[k][g3] s2[i + q (j + q g3)]
    for (int e = t; e < nl; e += blockDim.x) {
        const int ij = e % (q * q), k = e / (q * q);
        double s = 0.0;
        for (int g = 0; g < mq; ++g) s = fma(sW[2][k * mq + g], s2[ij + q * q * g], s);
        out[e] = s;
    }
}

inline unsigned grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 4 * 152 * 4 ? (b > 0 ? b : 1) : 4 * 152 * 4);
}

}  // namespace

inline bool aligned16(const void *a, const void *b, const void *c = nullptr, const void *d = nullptr,
                      const void *e = nullptr) {
    return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c) |
             reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(e)) & 15) == 0;
}

cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *partials, double *out, cudaStream_t s) {
    count_launches(2);
    if (aligned16(x, y))
        k_dot_partial_v<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(n, x, y, partials);
    else
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
    if (q > QMAX || mq > LV_MQ || ncell > 0x7fffffff) return cudaErrorInvalidValue;
    count_launches(1);
    k_load_vector<<<(unsigned)ncell, LV_THREADS, 0, s>>>(dim, q, mq, ncell, V, wq, fq, b);
    return cudaGetLastError();
}

cudaError_t launch_dotf(int64_t n, const float *x, const float *y, double *partials, double *out, cudaStream_t s) {
    count_launches(2);
    if (aligned16(x, y))
        k_dotf_partial_v<false><<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(n, x, y, nullptr, partials);
    else
        k_dotf_partial<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(n, x, y, partials);
    k_reduce<<<1, 512, 0, s>>>(DOT_BLOCKS, partials, out);
    return cudaGetLastError();
}

cudaError_t launch_dot2f(int64_t n, const float *x, const float *y, const float *z, double *partials,
                         double *out_xy, double *out_zy, cudaStream_t s) {
    count_launches(3);
    if (aligned16(x, y, z))
        k_dotf_partial_v<true><<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(n, x, y, z, partials);
    else
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

cudaError_t launch_update_xr_dot_f(int64_t n, float *xs, float *r, float *rold, const float *p, const float *q,
                                   const double *scal, double *partials, double *out_rr, cudaStream_t s) {
    if (!aligned16(xs, r, rold, p, q)) {
        const cudaError_t e = launch_update_xr_f(n, xs, r, rold, p, q, scal, s);
        if (e != cudaSuccess) return e;
        return launch_dotf(n, r, r, partials, out_rr, s);
    }
    count_launches(2);
    k_update_xr_dot_f<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(n, xs, r, rold, p, q, scal, partials);
    k_reduce<<<1, 512, 0, s>>>(DOT_BLOCKS, partials, out_rr);
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


// ---------------------------------------------------------------- FMA peak
// Every thread runs CH independent chains of fused multiply-adds (x <- x a + b,
// |a| < 1, so the values stay bounded); the chains' sum is stored only if it
// equals a value it cannot reach, which keeps the work live without a store.
__device__ double g_fma_sink;   // external linkage: the store cannot be dropped

// Register operands only: a and b pass through an opaque move per chain, so the
// multiply-add reads no constant-bank operand.
__device__ __forceinline__ double opaque(double v) {
    double r;
    asm volatile("mov.b64 %0, %1;" : "=d"(r) : "d"(v));
    return r;
}
__device__ __forceinline__ float opaque(float v) {
    float r;
    asm volatile("mov.b32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma_loop(int iters, T a, T b) {
    T x[CH], ac[CH], bc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        x[c] = (T)(threadIdx.x + c) * (T)1e-3;
        ac[c] = opaque(a);
        bc[c] = opaque(b);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = fma(x[c], ac[c], bc[c]);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    if (s == (T)-1.0) g_fma_sink = (double)s;
}

// The same on packed pairs: one instruction updates two lanes of a float2.
template <int CH>
__global__ void __launch_bounds__(256) k_fma_loop_x2(int iters, float a, float b) {
    float2 x[CH];
    const float2 a2 = make_float2(opaque(a), opaque(a)), b2 = make_float2(opaque(b), opaque(b));
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = make_float2((threadIdx.x + c) * 1e-3f, (threadIdx.x + c) * 2e-3f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c].x + x[c].y;
    if (s == -1.f) g_fma_sink = (double)s;
}

}  // namespace dgmg

extern "C" int dgmg_fma_peak(int kind, double *tflops, void *stream) {
    using namespace dgmg;
    if (!tflops) return fail(DGMG_EINVAL, "dgmg_fma_peak: tflops is NULL");
    if (kind < 0 || kind > 2) return fail(DGMG_EINVAL, "dgmg_fma_peak: kind must be 0, 1 or 2");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per = 0;
    DG_CUDA(cudaGetDevice(&dev));
    DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    constexpr int CH = 8, TPB = 256;
    if (kind == 0)
        DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_loop<double, CH>, TPB, 0));
    else if (kind == 1)
        DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_loop<float, CH>, TPB, 0));
    else
        DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_loop_x2<CH>, TPB, 0));
    per = per > 0 ? per : 1;
    const double lanes = kind == 2 ? 2.0 : 1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DG_CUDA(cudaEventCreate(&e0));
    DG_CUDA(cudaEventCreate(&e1));
    auto run = [&](int blocks, int iters) -> cudaError_t {
        count_launches(1);
        if (kind == 0)
            k_fma_loop<double, CH><<<blocks, TPB, 0, s>>>(iters, 0.999999, 1e-7);
        else if (kind == 1)
            k_fma_loop<float, CH><<<blocks, TPB, 0, s>>>(iters, 0.9999f, 1e-4f);
        else
            k_fma_loop_x2<CH><<<blocks, TPB, 0, s>>>(iters, 0.9999f, 1e-4f);
        return cudaGetLastError();
    };
    // resident blocks per SM from one to the occupancy limit; per shape the
    // iterations are calibrated to about 30 ms, then the best of three timed
    // launches is kept; the best shape gives the peak
    double best_rate = 0.0;
    cudaError_t e = cudaSuccess;
    int shapes[16], nshape = 0;
    for (int b = 1; b < per && nshape < 15; b *= 2) shapes[nshape++] = b;
    shapes[nshape++] = per;
    for (int si = 0; si < nshape && e == cudaSuccess; ++si) {
        const int blocks = sms * shapes[si];
        int iters = kind == 0 ? 64 : 2048;
        float ms = 0.f, best = 0.f;
        e = run(blocks, iters);   // warm-up
        for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = run(blocks, iters);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            if (k < 3) {
                if (ms < 30.f)
                    iters = (int)std::min<double>(iters * std::max(2.0, 30.0 / std::max(ms, 0.01f)), 1 << 26);
                continue;
            }
            if (best == 0.f || ms < best) best = ms;
        }
        if (e == cudaSuccess && best > 0.f) {
            const double fmas = (double)blocks * TPB * CH * 4.0 * iters * lanes;
            best_rate = std::max(best_rate, 2.0 * fmas / (best * 1e-3) / 1e12);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "dgmg_fma_peak");
    *tflops = best_rate;
    return DGMG_OK;
}
