// Per-cell fast-diagonalisation factors of the exact diagonal blocks, computed
// on the device at set-up: the GPU form of the paper's independent per-cell
// "matrix inversion" tasks (Technique 6), one thread per (cell, axis).
//
// For axis a of cell K the 1D block is
//   Kt_a = kappa_K K_a + low face  kF_L (w_L (e0 d0^T + d0 e0^T) + gamma e0 e0^T)
//                      + high face kF_R (-w_R (ep dp^T + dp ep^T) + gamma ep ep^T)
// (kF the harmonic mean of kappa and w = 1/2 inside, kF = kappa_K and w = 1 on
// the boundary; Technique 4: the interior values for every cell), and the
// factors solve Kt_a S = M_a S Lambda with S^T M_a S = I: with L L^T = M_a,
// C = L^-1 Kt_a L^-T = V Lambda V^T by cyclic Jacobi rotations, S = L^-T V.
// Everything is computed in FP64; the output is FP64 or rounded to FP32.
#include "internal.h"

namespace dgmg {

namespace {

// Eigen-decomposition of the symmetric n x n matrix A (overwritten) by cyclic
// Jacobi rotations, row by row (Jacobi 1846): V = eigenvectors (columns),
// lam = eigenvalues. Stops when the off-diagonal part is at rounding level or a
// sweep rotates nothing; at most 64 sweeps.
__device__ void jacobi_eig_dev(int n, double *A, double *V, double *lam) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double v = A[i * n + j] * A[i * n + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot) break;
        int rotations = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int r = p + 1; r < n; ++r) {
                const double apr = A[p * n + r];
                if (fabs(apr) <= 1e-18 * sqrt(fabs(A[p * n + p] * A[r * n + r])) || fabs(apr) < 1e-300) continue;
                ++rotations;
                // the rotation that zeroes A[p][r]: tan t = sign(theta) / (|theta| + sqrt(theta^2 + 1))
                const double theta = (A[r * n + r] - A[p * n + p]) / (2.0 * apr);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[k * n + p], akr = A[k * n + r];
                    A[k * n + p] = c * akp - s * akr;
                    A[k * n + r] = s * akp + c * akr;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[p * n + k], ark = A[r * n + k];
                    A[p * n + k] = c * apk - s * ark;
                    A[r * n + k] = s * apk + c * ark;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k * n + p], vkr = V[k * n + r];
                    V[k * n + p] = c * vkp - s * vkr;
                    V[k * n + r] = s * vkp + c * vkr;
                }
            }
        if (rotations == 0) break;
    }
    for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

template <typename T>
__global__ void __launch_bounds__(128) k_fd_factors(const __grid_constant__ FDInput in,
                                                    const double *__restrict__ kappa, int64_t ncell,
                                                    T *__restrict__ fd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncell * in.dim) return;
    const int64_t cell = idx / in.dim;
    const int a = (int)(idx - cell * in.dim), q = in.q;
    const int ci[3] = {(int)(cell % in.n[0]), (int)((cell / in.n[0]) % in.n[1]),
                       (int)(cell / ((int64_t)in.n[0] * in.n[1]))};
    const int64_t stride = a == 0 ? 1 : (a == 1 ? (int64_t)in.n[0] : (int64_t)in.n[0] * in.n[1]);
    const double kK = kappa[cell];
    double kL = kK, wL = 0.5, kR = kK, wR = 0.5;
    if (!in.interior_only) {
        if (ci[a] > 0) {
            const double kN = kappa[cell - stride];
            kL = 2.0 * kK * kN / (kK + kN);
        } else {
            wL = 1.0;
        }
        if (ci[a] < in.n[a] - 1) {
            const double kN = kappa[cell + stride];
            kR = 2.0 * kK * kN / (kK + kN);
        } else {
            wR = 1.0;
        }
    }
    const double *K = in.Kh[a], *L = in.Linv[a], *d0 = in.d0[a], *dp = in.dp[a];
    const double g = in.gam[a];
    double Kt[QMAX * QMAX], Tm[QMAX * QMAX], C[QMAX * QMAX], V[QMAX * QMAX], lam[QMAX];
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            const double e0i = in.e0[i], e0j = in.e0[j], epi = in.ep[i], epj = in.ep[j];
            Kt[i * q + j] = kK * K[i * q + j] + kL * (wL * (e0i * d0[j] + d0[i] * e0j) + g * e0i * e0j) +
                            kR * (-wR * (epi * dp[j] + dp[i] * epj) + g * epi * epj);
        }
    // C = L^-1 Kt L^-T, symmetrised
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            double s = 0.0;
            for (int k = 0; k < q; ++k) s += L[i * q + k] * Kt[k * q + j];
            Tm[i * q + j] = s;
        }
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            double s = 0.0;
            for (int k = 0; k < q; ++k) s += Tm[i * q + k] * L[j * q + k];
            C[i * q + j] = s;
        }
    for (int i = 0; i < q; ++i)
        for (int j = i + 1; j < q; ++j) C[i * q + j] = C[j * q + i] = 0.5 * (C[i * q + j] + C[j * q + i]);
    jacobi_eig_dev(q, C, V, lam);
    // S = L^-T V: S[m][i] = sum_k L[k][m] V[k][i]; stored [S (q x q) | lambda (q)]
    T *out = fd + idx * (q * q + q);
    for (int m = 0; m < q; ++m)
        for (int i = 0; i < q; ++i) {
            double s = 0.0;
            for (int k = m; k < q; ++k) s += L[k * q + m] * V[k * q + i];   // L^-1 is lower triangular
            out[m * q + i] = (T)s;
        }
    for (int i = 0; i < q; ++i) out[q * q + i] = (T)lam[i];
}

// linv[cell][node] = omega / (lambda_x[i] + lambda_y[j] (+ lambda_z[k])) from the
// factors: the inverse eigenvalue sums with the smoother's damping folded in
__global__ void k_inverse_eigen_sums(int dim, int q, int64_t ncell, const double *__restrict__ fd, double omega,
                                     double *__restrict__ linv) {
    const int64_t nloc = dim == 3 ? (int64_t)q * q * q : (int64_t)q * q;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncell * nloc) return;
    const int64_t cell = idx / nloc;
    const int node = (int)(idx - cell * nloc), fds = q * q + q;
    const double *f = fd + cell * dim * fds + q * q;
    double s = f[node % q] + f[fds + (node / q) % q];
    if (dim == 3) s += f[2 * fds + node / (q * q)];
    linv[idx] = omega / s;
}

// kfac[cell][f]: the harmonic mean of kappa across face f (0 on the boundary)
template <typename T>
__global__ void k_facet_coefficients(int dim, int n0, int n1, int n2, int64_t ncell, const double *__restrict__ kappa,
                                     T *__restrict__ kfac) {
    const int nface = 2 * dim;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncell * nface) return;
    const int64_t cell = idx / nface;
    const int f = (int)(idx - cell * nface), a = f >> 1, side = f & 1;
    const int64_t s1 = n0, s2 = (int64_t)n0 * n1;
    const int ci[3] = {(int)(cell % n0), (int)((cell / s1) % n1), (int)(cell / s2)};
    const int na = a == 0 ? n0 : (a == 1 ? n1 : n2);
    const int cn = ci[a] + (side ? 1 : -1);
    double v = 0.0;
    if (cn >= 0 && cn < na) {
        const int64_t st = a == 0 ? 1 : (a == 1 ? s1 : s2);
        const double kK = kappa[cell], kN = kappa[cell + (side ? st : -st)];
        v = 2.0 * kK * kN / (kK + kN);
    }
    kfac[idx] = (T)v;
}

}  // namespace

template <typename T>
cudaError_t launch_facet_coefficients(int dim, const int *n, int64_t ncell, const double *kappa, T *kfac,
                                      cudaStream_t s) {
    const int64_t m = ncell * 2 * dim;
    if (m == 0) return cudaSuccess;
    count_launches(1);
    k_facet_coefficients<T><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(dim, n[0], n[1], dim == 3 ? n[2] : 1, ncell,
                                                                        kappa, kfac);
    return cudaGetLastError();
}
template cudaError_t launch_facet_coefficients<double>(int, const int *, int64_t, const double *, double *, cudaStream_t);
template cudaError_t launch_facet_coefficients<float>(int, const int *, int64_t, const double *, float *, cudaStream_t);

template <typename T>
cudaError_t launch_fd_factors(const FDInput &in, const double *kappa, int64_t ncell, T *fd, cudaStream_t s) {
    const int64_t n = ncell * in.dim;
    if (n == 0) return cudaSuccess;
    count_launches(1);
    k_fd_factors<T><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(in, kappa, ncell, fd);
    return cudaGetLastError();
}
template cudaError_t launch_fd_factors<double>(const FDInput &, const double *, int64_t, double *, cudaStream_t);
template cudaError_t launch_fd_factors<float>(const FDInput &, const double *, int64_t, float *, cudaStream_t);

cudaError_t launch_inverse_eigen_sums(int dim, int q, int64_t ncell, const double *fd, double omega,
                                      double *linv, cudaStream_t s) {
    const int64_t n = ncell * (dim == 3 ? (int64_t)q * q * q : (int64_t)q * q);
    if (n == 0) return cudaSuccess;
    count_launches(1);
    k_inverse_eigen_sums<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dim, q, ncell, fd, omega, linv);
    return cudaGetLastError();
}

// Factors of the residual's A_KK u = (M S)^(xd) (sum of Lambda) (S^T M)^(xd):
// per (cell, axis) the matrix P = S^T M_a (q x q, row-major) and Lambda, in the
// layout of the smoother's factors [P | Lambda], from the cell's [S | Lambda]
// (FP64 or FP32) and the h-scaled 1D mass of the axis (FP64).
template <typename TI, typename TO>
__global__ void k_residual_factors(int dim, int q, int64_t ncell, const TI *__restrict__ fd, MassTables m,
                                   TO *__restrict__ fdr) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= ncell * dim) return;
    const int a = (int)(id % dim);
    const int fds = q * q + q;
    const TI *S = fd + id * fds;
    TO *P = fdr + id * fds;
    const double *M = m.M[a];
    for (int i = 0; i < q; ++i)
        for (int n = 0; n < q; ++n) {
            double v = 0.0;
            for (int l = 0; l < q; ++l) v += (double)S[l * q + i] * M[l * q + n];
            P[i * q + n] = (TO)v;
        }
    for (int i = 0; i < q; ++i) P[q * q + i] = (TO)S[q * q + i];
}

template <typename TI, typename TO>
cudaError_t launch_residual_factors(int dim, int q, int64_t ncell, const TI *fd, const MassTables &m, TO *fdr,
                                    cudaStream_t s) {
    const int64_t n = ncell * dim;
    if (n == 0) return cudaSuccess;
    count_launches(1);
    k_residual_factors<TI, TO><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(dim, q, ncell, fd, m, fdr);
    return cudaGetLastError();
}
template cudaError_t launch_residual_factors<double, double>(int, int, int64_t, const double *, const MassTables &,
                                                             double *, cudaStream_t);
template cudaError_t launch_residual_factors<double, float>(int, int, int64_t, const double *, const MassTables &,
                                                            float *, cudaStream_t);
template cudaError_t launch_residual_factors<float, float>(int, int, int64_t, const float *, const MassTables &,
                                                           float *, cudaStream_t);

}  // namespace dgmg
