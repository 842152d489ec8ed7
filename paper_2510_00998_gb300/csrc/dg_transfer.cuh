// Transfers between the DG levels of a gradual p-hierarchy (the nested DG spaces
// the outlook of Sec. 6.3 proposes; degree p_f on the
// same mesh as degree p_c = p_f - 1): the cellwise injection of the coarse
// polynomial space, P = I (x) I (x) I with I[i][j] = l_j^c(x_i^f) (the coarse
// Lagrange basis at the fine nodes), and its transpose for the restriction of
// residuals. Both are sum-factorised: one q_f x q_c contraction per axis.
#pragma once

namespace dgmg {

constexpr int TRANSFER_CELLS = 4;   // cells per CTA (static shared memory stays below 48 KB)
constexpr int TRANSFER_THREADS = 256;

// bc = (I^T (x) I^T (x) I^T) rf, cell by cell.
template <int DIM, int QF, typename T>
__global__ void __launch_bounds__(TRANSFER_THREADS) k_dg_restrict(int64_t ncell, const DGInterp<T> P,
                                                                  const T *__restrict__ rf, T *__restrict__ bc) {
    constexpr int QC = QF - 1;
    constexpr int NLF = DIM == 3 ? QF * QF * QF : QF * QF;
    constexpr int NLC = DIM == 3 ? QC * QC * QC : QC * QC;
    constexpr int NT1 = DIM == 3 ? QC * QF * QF : QC * QF;   // after the x contraction
    constexpr int NT2 = QC * QC * QF;                         // after the y contraction (3D)
    __shared__ T sR[TRANSFER_CELLS * NLF];
    __shared__ T s1[TRANSFER_CELLS * NT1];
    __shared__ T s2[TRANSFER_CELLS * (DIM == 3 ? NT2 : 1)];
    const int64_t cell0 = (int64_t)blockIdx.x * TRANSFER_CELLS;
    const int ncl = (int)min((int64_t)TRANSFER_CELLS, ncell - cell0);
    for (int e = threadIdx.x; e < ncl * NLF; e += blockDim.x) sR[e] = rf[cell0 * NLF + e];
    __syncthreads();
    // x: s1[c][ic + QC*(jf + QF*kf)] = sum_a I[a][ic] r[c][a + QF*(jf + QF*kf)]
    for (int e = threadIdx.x; e < ncl * NT1; e += blockDim.x) {
        const int c = e / NT1, o = e - c * NT1;
        const int ic = o % QC, rest = o / QC;
        T s = T(0);
#pragma unroll
        for (int a = 0; a < QF; ++a) s += P.I[a * QC + ic] * sR[c * NLF + a + QF * rest];
        s1[e] = s;
    }
    __syncthreads();
    if constexpr (DIM == 2) {
        // y: bc[c][ic + QC*jc] = sum_b I[b][jc] s1[c][ic + QC*b]
        for (int e = threadIdx.x; e < ncl * NLC; e += blockDim.x) {
            const int c = e / NLC, o = e - c * NLC;
            const int ic = o % QC, jc = o / QC;
            T s = T(0);
#pragma unroll
            for (int b = 0; b < QF; ++b) s += P.I[b * QC + jc] * s1[c * NT1 + ic + QC * b];
            bc[cell0 * NLC + e] = s;
        }
        return;
    }
    if constexpr (DIM == 3) {
        // y: s2[c][ic + QC*(jc + QC*kf)] = sum_b I[b][jc] s1[c][ic + QC*(b + QF*kf)]
        for (int e = threadIdx.x; e < ncl * NT2; e += blockDim.x) {
            const int c = e / NT2, o = e - c * NT2;
            const int ic = o % QC, jc = (o / QC) % QC, kf = o / (QC * QC);
            T s = T(0);
#pragma unroll
            for (int b = 0; b < QF; ++b) s += P.I[b * QC + jc] * s1[c * NT1 + ic + QC * (b + QF * kf)];
            s2[e] = s;
        }
        __syncthreads();
        // z: bc[c][ic + QC*(jc + QC*kc)] = sum_k I[k][kc] s2[c][ic + QC*(jc + QC*k)]
        for (int e = threadIdx.x; e < ncl * NLC; e += blockDim.x) {
            const int c = e / NLC, o = e - c * NLC;
            const int icjc = o % (QC * QC), kc = o / (QC * QC);
            T s = T(0);
#pragma unroll
            for (int k = 0; k < QF; ++k) s += P.I[k * QC + kc] * s2[c * NT2 + icjc + QC * QC * k];
            bc[cell0 * NLC + e] = s;
        }
    }
}

// zf += (I (x) I (x) I) ec, cell by cell.
template <int DIM, int QF, typename T>
__global__ void __launch_bounds__(TRANSFER_THREADS) k_dg_prolong(int64_t ncell, const DGInterp<T> P,
                                                                 const T *__restrict__ ec, T *__restrict__ zf) {
    constexpr int QC = QF - 1;
    constexpr int NLF = DIM == 3 ? QF * QF * QF : QF * QF;
    constexpr int NLC = DIM == 3 ? QC * QC * QC : QC * QC;
    constexpr int NT1 = DIM == 3 ? QF * QC * QC : QF * QC;   // after the x interpolation
    constexpr int NT2 = QF * QF * QC;                         // after the y interpolation (3D)
    __shared__ T sE[TRANSFER_CELLS * NLC];
    __shared__ T s1[TRANSFER_CELLS * NT1];
    __shared__ T s2[TRANSFER_CELLS * (DIM == 3 ? NT2 : 1)];
    const int64_t cell0 = (int64_t)blockIdx.x * TRANSFER_CELLS;
    const int ncl = (int)min((int64_t)TRANSFER_CELLS, ncell - cell0);
    for (int e = threadIdx.x; e < ncl * NLC; e += blockDim.x) sE[e] = ec[cell0 * NLC + e];
    __syncthreads();
    // x: s1[c][if + QF*(jc + QC*kc)] = sum_a I[if][a] e[c][a + QC*(jc + QC*kc)]
    for (int e = threadIdx.x; e < ncl * NT1; e += blockDim.x) {
        const int c = e / NT1, o = e - c * NT1;
        const int i = o % QF, rest = o / QF;
        T s = T(0);
#pragma unroll
        for (int a = 0; a < QC; ++a) s += P.I[i * QC + a] * sE[c * NLC + a + QC * rest];
        s1[e] = s;
    }
    __syncthreads();
    if constexpr (DIM == 2) {
        // y: zf[c][if + QF*jf] += sum_b I[jf][b] s1[c][if + QF*b]
        for (int e = threadIdx.x; e < ncl * NLF; e += blockDim.x) {
            const int c = e / NLF, o = e - c * NLF;
            const int i = o % QF, j = o / QF;
            T s = T(0);
#pragma unroll
            for (int b = 0; b < QC; ++b) s += P.I[j * QC + b] * s1[c * NT1 + i + QF * b];
            zf[cell0 * NLF + e] += s;
        }
        return;
    }
    if constexpr (DIM == 3) {
        // y: s2[c][if + QF*(jf + QF*kc)] = sum_b I[jf][b] s1[c][if + QF*(b + QC*kc)]
        for (int e = threadIdx.x; e < ncl * NT2; e += blockDim.x) {
            const int c = e / NT2, o = e - c * NT2;
            const int i = o % QF, j = (o / QF) % QF, kc = o / (QF * QF);
            T s = T(0);
#pragma unroll
            for (int b = 0; b < QC; ++b) s += P.I[j * QC + b] * s1[c * NT1 + i + QF * (b + QC * kc)];
            s2[e] = s;
        }
        __syncthreads();
        // z: zf[c][if + QF*(jf + QF*kf)] += sum_k I[kf][k] s2[c][if + QF*(jf + QF*k)]
        for (int e = threadIdx.x; e < ncl * NLF; e += blockDim.x) {
            const int c = e / NLF, o = e - c * NLF;
            const int ij = o % (QF * QF), kf = o / (QF * QF);
            T s = T(0);
#pragma unroll
            for (int k = 0; k < QC; ++k) s += P.I[kf * QC + k] * s2[c * NT2 + ij + QF * QF * k];
            zf[cell0 * NLF + e] += s;
        }
    }
}

template <int DIM, int QF, typename T>
cudaError_t launch_dg_transfer_q(bool prolong, int64_t ncell, const DGInterp<T> &P, const T *in, T *out,
                                 cudaStream_t s) {
    if constexpr (QF >= 3) {
        const unsigned grid = (unsigned)((ncell + TRANSFER_CELLS - 1) / TRANSFER_CELLS);
        if (grid == 0) return cudaSuccess;
        count_launches(1);
        if (prolong)
            k_dg_prolong<DIM, QF, T><<<grid, TRANSFER_THREADS, 0, s>>>(ncell, P, in, out);
        else
            k_dg_restrict<DIM, QF, T><<<grid, TRANSFER_THREADS, 0, s>>>(ncell, P, in, out);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_dg_transfer_impl(int dim, int qf, bool prolong, int64_t ncell, const DGInterp<T> &P, const T *in,
                                    T *out, cudaStream_t s) {
    switch (dim * 16 + qf) {
        case 2 * 16 + 3: return launch_dg_transfer_q<2, 3, T>(prolong, ncell, P, in, out, s);
        case 2 * 16 + 4: return launch_dg_transfer_q<2, 4, T>(prolong, ncell, P, in, out, s);
        case 2 * 16 + 5: return launch_dg_transfer_q<2, 5, T>(prolong, ncell, P, in, out, s);
        case 2 * 16 + 6: return launch_dg_transfer_q<2, 6, T>(prolong, ncell, P, in, out, s);
        case 2 * 16 + 7: return launch_dg_transfer_q<2, 7, T>(prolong, ncell, P, in, out, s);
        case 3 * 16 + 3: return launch_dg_transfer_q<3, 3, T>(prolong, ncell, P, in, out, s);
        case 3 * 16 + 4: return launch_dg_transfer_q<3, 4, T>(prolong, ncell, P, in, out, s);
        case 3 * 16 + 5: return launch_dg_transfer_q<3, 5, T>(prolong, ncell, P, in, out, s);
        case 3 * 16 + 6: return launch_dg_transfer_q<3, 6, T>(prolong, ncell, P, in, out, s);
        case 3 * 16 + 7: return launch_dg_transfer_q<3, 7, T>(prolong, ncell, P, in, out, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dgmg
