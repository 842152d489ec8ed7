// DG-level kernels of the SIPG hp-multigrid path: warm-up projection (with the
// fused p-prolongation), the single-touch block-Jacobi smoothing step and the
// residual (with the fused p-restriction). Templated on dimension, nodes per
// axis and arithmetic type; instantiated in dg_fp64.cu and dg_fp32.cu.
//
// Work decomposition. A CTA owns `cpb` consecutive cells; each cell is served
// by q^(d-1) threads. In a "pass along axis a" thread t of a cell owns the
// pencil of q nodes along axis a through the tangential position t (t = lower
// remaining axis + q * upper remaining axis), loads it from shared memory into
// registers, applies a q x q matrix and stores it back; a CTA barrier separates
// passes along different axes. Face node t of the two faces normal to axis a
// is the end of pencil t, so facet work maps onto the same threads.
//
// Trace layout (the projection variables of the paper's Technique 1, stored
// per cell): tr[cell][face][comp][t], face = 2*axis + side (side 0 = low end,
// 1 = high end), comp 0 = value u, comp 1 = derivative along +axis.
#pragma once

#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace dgmg {

template <int DIM, int Q, typename T = float>
struct Geo {
    static constexpr int NL = DIM == 3 ? Q * Q * Q : Q * Q;   // nodes per cell
    static constexpr int NF = NL / Q;                          // nodes per face = threads per cell
    static constexpr int NFACE = 2 * DIM;
    static constexpr int FS = trace_face_stride<T>(NF);         // trace values per face (padded)
    static constexpr int TR = NFACE * FS;                      // trace values per cell
    static constexpr int NC = 1 << DIM;                        // corners per cell
    static constexpr int FDS = Q * Q + Q;                      // fast-diag factors per axis (global)
    static constexpr int VEC = 16 / (int)sizeof(T);            // elements per 16-byte vector
    static constexpr int FDSP = (FDS + VEC - 1) / VEC * VEC;   // per axis in shared memory (padded)
    static constexpr int QQV = (Q * Q + VEC - 1) / VEC;        // 16-byte vectors covering S
    static constexpr int NDOT = NFACE * 2 * (DIM == 3 ? Q : 1); // facet-mass dot products per cell
    static constexpr int NLC = NFACE * 2 * Q;                  // lifting coefficients per cell
    // volume index of node i of the pencil along `dir` at tangential position t
    static __device__ __forceinline__ int vidx(int dir, int t, int i) {
        if (DIM == 2) return dir == 0 ? i + Q * t : t + Q * i;
        if (dir == 0) return i + Q * t;
        if (dir == 1) return (t % Q) + Q * (i + Q * (t / Q));
        return t + Q * Q * i;
    }
};

template <int DIM>
__device__ __forceinline__ void cell_coords(int64_t cell, const int *n, int *ci) {
    ci[0] = (int)(cell % n[0]);
    int64_t r = cell / n[0];
    if (DIM == 3) {
        ci[1] = (int)(r % n[1]);
        ci[2] = (int)(r / n[1]);
    } else {
        ci[1] = (int)r;
    }
}

template <int DIM>
__device__ __forceinline__ int64_t axis_stride(const int *n, int dir) {
    return dir == 0 ? 1 : (dir == 1 ? (int64_t)n[0] : (int64_t)n[0] * n[1]);
}

// Cooperative copy of `count` contiguous elements (all threads of the CTA).
template <typename T>
__device__ __forceinline__ void block_copy(T *__restrict__ dst, const T *__restrict__ src, int64_t count) {
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) dst[i] = src[i];
}

// Load one q x q factor matrix (16-byte aligned in shared memory) into
// registers with 16-byte vector loads.
template <int DIM, int Q, typename T>
__device__ __forceinline__ void load_factor(const T *src, T *dst) {
    using G = Geo<DIM, Q, T>;
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const V *s = reinterpret_cast<const V *>(src);
#pragma unroll
    for (int k = 0; k < G::QQV; ++k) reinterpret_cast<V *>(dst)[k] = s[k];
}

// 1D tables read with thread-dependent indices by build_block_1d, staged in
// shared memory: K [axis][q*q], then d0 [axis][q], then dp [axis][q].
template <int DIM, int Q, typename T>
__device__ __forceinline__ void stage_block_tables(const DGConst<T> &c, T *sT) {
    for (int e = threadIdx.x; e < DIM * Q * Q; e += blockDim.x) sT[e] = c.K[e / (Q * Q)][e % (Q * Q)];
    for (int e = threadIdx.x; e < DIM * Q; e += blockDim.x) {
        sT[DIM * Q * Q + e] = c.d0[e / Q][e % Q];
        sT[DIM * Q * Q + DIM * Q + e] = c.dp[e / Q][e % Q];
    }
}

// Bit f set when face f (= 2*axis + side) of the cell has a neighbour.
template <int DIM>
__device__ __forceinline__ int interior_mask(const int *ci, const int *n) {
    int m = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (ci[a] > 0) m |= 1 << (2 * a);
        if (ci[a] < n[a] - 1) m |= 1 << (2 * a + 1);
    }
    return m;
}

// Load the neighbours' traces of the faces of one cell into sF[face][comp][t]
// and the facet coefficient kF[face] (harmonic mean of kappa; 0 on the boundary,
// where the facet has no neighbour contribution).
template <int DIM, int Q, typename T>
__device__ __forceinline__ void load_neighbour_traces(const DGConst<T> &c, int64_t cell, const int *ci, int t,
                                                      const T *__restrict__ tr, const T *__restrict__ kappa,
                                                      T *sF, T *sKF, T *sKappa) {
    using G = Geo<DIM, Q, T>;
    const T kK = kappa[cell];
#pragma unroll
    for (int f = 0; f < G::NFACE; ++f) {
        const int dir = f >> 1, side = f & 1;
        const int cn = ci[dir] + (side ? 1 : -1);
        const bool inside = cn >= 0 && cn < c.n[dir];
        T g = T(0), h = T(0);
        if (inside) {
            const int64_t nb = cell + (side ? axis_stride<DIM>(c.n, dir) : -axis_stride<DIM>(c.n, dir));
            const T *src = tr + nb * G::TR + (f ^ 1) * G::FS;
            g = src[t];
            h = src[G::NF + t];
        }
        sF[(f * 2 + 0) * G::NF + t] = g;
        sF[(f * 2 + 1) * G::NF + t] = h;
    }
    // the facet coefficients (formed at set-up: the harmonic means of kappa)
    for (int f = t; f < G::NFACE; f += G::NF) sKF[f] = c.kfac[cell * G::NFACE + f];
    if (t == 0) *sKappa = kK;
}

// Apply the facet mass matrix (tensor product of the tangential 1D masses) to
// both components of every interior face of the cell, in place. Needs all
// threads of the CTA (contains barriers); `active` threads do the arithmetic.
// Each 1D mass in its rank-one form M = diag(w) - mu mu^T (sW, sU: [axis][q]
// in shared memory): per pass, first the dot products mu . (pencil) of every
// face, component and pencil, spread over the cell's threads into sD
// ([NFACE][2][lines], lines = q in 3D, 1 in 2D), then every node
// out = w f - mu (dot). Pass 0 runs along the lower tangential index ia,
// pass 1 (3D) along the upper one ib.
template <int DIM, int Q, typename T>
__device__ __forceinline__ void facet_mass(const T *sW, const T *sU, bool active, int t, T *sF, T *sD, int mask) {
    using G = Geo<DIM, Q, T>;
    constexpr int NPASS = DIM - 1;
    constexpr int LINES = DIM == 3 ? Q : 1;
    constexpr int ND = G::NFACE * 2 * LINES;
    const int ia = t % Q, ib = t / Q;
#pragma unroll
    for (int pass = 0; pass < NPASS; ++pass) {
        if (active) {
            for (int d = t; d < ND; d += G::NF) {
                const int line = d % LINES, fc = d / LINES, f = fc >> 1;
                const int dir = f >> 1;
                const int ax = pass == 0 ? (dir == 0 ? 1 : 0) : (dir == 2 ? 1 : 2);   // the pass's axis
                T s = T(0);
                if (mask & (1 << f)) {
                    const T *fld = sF + fc * G::NF;
#pragma unroll
                    for (int m = 0; m < Q; ++m)
                        s += sU[ax * Q + m] * (pass == 0 ? fld[m + Q * line] : fld[line + Q * m]);
                }
                sD[d] = s;
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int f = 0; f < G::NFACE; ++f) {
                if (!(mask & (1 << f))) continue;
                const int dir = f >> 1;
                const int ax = pass == 0 ? (dir == 0 ? 1 : 0) : (dir == 2 ? 1 : 2);
                const int node = pass == 0 ? ia : ib, line = DIM == 3 ? (pass == 0 ? ib : ia) : 0;
                const T w = sW[ax * Q + node], mu = sU[ax * Q + node];
#pragma unroll
                for (int comp = 0; comp < 2; ++comp) {
                    T *fld = sF + (f * 2 + comp) * G::NF;
                    fld[t] = w * fld[t] - mu * sD[(f * 2 + comp) * LINES + line];
                }
            }
        }
        __syncthreads();
    }
}

// stage the rank-one mass data of every axis: sW[a][i], sU[a][i]
template <int DIM, int Q, typename T>
__device__ __forceinline__ void stage_mass_rank1(const DGConst<T> &c, T *sW, T *sU) {
    for (int e = threadIdx.x; e < DIM * Q; e += blockDim.x) {
        sW[e] = c.mw[e / Q][e % Q];
        sU[e] = c.mu[e / Q][e % Q];
    }
}

// r -= N u_nb: the neighbours' part of the facet terms of the cell equation
// (all terms of Eq. weak_form_IP_facet_spaces that involve the neighbour's
// projections), lifted into the cell. sF holds the mass-applied neighbour
// fields G = M_t g, H = M_t h; e_0, e_p are the end values of the 1D basis
// (the first / last unit vector for GLL nodes). For the low face (cell = K^+):
//   N = kF [ e_0 (x) (H/2 - gamma G) - d_0 (x) G/2 ],
// for the high face (cell = K^-):
//   N = kF [ e_p (x) (-H/2 - gamma G) + d_p (x) G/2 ],
// so the pencil at a face node takes G cG - H cH with, per face,
//   low:  cG = kF (d_0/2 + gamma e_0),   cH = kF e_0 / 2,
//   high: cG = kF (gamma e_p - d_p/2),   cH = -kF e_p / 2,
// formed once per cell (lift_coefficients: sC[face][cG | cH]).
template <int DIM, int Q, typename T>
__device__ __forceinline__ void lift_coefficients(const DGConst<T> &c, bool active, int t, const T *sKF, int mask,
                                                  T *sC) {
    using G = Geo<DIM, Q, T>;
    if (!active) return;
    for (int e = t; e < G::NFACE * Q; e += G::NF) {
        const int f = e / Q, i = e - f * Q, dir = f >> 1, side = f & 1;
        if (!(mask & (1 << f))) continue;
        const T kF = sKF[f], h = T(0.5);
        const T ev = c.gl ? (side ? c.vp[i] : c.v0[i]) : T(i == (side ? Q - 1 : 0) ? 1 : 0);
        sC[f * 2 * Q + i] = side ? kF * (c.gamma[dir] * ev - h * c.dp[dir][i]) : kF * (h * c.d0[dir][i] + c.gamma[dir] * ev);
        sC[f * 2 * Q + Q + i] = side ? -(kF * h * ev) : kF * h * ev;
    }
}

template <int DIM, int Q, typename T>
__device__ __forceinline__ void lift_neighbours(const DGConst<T> &c, bool active, int t, T *sR, const T *sF,
                                                const T *sC, int mask) {
    using G = Geo<DIM, Q, T>;
#pragma unroll
    for (int dir = 0; dir < DIM; ++dir) {
        if (active) {
            T x[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) x[i] = sR[G::vidx(dir, t, i)];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int f = 2 * dir + side;
                if (!(mask & (1 << f))) continue;
                const T Gv = sF[(f * 2 + 0) * G::NF + t];
                const T Hv = sF[(f * 2 + 1) * G::NF + t];
                const T *cf = sC + f * 2 * Q;
#pragma unroll
                for (int i = 0; i < Q; ++i) x[i] += Gv * cf[i];
                if (c.gl) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) x[i] -= Hv * cf[Q + i];
                } else {
                    const int end = side ? Q - 1 : 0;
                    x[end] -= Hv * cf[Q + end];
                }
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) sR[G::vidx(dir, t, i)] = x[i];
        }
        __syncthreads();
    }
}

// Kt_a = kappa_K K_a + own facet terms of the two faces normal to axis a:
// low face  kF_L ( w_L (e0 d0^T + d0 e0^T) + gamma e0 e0^T ),
// high face kF_R (-w_R (ep dp^T + dp ep^T) + gamma ep ep^T ),
// kF = harmonic mean and w = 1/2 inside, kF = kappa_K and w = 1 on the boundary.
// With GLL nodes e0 / ep are the first / last unit vector, so the face terms
// live in row and column 0 and q-1 only.
template <int DIM, int Q, typename T>
__device__ __forceinline__ void build_block_1d(const DGConst<T> &c, const T *sT, bool active, int t, const T *myK,
                                               int mask, T *myKT) {
    using G = Geo<DIM, Q, T>;
    if (!active) return;
    const T *K = sT, *d0 = sT + DIM * Q * Q, *dp = d0 + DIM * Q;
    const T kK = myK[G::NFACE];
    if (c.gl) {                               // dense end values: every entry has face terms
        for (int e = t; e < DIM * Q * Q; e += G::NF) {
            const int a = e / (Q * Q), i = (e / Q) % Q, j = e % Q;
            const bool inL = mask & (1 << (2 * a)), inR = mask & (1 << (2 * a + 1));
            const T kL = inL ? myK[2 * a] : kK, wL = inL ? T(0.5) : T(1);
            const T kR = inR ? myK[2 * a + 1] : kK, wR = inR ? T(0.5) : T(1);
            const T e0i = c.v0[i], e0j = c.v0[j], epi = c.vp[i], epj = c.vp[j];
            T v = kK * K[e];
            v += kL * (wL * (e0i * d0[a * Q + j] + d0[a * Q + i] * e0j) + c.gamma[a] * e0i * e0j);
            v += kR * (-wR * (epi * dp[a * Q + j] + dp[a * Q + i] * epj) + c.gamma[a] * epi * epj);
            myKT[e] = v;
        }
        return;
    }
    for (int e = t; e < DIM * Q * Q; e += G::NF) {
        const int a = e / (Q * Q), i = (e / Q) % Q, j = e % Q;
        T v = kK * K[e];
        if (i == 0 || j == 0) {               // low-face terms live in row / column 0
            const bool in = mask & (1 << (2 * a));
            const T kL = in ? myK[2 * a] : kK;
            const T w = in ? T(0.5) : T(1);
            if (i == 0 && j == 0)
                v += kL * (T(2) * w * d0[a * Q] + c.gamma[a]);
            else
                v += kL * w * d0[a * Q + (i == 0 ? j : i)];
        }
        if (i == Q - 1 || j == Q - 1) {       // high-face terms live in row / column q-1
            const bool in = mask & (1 << (2 * a + 1));
            const T kR = in ? myK[2 * a + 1] : kK;
            const T w = in ? T(0.5) : T(1);
            if (i == Q - 1 && j == Q - 1)
                v += kR * (c.gamma[a] - T(2) * w * dp[a * Q + Q - 1]);
            else
                v -= kR * w * dp[a * Q + (i == Q - 1 ? j : i)];
        }
        myKT[e] = v;
    }
}

// R -= A_KK U with A_KK = sum_a Kt_a (x) M (x) M by sum factorisation:
// 3D: a = M_z u, bb = Kt_z u; c = M_y a, e = Kt_y a + M_y bb; y = Kt_x c + M_x e.
// 2D: a = M_y u, bb = Kt_y u; y = Kt_x a + M_x bb. Contains barriers.
// myB may be myU: each thread reads its whole pencil of u before writing the
// same positions, and u is not read again.
template <int DIM, int Q, typename T>
__device__ __forceinline__ void subtract_block_apply(const DGConst<T> &c, bool active, int t, const T *myU, T *myR,
                                                     T *myA, T *myB, const T *myKT, const T *sMw, const T *sMu) {
    using G = Geo<DIM, Q, T>;
    constexpr int D = DIM - 1;   // first pass along the highest axis
    // the 1D masses in their rank-one form M x = w o x - mu (mu . x) (exact
    // for the GLL mass; mu = 0 for the diagonal GL mass): 3q operations per
    // pencil instead of q^2
    if (active) {
        T x[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) x[i] = myU[G::vidx(D, t, i)];
        T dz = T(0);
#pragma unroll
        for (int m = 0; m < Q; ++m) dz += sMu[D * Q + m] * x[m];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T sb = T(0);
#pragma unroll
            for (int m = 0; m < Q; ++m) sb += myKT[D * Q * Q + i * Q + m] * x[m];
            myA[G::vidx(D, t, i)] = sMw[D * Q + i] * x[i] - sMu[D * Q + i] * dz;
            myB[G::vidx(D, t, i)] = sb;
        }
    }
    __syncthreads();
    if (DIM == 3) {
        if (active) {
            T xa[Q], xb[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                xa[i] = myA[G::vidx(1, t, i)];
                xb[i] = myB[G::vidx(1, t, i)];
            }
            T da = T(0), db = T(0);
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                da += sMu[Q + m] * xa[m];
                db += sMu[Q + m] * xb[m];
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T se = sMw[Q + i] * xb[i] - sMu[Q + i] * db;
#pragma unroll
                for (int m = 0; m < Q; ++m) se += myKT[1 * Q * Q + i * Q + m] * xa[m];
                myA[G::vidx(1, t, i)] = sMw[Q + i] * xa[i] - sMu[Q + i] * da;
                myB[G::vidx(1, t, i)] = se;
            }
        }
        __syncthreads();
    }
    if (active) {
        T xa[Q], xb[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            xa[i] = myA[G::vidx(0, t, i)];
            xb[i] = myB[G::vidx(0, t, i)];
        }
        T db = T(0);
#pragma unroll
        for (int m = 0; m < Q; ++m) db += sMu[m] * xb[m];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T s = sMw[i] * xb[i] - sMu[i] * db;
#pragma unroll
            for (int m = 0; m < Q; ++m) s += myKT[i * Q + m] * xa[m];
            myR[G::vidx(0, t, i)] -= s;
        }
    }
    __syncthreads();
}

// Value and +axis derivative of a pencil at both ends (Sec. 4.1 projection onto
// the facet spaces), written to the trace array.
template <int DIM, int Q, typename T>
__device__ __forceinline__ void write_pencil_traces(const DGConst<T> &c, int dir, int t, const T *x,
                                                    T *__restrict__ trc) {
    using G = Geo<DIM, Q, T>;
    T dlo = T(0), dhi = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        dlo += c.d0[dir][i] * x[i];
        dhi += c.dp[dir][i] * x[i];
    }
    T vlo = x[0], vhi = x[Q - 1];
    if (c.gl) {                               // GL nodes: the end values are dense dot products
        vlo = T(0);
        vhi = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            vlo += c.v0[i] * x[i];
            vhi += c.vp[i] * x[i];
        }
    }
    T *lo = trc + (2 * dir) * G::FS;
    T *hi = trc + (2 * dir + 1) * G::FS;
    lo[t] = vlo;
    lo[G::NF + t] = dlo;
    hi[t] = vhi;
    hi[G::NF + t] = dhi;
}

// ---------------------------------------------------------------------------
// Warm-up projection (Alg. 4 preamble), optionally preceded by u += P e
// (the p-prolongation fused into the projection, Sec. 5.1 "Prolongation").
// ---------------------------------------------------------------------------
template <int DIM, int Q, typename T>
__device__ __forceinline__ void k_project_body(const DGConst<T> &c, int64_t cell0, int cpb, T *__restrict__ u, const T *__restrict__ e0, T *__restrict__ tr) {
    using G = Geo<DIM, Q, T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sU = reinterpret_cast<T *>(smem_raw);
    T *sE = sU + cpb * G::NL;
    const int lc = threadIdx.x / G::NF, t = threadIdx.x - lc * G::NF;
    const int ncl = (int)min((int64_t)cpb, c.ncell - cell0);
    const bool active = lc < ncl;
    const int64_t cell = cell0 + lc;
    int ci[3] = {0, 0, 0};
    if (active) cell_coords<DIM>(cell, c.n, ci);
    block_copy(sU, u + cell0 * G::NL, (int64_t)ncl * G::NL);
    if (e0 != nullptr && active) {
        for (int k = t; k < G::NC; k += G::NF) {
            bool interior = true;
            int64_t vid = 0, stride = 1;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const int v = ci[a] + ((k >> a) & 1);
                interior = interior && v >= 1 && v <= c.n[a] - 1;
                vid += (int64_t)(v - 1) * stride;
                stride *= (c.n[a] - 1);
            }
            sE[lc * G::NC + k] = interior ? e0[vid] : T(0);
        }
    }
    __syncthreads();
    T *trc = tr + cell * G::TR;
    // pass along x: prolongation and x-face traces
    if (active) {
        T x[Q];
        T *pu = sU + lc * G::NL;
#pragma unroll
        for (int i = 0; i < Q; ++i) x[i] = pu[G::vidx(0, t, i)];
        if (e0 != nullptr) {
            const T *e = sE + lc * G::NC;
            T A0, A1;
            if (DIM == 2) {
                A0 = e[0] * c.hat[0][t] + e[2] * c.hat[1][t];
                A1 = e[1] * c.hat[0][t] + e[3] * c.hat[1][t];
            } else {
                const int a = t % Q, b = t / Q;
                const T w00 = c.hat[0][a] * c.hat[0][b], w10 = c.hat[1][a] * c.hat[0][b];
                const T w01 = c.hat[0][a] * c.hat[1][b], w11 = c.hat[1][a] * c.hat[1][b];
                A0 = e[0] * w00 + e[2] * w10 + e[4] * w01 + e[6] * w11;
                A1 = e[1] * w00 + e[3] * w10 + e[5] * w01 + e[7] * w11;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) x[i] += A0 * c.hat[0][i] + A1 * c.hat[1][i];
#pragma unroll
            for (int i = 0; i < Q; ++i) pu[G::vidx(0, t, i)] = x[i];
        }
        write_pencil_traces<DIM, Q, T>(c, 0, t, x, trc);
    }
    if (e0 != nullptr) __syncthreads();
    if (active) {
#pragma unroll
        for (int dir = 1; dir < DIM; ++dir) {
            T x[Q];
            const T *pu = sU + lc * G::NL;
#pragma unroll
            for (int i = 0; i < Q; ++i) x[i] = pu[G::vidx(dir, t, i)];
            write_pencil_traces<DIM, Q, T>(c, dir, t, x, trc);
        }
    }
    if (e0 != nullptr) {
        __syncthreads();
        block_copy(u + cell0 * G::NL, sU, (int64_t)ncl * G::NL);
    }
}

template <int DIM, int Q, typename T>
__global__ void __launch_bounds__(256) k_project(DGConst<T> c, int cpb, T *__restrict__ u, const T *__restrict__ e0, T *__restrict__ tr) {
    k_project_body<DIM, Q, T>(c, (int64_t)blockIdx.x * cpb, cpb, u, e0, tr);
}

// ---------------------------------------------------------------------------
// Single-touch block-Jacobi smoothing step (Alg. 4 fused loop body, Technique 5):
//   u_K <- u_K + omega B_K^{-1} (b - A u)_K,   B_K = A_KK (exact) or the block of
//   an interior cell (Technique 4).
// With the exact block the update is evaluated as
//   u_K <- (1 - omega) u_K + omega A_KK^{-1} (b_K - N_K u_nb),
// where N_K u_nb are the facet terms that involve the neighbours' stored
// projections (A u = A_KK u_K + N_K u_nb, so both forms are the same update
// and the volume operator is never applied). With the interior-only block the
// full residual b - N_K u_nb - A_KK u_K is formed first (c.exact == 0).
// B^{-1} by fast diagonalisation: B = sum over axes of Kt_a (x) M (x) M with
// Kt_a S_a = M S_a Lambda_a, S_a^T M S_a = I, so
// B^{-1} = (S_x (x) S_y (x) S_z) (Lambda_x + Lambda_y + Lambda_z)^{-1} (...)^T.
// Reads the neighbours' traces from tr_in and writes the cell's new traces to
// tr_out (ping-pong: every cell reads projections of the same iterate).
// ---------------------------------------------------------------------------
template <int DIM, int Q, typename T>
__device__ __forceinline__ void k_smooth_body(const DGConst<T> &c, int64_t cell0, int cpb, int exact, T *__restrict__ u, const T *__restrict__ b, const T *__restrict__ kappa, const T *__restrict__ fd, const T *__restrict__ linv, const T *__restrict__ tr_in, T *__restrict__ tr_out) {
    using G = Geo<DIM, Q, T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sFD = reinterpret_cast<T *>(smem_raw);   // [cpb][DIM][FDSP], 16-byte aligned blocks
    T *sU = sFD + cpb * DIM * G::FDSP;
    T *sR = sU + cpb * G::NL;
    T *sF = sR + cpb * G::NL;
    T *sK = sF + cpb * G::NFACE * 2 * G::NF;   // [cpb][NFACE + 1]
    T *sDot = sK + cpb * (G::NFACE + 1);       // [cpb][facet-mass dot products]
    T *sC = sDot + cpb * G::NDOT;              // [cpb][lifting coefficients]
    T *sA = sC + cpb * G::NLC;                 // inexact block only: [cpb][NL] x 2, [cpb][DIM*Q*Q]
    T *sB = sA + cpb * G::NL;
    T *sKT = sB + cpb * G::NL;
    const int lc = threadIdx.x / G::NF, t = threadIdx.x - lc * G::NF;
    const int ncl = (int)min((int64_t)cpb, c.ncell - cell0);
    const bool active = lc < ncl;
    const int64_t cell = cell0 + lc;
    int ci[3] = {0, 0, 0};
    __shared__ T sMw[DIM * Q], sMu[DIM * Q];
    __shared__ T sT[DIM * Q * Q + 2 * DIM * Q];
    stage_mass_rank1<DIM, Q, T>(c, sMw, sMu);
    if (!exact) stage_block_tables<DIM, Q, T>(c, sT);
    block_copy(sU, u + cell0 * G::NL, (int64_t)ncl * G::NL);
    block_copy(sR, b + cell0 * G::NL, (int64_t)ncl * G::NL);
    for (int64_t i = threadIdx.x; i < (int64_t)ncl * DIM * G::FDS; i += blockDim.x)
        sFD[(i / G::FDS) * G::FDSP + i % G::FDS] = fd[cell0 * DIM * G::FDS + i];
    T *myF = sF + lc * G::NFACE * 2 * G::NF;
    T *myK = sK + lc * (G::NFACE + 1);
    if (active) {
        cell_coords<DIM>(cell, c.n, ci);
        load_neighbour_traces<DIM, Q, T>(c, cell, ci, t, tr_in, kappa, myF, myK, myK + G::NFACE);
    }
    __syncthreads();
    T *myR = sR + lc * G::NL;
    T *myU = sU + lc * G::NL;
    const int mask = active ? interior_mask<DIM>(ci, c.n) : 0;
    if (!exact) build_block_1d<DIM, Q, T>(c, sT, active, t, myK, mask, sKT + lc * DIM * Q * Q);
    lift_coefficients<DIM, Q, T>(c, active, t, myK, mask, sC + lc * G::NLC);   // read after facet_mass's barriers
    facet_mass<DIM, Q, T>(sMw, sMu, active, t, myF, sDot + lc * G::NDOT, mask);
    lift_neighbours<DIM, Q, T>(c, active, t, myR, myF, sC + lc * G::NLC, mask);
    if (!exact)
        subtract_block_apply<DIM, Q, T>(c, active, t, myU, myR, sA + lc * G::NL, sB + lc * G::NL,
                                        sKT + lc * DIM * Q * Q, sMw, sMu);
    const T *myS = sFD + lc * DIM * G::FDSP;     // S_a at a*FDSP, lambda_a at a*FDSP + Q*Q
    // S^T along the axes 0..DIM-2
#pragma unroll
    for (int dir = 0; dir < DIM - 1; ++dir) {
        if (active) {
            T x[Q], y[Q];
            __align__(16) T S[G::QQV * G::VEC];
            load_factor<DIM, Q, T>(myS + dir * G::FDSP, S);
#pragma unroll
            for (int i = 0; i < Q; ++i) x[i] = myR[G::vidx(dir, t, i)];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T s = T(0);
#pragma unroll
                for (int m = 0; m < Q; ++m) s += S[m * Q + i] * x[m];
                y[i] = s;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) myR[G::vidx(dir, t, i)] = y[i];
        }
        __syncthreads();
    }
    // last axis: S^T, divide by the eigenvalue sums, S
    {
        constexpr int D = DIM - 1;
        if (active) {
            T x[Q], y[Q];
            __align__(16) T S[G::QQV * G::VEC];
            load_factor<DIM, Q, T>(myS + D * G::FDSP, S);
            const T *lam = myS + D * G::FDSP + Q * Q;
            T lt;
            if (DIM == 2) {
                lt = myS[0 * G::FDSP + Q * Q + t];
            } else {
                lt = myS[0 * G::FDSP + Q * Q + (t % Q)] + myS[1 * G::FDSP + Q * Q + (t / Q)];
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) x[i] = myR[G::vidx(D, t, i)];
            // 1 / (lambda_x + lambda_y + lambda_z): from the per-node table when
            // one is given (saves a division per node; the table holds omega /
            // the sum, so the damping is then already applied), else divided here
            const T *li = linv ? linv + cell * G::NL : nullptr;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T s = T(0);
#pragma unroll
                for (int m = 0; m < Q; ++m) s += S[m * Q + i] * x[m];
                y[i] = li ? s * li[G::vidx(D, t, i)] : s / (lt + lam[i]);
            }
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) s += S[m * Q + i] * y[i];
                x[m] = s;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) myR[G::vidx(D, t, i)] = x[i];
        }
        __syncthreads();
    }
#pragma unroll
    for (int dir = DIM - 2; dir >= 1; --dir) {
        if (active) {
            T x[Q], y[Q];
            __align__(16) T S[G::QQV * G::VEC];
            load_factor<DIM, Q, T>(myS + dir * G::FDSP, S);
#pragma unroll
            for (int i = 0; i < Q; ++i) x[i] = myR[G::vidx(dir, t, i)];
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) s += S[m * Q + i] * x[i];
                y[m] = s;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) myR[G::vidx(dir, t, i)] = y[i];
        }
        __syncthreads();
    }
    // axis 0: S, damped update, x-face traces
    T *trc = tr_out + cell * G::TR;
    if (active) {
        T x[Q], un[Q];
        __align__(16) T S[G::QQV * G::VEC];
        load_factor<DIM, Q, T>(myS, S);
#pragma unroll
        for (int i = 0; i < Q; ++i) x[i] = myR[G::vidx(0, t, i)];
        const T om = c.omega;
        const T keep = exact ? T(1) - om : T(1);
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            T s = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) s += S[m * Q + i] * x[i];
            un[m] = linv ? keep * myU[G::vidx(0, t, m)] + s : keep * myU[G::vidx(0, t, m)] + om * s;
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) myU[G::vidx(0, t, i)] = un[i];
        write_pencil_traces<DIM, Q, T>(c, 0, t, un, trc);
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int dir = 1; dir < DIM; ++dir) {
            T x[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) x[i] = myU[G::vidx(dir, t, i)];
            write_pencil_traces<DIM, Q, T>(c, dir, t, x, trc);
        }
    }
    block_copy(u + cell0 * G::NL, sU, (int64_t)ncl * G::NL);
}

template <int DIM, int Q, typename T>
__global__ void __launch_bounds__(256) k_smooth(DGConst<T> c, int cpb, int exact, T *__restrict__ u, const T *__restrict__ b, const T *__restrict__ kappa, const T *__restrict__ fd, const T *__restrict__ linv, const T *__restrict__ tr_in, T *__restrict__ tr_out) {
    k_smooth_body<DIM, Q, T>(c, (int64_t)blockIdx.x * cpb, cpb, exact, u, b, kappa, fd, linv, tr_in, tr_out);
}

// ---------------------------------------------------------------------------
// Residual r = b - A u (Alg. 2 stage 3 / Alg. 6 residual traversal) from u and
// the stored projections of u, with A u = A_KK u_K + N_K u_nb, and the optional
// fused p-restriction: per cell and corner, sum_i hat_corner(x_i) r_i, gathered
// per vertex afterwards in a fixed order.
// ---------------------------------------------------------------------------
template <int DIM, int Q, typename T>
__device__ __forceinline__ void k_residual_body(const DGConst<T> &c, int64_t cell0, int cpb, int mode, const T *__restrict__ u, const T *__restrict__ b, const T *__restrict__ kappa, const T *__restrict__ tr, T *__restrict__ rout, T *__restrict__ corners) {
    using G = Geo<DIM, Q, T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // u is read once, by the first pass of the A_KK apply, which overwrites it
    // with one of its two intermediate tensors (sA holds the other)
    T *sU = reinterpret_cast<T *>(smem_raw);
    T *sR = sU + cpb * G::NL;
    T *sA = sR + cpb * G::NL;
    T *sF = sA + cpb * G::NL;
    T *sKT = sF + cpb * G::NFACE * 2 * G::NF;   // [cpb][DIM][Q*Q]
    T *sK = sKT + cpb * DIM * Q * Q;            // [cpb][NFACE + 1]
    T *sDot = sK + cpb * (G::NFACE + 1);        // [cpb][facet-mass dot products]
    T *sC = sDot + cpb * G::NDOT;               // [cpb][lifting coefficients]
    const int lc = threadIdx.x / G::NF, t = threadIdx.x - lc * G::NF;
    const int ncl = (int)min((int64_t)cpb, c.ncell - cell0);
    const bool active = lc < ncl;
    const int64_t cell = cell0 + lc;
    int ci[3] = {0, 0, 0};
    __shared__ T sMw[DIM * Q], sMu[DIM * Q];
    __shared__ T sT[DIM * Q * Q + 2 * DIM * Q];
    stage_mass_rank1<DIM, Q, T>(c, sMw, sMu);
    stage_block_tables<DIM, Q, T>(c, sT);
    block_copy(sU, u + cell0 * G::NL, (int64_t)ncl * G::NL);
    if (mode & RES_HAS_B) {
        block_copy(sR, b + cell0 * G::NL, (int64_t)ncl * G::NL);
    } else {
        for (int64_t i = threadIdx.x; i < (int64_t)ncl * G::NL; i += blockDim.x) sR[i] = T(0);
    }
    T *myF = sF + lc * G::NFACE * 2 * G::NF;
    T *myK = sK + lc * (G::NFACE + 1);
    if (active) {
        cell_coords<DIM>(cell, c.n, ci);
        load_neighbour_traces<DIM, Q, T>(c, cell, ci, t, tr, kappa, myF, myK, myK + G::NFACE);
    }
    __syncthreads();
    T *myKT = sKT + lc * DIM * Q * Q;
    const int mask = active ? interior_mask<DIM>(ci, c.n) : 0;
    build_block_1d<DIM, Q, T>(c, sT, active, t, myK, mask, myKT);
    lift_coefficients<DIM, Q, T>(c, active, t, myK, mask, sC + lc * G::NLC);   // read after facet_mass's barriers
    facet_mass<DIM, Q, T>(sMw, sMu, active, t, myF, sDot + lc * G::NDOT, mask);   // contains barriers
    T *myR = sR + lc * G::NL;
    T *myU = sU + lc * G::NL;
    lift_neighbours<DIM, Q, T>(c, active, t, myR, myF, sC + lc * G::NLC, mask);
    subtract_block_apply<DIM, Q, T>(c, active, t, myU, myR, sA + lc * G::NL, myU, myKT, sMw, sMu);
    T rr[Q];
    if (active) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            rr[i] = myR[G::vidx(0, t, i)];
            if (mode & RES_NEGATE) rr[i] = -rr[i];
        }
        if (mode & RES_WRITE_R) {
            T *dst = rout + cell * G::NL;
#pragma unroll
            for (int i = 0; i < Q; ++i) dst[G::vidx(0, t, i)] = rr[i];
        }
    }
    if (mode & RES_CORNERS) {
        // partial sums over x of hat_cx(x_i) r_i, then over the tangential axes
        T *px = sF;                     // reuse: [cpb][2][NF]
        if (active) {
            T p0 = T(0), p1 = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                p0 += c.hat[0][i] * rr[i];
                p1 += c.hat[1][i] * rr[i];
            }
            px[(lc * 2 + 0) * G::NF + t] = p0;
            px[(lc * 2 + 1) * G::NF + t] = p1;
        }
        __syncthreads();
        if (active) {
            for (int k = t; k < G::NC; k += G::NF) {
                const int cx = k & 1, cy = (k >> 1) & 1, cz = (k >> 2) & 1;
                const T *src = px + (lc * 2 + cx) * G::NF;
                T s = T(0);
                if (DIM == 2) {
                    for (int a = 0; a < Q; ++a) s += c.hat[cy][a] * src[a];
                } else {
                    for (int bb = 0; bb < Q; ++bb) {
                        T sa = T(0);
                        for (int a = 0; a < Q; ++a) sa += c.hat[cy][a] * src[a + Q * bb];
                        s += c.hat[cz][bb] * sa;
                    }
                }
                corners[cell * G::NC + k] = s;
            }
        }
    }
}

template <int DIM, int Q, typename T>
__global__ void __launch_bounds__(256) k_residual(DGConst<T> c, int cpb, int mode, const T *__restrict__ u, const T *__restrict__ b, const T *__restrict__ kappa, const T *__restrict__ tr, T *__restrict__ rout, T *__restrict__ corners) {
    k_residual_body<DIM, Q, T>(c, (int64_t)blockIdx.x * cpb, cpb, mode, u, b, kappa, tr, rout, corners);
}


}  // namespace dgmg

#include "smooth_cells.cuh"
#include "dg_transfer.cuh"

namespace dgmg {

// ---------------------------------------------------------------------------
// Batched launches: work item k serves the cells [cell0, cell0 + tile) of
// instance map[k].inst; its CTA copies that instance's descriptor (constants
// and array pointers) into shared memory and runs the same body as the
// single-instance kernel on the instance's slice of the group vectors. One
// persistent launch per stage: as many CTAs as stay resident, each striding
// through the work items.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void load_batch_desc(const BatchDG<T> *__restrict__ src, BatchDG<T> *dst) {
    static_assert(sizeof(BatchDG<T>) % 8 == 0, "descriptor copied in 8-byte words");
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(BatchDG<T>) / 8); i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// Persistent: the CTAs stride through the nblocks work items of the map; a
// barrier ends every thread's use of the descriptor and of the staging memory
// before the next item is loaded.
template <int DIM, int Q, typename T>
__global__ void __launch_bounds__(256) k_project_batch(const BatchDG<T> *__restrict__ D,
                                                        const BlockMap *__restrict__ map, int nblocks, int cpb, T *u,
                                                        int with_e0) {
    using G = Geo<DIM, Q, T>;
    __shared__ __align__(16) BatchDG<T> sd;
    for (int k = blockIdx.x; k < nblocks; k += gridDim.x) {
        if (k != (int)blockIdx.x) __syncthreads();
        const BlockMap m = map[k];
        load_batch_desc(D + m.inst, &sd);
        k_project_body<DIM, Q, T>(sd.c, m.cell0, cpb, u + sd.off * G::NL, with_e0 ? sd.e0 : nullptr, sd.tr[0]);
    }
}

template <int DIM, int Q, typename T>
__global__ void __launch_bounds__(256) k_smooth_batch(const BatchDG<T> *__restrict__ D,
                                                       const BlockMap *__restrict__ map, int nblocks, int cpb,
                                                       int exact, T *u, const T *b, int cur) {
    using G = Geo<DIM, Q, T>;
    __shared__ __align__(16) BatchDG<T> sd;
    for (int k = blockIdx.x; k < nblocks; k += gridDim.x) {
        if (k != (int)blockIdx.x) __syncthreads();
        const BlockMap m = map[k];
        load_batch_desc(D + m.inst, &sd);
        k_smooth_body<DIM, Q, T>(sd.c, m.cell0, cpb, exact, u + sd.off * G::NL, b + sd.off * G::NL, sd.kappa, sd.fd,
                                 sd.linv, sd.tr[cur], sd.tr[cur ^ 1]);
    }
}

template <typename T, int Q>
__global__ void __launch_bounds__(32) k_smooth_cells_batch(const BatchDG<T> *__restrict__ D,
                                                            const BlockMap *__restrict__ map, int nblocks, T *u,
                                                            const T *b, int cur) {
    constexpr int NL = Q * Q * Q;
    __shared__ __align__(16) BatchDG<T> sd;
    for (int k = blockIdx.x; k < nblocks; k += gridDim.x) {
        if (k != (int)blockIdx.x) __syncthreads();
        const BlockMap m = map[k];
        load_batch_desc(D + m.inst, &sd);
        smooth_cells_body<T, Q>(sd.c, m.cell0, u + sd.off * NL, b + sd.off * NL, sd.kappa, sd.fd, sd.linv,
                                sd.tr[cur], sd.tr[cur ^ 1], k != (int)blockIdx.x);
    }
}

template <typename T, int Q>
__global__ void __launch_bounds__(32) k_residual_cells_batch(const BatchDG<T> *__restrict__ D,
                                                              const BlockMap *__restrict__ map, int nblocks, int mode,
                                                              const T *u, const T *b, T *r, int cur) {
    constexpr int NL = Q * Q * Q;
    __shared__ __align__(16) BatchDG<T> sd;
    for (int k = blockIdx.x; k < nblocks; k += gridDim.x) {
        if (k != (int)blockIdx.x) __syncthreads();
        const BlockMap m = map[k];
        load_batch_desc(D + m.inst, &sd);
        residual_cells_body<T, Q>(sd.c, m.cell0, mode, u + sd.off * NL, b ? b + sd.off * NL : nullptr, sd.kappa,
                                  sd.fdr, sd.tr[cur], r ? r + sd.off * NL : nullptr, sd.corners, k != (int)blockIdx.x);
    }
}

template <typename T, int Q>
__global__ void __launch_bounds__(32) k_residual_cells_batch_direct(const BatchDG<T> *__restrict__ D,
                                                                     const BlockMap *__restrict__ map, int nblocks,
                                                                     int mode, const T *u, T *r, int cur) {
    constexpr int NL = Q * Q * Q;
    __shared__ __align__(16) BatchDG<T> sd;
    for (int k = blockIdx.x; k < nblocks; k += gridDim.x) {
        if (k != (int)blockIdx.x) __syncthreads();
        const BlockMap m = map[k];
        load_batch_desc(D + m.inst, &sd);
        residual_cells_body<T, Q, true>(sd.c, m.cell0, mode, u + sd.off * NL, nullptr, sd.kappa, nullptr, sd.tr[cur],
                                        r ? r + sd.off * NL : nullptr, nullptr, k != (int)blockIdx.x);
    }
}

template <int DIM, int Q, typename T>
__global__ void __launch_bounds__(256) k_residual_batch(const BatchDG<T> *__restrict__ D,
                                                         const BlockMap *__restrict__ map, int nblocks, int cpb,
                                                         int mode, const T *u, const T *b, T *r, int cur) {
    using G = Geo<DIM, Q, T>;
    __shared__ __align__(16) BatchDG<T> sd;
    for (int k = blockIdx.x; k < nblocks; k += gridDim.x) {
        if (k != (int)blockIdx.x) __syncthreads();
        const BlockMap m = map[k];
        load_batch_desc(D + m.inst, &sd);
        k_residual_body<DIM, Q, T>(sd.c, m.cell0, cpb, mode, u + sd.off * G::NL, b ? b + sd.off * G::NL : nullptr,
                                   sd.kappa, sd.tr[cur], r ? r + sd.off * G::NL : nullptr, sd.corners);
    }
}

// tr[0] of instance blockIdx.x := 0 (projections of a zero iterate)
template <int DIM, int Q, typename T>
__global__ void k_zero_traces_batch(const BatchDG<T> *__restrict__ D) {
    using G = Geo<DIM, Q, T>;
    const BatchDG<T> &d = D[blockIdx.x];
    const int64_t n = d.c.ncell * G::TR;
    T *tr = d.tr[0];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) tr[i] = T(0);
}

// Shared-memory bytes per CTA of each kernel.
template <int DIM, int Q, typename T>
constexpr size_t smem_project(int cpb) {
    return (size_t)cpb * (Geo<DIM, Q, T>::NL + Geo<DIM, Q, T>::NC) * sizeof(T);
}
template <int DIM, int Q, typename T>
constexpr size_t smem_smooth(int cpb, bool exact) {
    using G = Geo<DIM, Q, T>;
    return (size_t)cpb *
           (DIM * G::FDSP + 2 * G::NL + G::NFACE * 2 * G::NF + G::NFACE + 1 + G::NDOT + G::NLC +
            (exact ? 0 : 2 * G::NL + DIM * Q * Q)) *
           sizeof(T);
}
template <int DIM, int Q, typename T>
constexpr size_t smem_residual(int cpb) {
    using G = Geo<DIM, Q, T>;
    return (size_t)cpb * (3 * G::NL + G::NFACE * 2 * G::NF + DIM * Q * Q + G::NFACE + 1 + G::NDOT + G::NLC) *
           sizeof(T);
}

template <int DIM, int Q, typename T>
struct DGLaunch {
    using G = Geo<DIM, Q, T>;
    // cells per CTA when the caller leaves the choice (cpb <= 0): as many as fit
    // 256 threads (q = 5: 10 cells, 250 threads), so the last warp is nearly
    // full (FP64 work of idle lanes is lost)
    static int default_cpb() { return std::max(1, 256 / G::NF); }
    static cudaError_t project(const DGConst<T> &c, int cpb, T *u, const T *e0, T *tr, cudaStream_t s) {
        if constexpr (CELLS_OK) if (c.ncell < (int64_t(1) << 31)) {   // 32-bit cell indices
            // bulk copies want a 16-byte aligned u; the trace pieces 8- (FP32) or 16-byte (FP64) aligned traces
            const uintptr_t tra = 15;   // bulk copies of whole (padded) faces
            if (cpb <= 0 && !c.gl && (reinterpret_cast<uintptr_t>(u) & 15) == 0 &&
                (reinterpret_cast<uintptr_t>(tr) & tra) == 0) {
                using CG = CellGeo<T, Q>;
                static bool attr_c = false;
                if (!attr_c) {
                    cudaFuncSetAttribute(k_project_cells<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CG::BYTES);
                    attr_c = true;
                }
                const int64_t grid = (c.ncell + CG::W - 1) / CG::W;
                if (grid == 0) return cudaSuccess;
                count_launches(1);
                k_project_cells<T, Q><<<(unsigned)grid, CG::W, CG::BYTES, s>>>(c, u, e0, tr);
                return cudaGetLastError();
            }
        }
        if (cpb <= 0) cpb = default_cpb();
        const size_t sm = smem_project<DIM, Q, T>(cpb);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_project<DIM, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr = true;
        }
        const int64_t grid = (c.ncell + cpb - 1) / cpb;
        if (grid == 0) return cudaSuccess;
        count_launches(1);
        k_project<DIM, Q, T><<<(unsigned)grid, cpb * G::NF, sm, s>>>(c, cpb, u, e0, tr);
        return cudaGetLastError();
    }
    static cudaError_t smooth(const DGConst<T> &c, int cpb, int exact, T *u, const T *b, const T *kappa,
                              const T *fd, const T *linv, const T *tri, T *tro, cudaStream_t s) {
        if constexpr (CELLS_OK) if (c.ncell < (int64_t(1) << 31)) {   // 32-bit cell indices
            // bulk copies want 16-byte aligned vectors, factors and table; the face
            // pieces 8- (FP32) or 16-byte (FP64) aligned traces
            const uintptr_t tra = 15;   // bulk copies of whole (padded) faces
            const bool aligned = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(b) |
                                   reinterpret_cast<uintptr_t>(fd) | reinterpret_cast<uintptr_t>(linv)) & 15) == 0 &&
                                 ((reinterpret_cast<uintptr_t>(tri) | reinterpret_cast<uintptr_t>(tro)) & tra) == 0;
            if (cpb <= 0 && exact && aligned && !c.gl) return smooth_cells(c, u, b, kappa, fd, linv, tri, tro, s);
        }
        if (cpb <= 0) cpb = default_cpb();
        const size_t sm = smem_smooth<DIM, Q, T>(cpb, exact != 0);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_smooth<DIM, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr = true;
        }
        const int64_t grid = (c.ncell + cpb - 1) / cpb;
        if (grid == 0) return cudaSuccess;
        count_launches(1);
        k_smooth<DIM, Q, T><<<(unsigned)grid, cpb * G::NF, sm, s>>>(c, cpb, exact, u, b, kappa, fd, linv, tri, tro);
        return cudaGetLastError();
    }
    // 3D exact-block smoothing step with one thread per cell (k_smooth_cells):
    // FP32 q <= 5, FP64 q <= 4 (the cell must fit in the registers of a thread)
    static constexpr bool CELLS_OK = DIM == 3 && (std::is_same<T, float>::value ? Q <= 5 : Q <= 4);
    static cudaError_t smooth_cells(const DGConst<T> &c, T *u, const T *b, const T *kappa, const T *fd,
                                    const T *linv, const T *tri, T *tro, cudaStream_t s) {
        if constexpr (CELLS_OK) {
            using CG = CellGeo<T, Q>;
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_smooth_cells<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)CG::BYTES);
                attr = true;
            }
            const int64_t grid = (c.ncell + CG::W - 1) / CG::W;
            if (grid == 0) return cudaSuccess;
            count_launches(1);
            k_smooth_cells<T, Q><<<(unsigned)grid, CG::W, CG::BYTES, s>>>(c, u, b, kappa, fd, linv, tri, tro);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }
    static cudaError_t residual_cells(const DGConst<T> &c, int mode, const T *u, const T *b, const T *kappa,
                                      const T *fd, const T *tr, T *r, T *corners, cudaStream_t s) {
        if constexpr (CELLS_OK) {
            using CG = CellGeo<T, Q>;
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_residual_cells<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)CG::BYTES);
                attr = true;
            }
            const int64_t grid = (c.ncell + CG::W - 1) / CG::W;
            if (grid == 0) return cudaSuccess;
            count_launches(1);
            k_residual_cells<T, Q><<<(unsigned)grid, CG::W, CG::BYTES, s>>>(c, mode, u, b, kappa, fd, tr, r, corners);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }
    // the direct-form one-thread-per-cell residual (FP32: the CG operator)
    static cudaError_t residual_cells_direct(const DGConst<T> &c, int mode, const T *u, const T *b, const T *kappa,
                                             const T *tr, T *r, T *corners, cudaStream_t s) {
        if constexpr (CELLS_OK && sizeof(T) == 4) {
            using CG = CellGeo<T, Q>;
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_residual_cells_direct<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)CG::BYTES);
                attr = true;
            }
            const int64_t grid = (c.ncell + CG::W - 1) / CG::W;
            if (grid == 0) return cudaSuccess;
            count_launches(1);
            k_residual_cells_direct<T, Q><<<(unsigned)grid, CG::W, CG::BYTES, s>>>(c, mode, u, b, kappa, tr, r,
                                                                                   corners);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }
    // ---- batched forms (map: one entry per work item of cpb cells, 32 for the
    // one-thread-per-cell kernels; persistent grids)
    static cudaError_t project_batch(const BatchDG<T> *D, const BlockMap *map, int nblocks, int cpb, T *u,
                                     int with_e0, cudaStream_t s) {
        if (nblocks <= 0) return cudaSuccess;
        if (cpb <= 0) cpb = default_cpb();
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_project_batch<DIM, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            attr = true;
        }
        count_launches(1);
        const size_t smp = smem_project<DIM, Q, T>(cpb);
        k_project_batch<DIM, Q, T><<<persistent_grid((const void *)k_project_batch<DIM, Q, T>, cpb * G::NF, smp, nblocks),
                                     cpb * G::NF, smp, s>>>(D, map, nblocks, cpb, u, with_e0);
        return cudaGetLastError();
    }
    static cudaError_t smooth_batch(const BatchDG<T> *D, const BlockMap *map, int nblocks, int cpb, int exact, T *u,
                                    const T *b, int cur, cudaStream_t s) {
        if (nblocks <= 0) return cudaSuccess;
        if constexpr (CELLS_OK) {
            if (cpb <= 0 && exact) {
                using CG = CellGeo<T, Q>;
                static bool attr = false;
                if (!attr) {
                    cudaFuncSetAttribute(k_smooth_cells_batch<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CG::BYTES);
                    attr = true;
                }
                count_launches(1);
                k_smooth_cells_batch<T, Q><<<persistent_grid((const void *)k_smooth_cells_batch<T, Q>, CG::W, CG::BYTES,
                                                             nblocks),
                                             CG::W, CG::BYTES, s>>>(D, map, nblocks, u, b, cur);
                return cudaGetLastError();
            }
        }
        if (cpb <= 0) return cudaErrorInvalidValue;   // the map was built for 32-cell blocks
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_smooth_batch<DIM, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            attr = true;
        }
        count_launches(1);
        const size_t sms = smem_smooth<DIM, Q, T>(cpb, exact != 0);
        k_smooth_batch<DIM, Q, T><<<persistent_grid((const void *)k_smooth_batch<DIM, Q, T>, cpb * G::NF, sms, nblocks),
                                    cpb * G::NF, sms, s>>>(D, map, nblocks, cpb, exact, u, b, cur);
        return cudaGetLastError();
    }
    static cudaError_t residual_batch(const BatchDG<T> *D, const BlockMap *map, int nblocks, int cpb, int mode,
                                      const T *u, const T *b, T *r, int cur, cudaStream_t s) {
        if (nblocks <= 0) return cudaSuccess;
        if constexpr (CELLS_OK) {
            if constexpr (sizeof(T) == 4) {
                if (cpb <= 0 && (mode & RES_DIRECT)) {   // the FP32 CG operator: no b, no corners
                    using CG = CellGeo<T, Q>;
                    static bool attr = false;
                    if (!attr) {
                        cudaFuncSetAttribute(k_residual_cells_batch_direct<T, Q>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG::BYTES);
                        attr = true;
                    }
                    count_launches(1);
                    k_residual_cells_batch_direct<T, Q>
                        <<<persistent_grid((const void *)k_residual_cells_batch_direct<T, Q>, CG::W, CG::BYTES,
                                           nblocks),
                           CG::W, CG::BYTES, s>>>(D, map, nblocks, mode, u, r, cur);
                    return cudaGetLastError();
                }
            }
            if (cpb <= 0) {          // the map holds 32-cell blocks; every problem carries its factors
                using CG = CellGeo<T, Q>;
                static bool attr = false;
                if (!attr) {
                    cudaFuncSetAttribute(k_residual_cells_batch<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CG::BYTES);
                    attr = true;
                }
                count_launches(1);
                k_residual_cells_batch<T, Q><<<persistent_grid((const void *)k_residual_cells_batch<T, Q>, CG::W,
                                                               CG::BYTES, nblocks),
                                               CG::W, CG::BYTES, s>>>(D, map, nblocks, mode, u, b, r, cur);
                return cudaGetLastError();
            }
        }
        if (cpb <= 0) return cudaErrorInvalidValue;   // the map was built for 32-cell blocks
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_residual_batch<DIM, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 160 * 1024);
            attr = true;
        }
        count_launches(1);
        const size_t smr = smem_residual<DIM, Q, T>(cpb);
        k_residual_batch<DIM, Q, T><<<persistent_grid((const void *)k_residual_batch<DIM, Q, T>, cpb * G::NF, smr, nblocks),
                                      cpb * G::NF, smr, s>>>(D, map, nblocks, cpb, mode, u, b, r, cur);
        return cudaGetLastError();
    }
    static cudaError_t zero_traces_batch(const BatchDG<T> *D, int count, cudaStream_t s) {
        if (count <= 0) return cudaSuccess;
        count_launches(1);
        k_zero_traces_batch<DIM, Q, T><<<count, 256, 0, s>>>(D);
        return cudaGetLastError();
    }
    static cudaError_t residual(const DGConst<T> &c, int cpb, int mode, const T *u, const T *b, const T *kappa,
                                const T *tr, T *r, T *corners, const T *fd, cudaStream_t s) {
        if constexpr (CELLS_OK) if (c.ncell < (int64_t(1) << 31)) {   // 32-bit cell indices
            // bulk copies of u, b, the factors and r want 16-byte alignment; the
            // face pieces 8- (FP32) or 16-byte (FP64) aligned traces
            const uintptr_t tra = 15;   // bulk copies of whole (padded) faces
            const uintptr_t vec = reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(fd) |
                                  ((mode & RES_HAS_B) ? reinterpret_cast<uintptr_t>(b) : 0) |
                                  ((mode & RES_WRITE_R) ? reinterpret_cast<uintptr_t>(r) : 0);
            if (cpb <= 0 && fd && !c.gl && (vec & 15) == 0 && (reinterpret_cast<uintptr_t>(tr) & tra) == 0)
                return residual_cells(c, mode, u, b, kappa, fd, tr, r, corners, s);
            // without factors (the FP32 CG operator): A_KK u in the direct form
            if (sizeof(T) == 4 && cpb <= 0 && !fd && !c.gl && (vec & 15) == 0 &&
                (reinterpret_cast<uintptr_t>(tr) & tra) == 0)
                return residual_cells_direct(c, mode, u, b, kappa, tr, r, corners, s);
        }
        if (cpb <= 0) cpb = default_cpb();
        const size_t sm = smem_residual<DIM, Q, T>(cpb);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_residual<DIM, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr = true;
        }
        const int64_t grid = (c.ncell + cpb - 1) / cpb;
        if (grid == 0) return cudaSuccess;
        count_launches(1);
        k_residual<DIM, Q, T><<<(unsigned)grid, cpb * G::NF, sm, s>>>(c, cpb, mode, u, b, kappa, tr, r, corners);
        return cudaGetLastError();
    }
};

#define DGMG_DISPATCH(dim, q, CALL)                      \
    switch ((dim) * 16 + (q)) {                          \
        case 2 * 16 + 2: return DGLaunch<2, 2, T>::CALL; \
        case 2 * 16 + 3: return DGLaunch<2, 3, T>::CALL; \
        case 2 * 16 + 4: return DGLaunch<2, 4, T>::CALL; \
        case 2 * 16 + 5: return DGLaunch<2, 5, T>::CALL; \
        case 2 * 16 + 6: return DGLaunch<2, 6, T>::CALL; \
        case 2 * 16 + 7: return DGLaunch<2, 7, T>::CALL; \
        case 3 * 16 + 2: return DGLaunch<3, 2, T>::CALL; \
        case 3 * 16 + 3: return DGLaunch<3, 3, T>::CALL; \
        case 3 * 16 + 4: return DGLaunch<3, 4, T>::CALL; \
        case 3 * 16 + 5: return DGLaunch<3, 5, T>::CALL; \
        case 3 * 16 + 6: return DGLaunch<3, 6, T>::CALL; \
        case 3 * 16 + 7: return DGLaunch<3, 7, T>::CALL; \
        default: return cudaErrorInvalidValue;           \
    }

template <typename T>
cudaError_t launch_project_impl(int dim, int q, const DGConst<T> &c, int cpb, T *u, const T *e0, T *tr,
                                cudaStream_t s) {
    DGMG_DISPATCH(dim, q, project(c, cpb, u, e0, tr, s))
}
template <typename T>
cudaError_t launch_smooth_impl(int dim, int q, const DGConst<T> &c, int cpb, int exact, T *u, const T *b,
                               const T *kappa, const T *fd, const T *linv, const T *tri, T *tro, cudaStream_t s) {
    DGMG_DISPATCH(dim, q, smooth(c, cpb, exact, u, b, kappa, fd, linv, tri, tro, s))
}
template <typename T>
cudaError_t launch_residual_impl(int dim, int q, const DGConst<T> &c, int cpb, int mode, const T *u, const T *b,
                                 const T *kappa, const T *tr, T *r, T *corners, const T *fd, cudaStream_t s) {
    DGMG_DISPATCH(dim, q, residual(c, cpb, mode, u, b, kappa, tr, r, corners, fd, s))
}
template <typename T>
cudaError_t launch_project_batch_impl(int dim, int q, const BatchDG<T> *D, const BlockMap *map, int nblocks, int cpb,
                                      T *u, int with_e0, cudaStream_t s) {
    DGMG_DISPATCH(dim, q, project_batch(D, map, nblocks, cpb, u, with_e0, s))
}
template <typename T>
cudaError_t launch_smooth_batch_impl(int dim, int q, const BatchDG<T> *D, const BlockMap *map, int nblocks, int cpb,
                                     int exact, T *u, const T *b, int cur, cudaStream_t s) {
    DGMG_DISPATCH(dim, q, smooth_batch(D, map, nblocks, cpb, exact, u, b, cur, s))
}
template <typename T>
cudaError_t launch_residual_batch_impl(int dim, int q, const BatchDG<T> *D, const BlockMap *map, int nblocks,
                                       int cpb, int mode, const T *u, const T *b, T *r, int cur, cudaStream_t s) {
    DGMG_DISPATCH(dim, q, residual_batch(D, map, nblocks, cpb, mode, u, b, r, cur, s))
}
template <typename T>
cudaError_t launch_zero_traces_batch_impl(int dim, int q, const BatchDG<T> *D, int count, cudaStream_t s) {
    DGMG_DISPATCH(dim, q, zero_traces_batch(D, count, s))
}

}  // namespace dgmg
