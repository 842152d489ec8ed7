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
    if (v <= 0x7fffffff) {   // 32-bit division where it suffices
        const unsigned u = (unsigned)v, m0 = (unsigned)m[0], r = u / m0;
        c[0] = (int)(u - r * m0);
        if (DIM == 3) {
            const unsigned m1 = (unsigned)m[1], z = r / m1;
            c[1] = (int)(r - z * m1);
            c[2] = (int)z;
        } else {
            c[1] = (int)r;
        }
        return;
    }
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

// (A u)[v] with the 3^d-point stencil. All loads are issued before the
// products, so that a vertex costs one memory round trip, not one per point.
template <int DIM, typename T>
__device__ __forceinline__ T stencil_apply(const CGLevelDev<T> &L, int64_t v, const int *c, const T *u) {
    constexpr int NS = DIM == 3 ? 27 : 9;
    T sv[NS], uv[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const int sx = k % 3 - 1, sy = (k / 3) % 3 - 1, sz = DIM == 3 ? k / 9 - 1 : 0;
        const int x = c[0] + sx, y = c[1] + sy, z = DIM == 3 ? c[2] + sz : 0;
        const bool in = x >= 0 && x < L.m[0] && y >= 0 && y < L.m[1] && (DIM == 2 || (z >= 0 && z < L.m[2]));
        const int64_t w = x + (int64_t)L.m[0] * (y + (int64_t)L.m[1] * z);
        sv[k] = in ? __ldg(L.st + (int64_t)k * L.nv + v) : T(0);
        uv[k] = in ? u[w] : T(0);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < NS; ++k) s += sv[k] * uv[k];
    return s;
}

template <int DIM, typename T>
__device__ __forceinline__ void cg_jacobi_at(const CGLevelDev<T> &L, const T *u_in,
                                             const T *b, T *u_out, T omega,
                                             int zero_guess, int64_t v) {
    constexpr int NS = DIM == 3 ? 27 : 9;
    if (v >= L.nv) return;
    const T diag = __ldg(L.st + (int64_t)(NS / 2) * L.nv + v);
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
__device__ __forceinline__ void cg_residual_at(const CGLevelDev<T> &L, const T *u,
                                               const T *b, T *r, int64_t v) {
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
__device__ __forceinline__ void h_restrict_at(const CGLevelDev<T> &L, const T *rf, T *rc,
                                              int64_t V) {
    const int64_t ncv = DIM == 3 ? (int64_t)L.mc[0] * L.mc[1] * L.mc[2] : (int64_t)L.mc[0] * L.mc[1];
    if (V >= ncv) return;
    int C[3] = {0, 0, 0};
    vcoords<DIM>(V, L.mc, C);
    const int sx = __ldg(L.rs_start[0] + C[0]), nx = __ldg(L.rs_cnt[0] + C[0]);
    const int sy = __ldg(L.rs_start[1] + C[1]), ny = __ldg(L.rs_cnt[1] + C[1]);
    const int sz = DIM == 3 ? __ldg(L.rs_start[2] + C[2]) : 0, nz = DIM == 3 ? __ldg(L.rs_cnt[2] + C[2]) : 1;
    // at most 2f - 1 <= 5 children per axis (weights padded to 5): loops unrolled
    // to 5 with the counts as predicates, so that all loads are in flight together
    T wx[5], wy[5], wz[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        wx[i] = __ldg(L.rs_w[0] + C[0] * 5 + i);
        wy[i] = __ldg(L.rs_w[1] + C[1] * 5 + i);
        wz[i] = DIM == 3 ? __ldg(L.rs_w[2] + C[2] * 5 + i) : T(i == 0 ? 1 : 0);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < (DIM == 3 ? 5 : 1); ++k) {
        if (k >= nz) break;
        T f[25];   // the plane's children, loaded before they are summed
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const T *row = rf + (int64_t)L.m[0] * ((sy + j) + (int64_t)L.m[1] * (sz + k)) + sx;
#pragma unroll
            for (int i = 0; i < 5; ++i) f[j * 5 + i] = (j < ny && i < nx) ? row[i] : T(0);
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            T sr = T(0);
#pragma unroll
            for (int i = 0; i < 5; ++i) sr += wx[i] * f[j * 5 + i];
            s += wz[k] * wy[j] * sr;
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
__device__ __forceinline__ void h_prolong_at(const CGLevelDev<T> &L, const T *ec, T *uf,
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
    T e[8];   // the (up to 8) parents, loaded before they are summed
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        const int i = n & 1, j = (n >> 1) & 1, k = n >> 2;
        e[n] = (px[i] >= 0 && py[j] >= 0 && pz[k] >= 0)
                   ? ec[px[i] + (int64_t)L.mc[0] * (py[j] + (int64_t)L.mc[1] * pz[k])]
                   : T(0);
    }
    T s = T(0);
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        const int i = n & 1, j = (n >> 1) & 1, k = n >> 2;
        if (px[i] >= 0 && py[j] >= 0 && pz[k] >= 0) s += wx[i] * wy[j] * wz[k] * e[n];
    }
    uf[v] += s;
}

template <int DIM, typename T>
__global__ void k_h_prolong(CGLevelDev<T> L, const T *__restrict__ ec, T *__restrict__ uf) {
    h_prolong_at<DIM, T>(L, ec, uf, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// e = A_c^{-1} r with the explicit FP64 inverse of the coarsest operator.
template <typename T>
__device__ __forceinline__ void coarse_row(int64_t nc, const double *Ainv, const T *r,
                                           T *e, int64_t i) {
    if (i >= nc) return;
    // four partial sums: four loads of the row in flight at a time
    const double *a = Ainv + i * nc;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t j = 0;
    for (; j + 4 <= nc; j += 4) {
        s0 += __ldg(a + j) * (double)r[j];
        s1 += __ldg(a + j + 1) * (double)r[j + 1];
        s2 += __ldg(a + j + 2) * (double)r[j + 2];
        s3 += __ldg(a + j + 3) * (double)r[j + 3];
    }
    for (; j < nc; ++j) s0 += __ldg(a + j) * (double)r[j];
    e[i] = (T)((s0 + s1) + (s2 + s3));
}

template <typename T>
__global__ void k_coarse_solve(int64_t nc, const double *__restrict__ Ainv, const T *__restrict__ r,
                               T *__restrict__ e) {
    coarse_row<T>(nc, Ainv, r, e, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---- the whole Q1 h-cycle of one problem in one cooperative launch: every step
// of the launch-per-step cycle (point Jacobi, residual, restriction, the dense
// coarsest solve, prolongation) as a loop over the level's vertices split among
// the blocks, the steps separated by a grid-wide barrier instead of kernel
// boundaries. The vectors
// are written and read again inside the one launch, so the per-vertex bodies
// take them through plain pointers (no __restrict__: no loads through the
// non-coherent read-only cache); only the stencils and tables use __ldg.

// Waits of the grid barrier that gave up (zero in every healthy run). Once one
// has, every later cycle launch returns at once: its output is then not to be
// trusted, and this counter (part of dgmg_wait_timeouts) says so.
__device__ unsigned long long g_q1_barrier_timeouts;

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

// Grid-wide barrier of a co-resident (cooperative) grid on a 64-bit arrival
// counter that only grows: every launch on it has the same number of blocks B
// and passes all its barriers, so the counter is a multiple of B when a launch
// starts and barrier k of the launch is passed once it reaches base + (k+1) B
// (base read off the first arrival). One read-modify-write with release and
// acquire order per block, then polling reads with acquire order: the writes
// of the whole grid before the barrier are visible after it. The wait is
// bounded (about a second); a wait that runs out is counted.
struct GridSync {
    unsigned long long *cnt;
    unsigned long long base;
    unsigned k;
    __device__ __forceinline__ void operator()() {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long o = atom_add_acq_rel_gpu(cnt, 1ull);
            if (k == 0) base = o - o % gridDim.x;
            const unsigned long long target = base + (unsigned long long)(k + 1) * gridDim.x;
            if (o + 1 != target) {
                int it = 0;
                while ((long long)(ld_acquire_gpu(cnt) - target) < 0 && ++it < (1 << 20)) __nanosleep(32);
                if (it >= (1 << 20)) atomicAdd(&g_q1_barrier_timeouts, 1ull);
            }
        }
        ++k;
        __syncthreads();
    }
};
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Work split of one step: on the whole grid every block takes an equal run of
// consecutive items (a multiple of 32), its threads stride through it, so a
// level of a few thousand vertices still spreads over all SMs (FP64 FMA
// throughput per SM is low); in one block the threads stride through all.
struct GridEach {
    template <typename F>
    __device__ __forceinline__ void operator()(int64_t n, F &&f) const {
        const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
        const int64_t b = (int64_t)blockIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
        for (int64_t v = b + threadIdx.x; v < e; v += blockDim.x) f(v);
    }
};
struct BlockEach {
    template <typename F>
    __device__ __forceinline__ void operator()(int64_t n, F &&f) const {
        for (int64_t v = threadIdx.x; v < n; v += blockDim.x) f(v);
    }
};

// Down the cycle on level l (not the coarsest): nu_pre Jacobi steps from the
// zero guess, the residual, its restriction into b of level l + 1. The
// iterate ends in u[nu_pre & 1].
template <int DIM, typename T, typename Each, typename Sync>
__device__ __forceinline__ void q1_down(const Q1Plan<T> &p, int l, const Each &each, Sync &sync) {
    const CGLevelDev<T> &L = p.L[l];
    T *u[2] = {p.u0[l], p.u1[l]};
    T *b = p.b[l], *r = p.r[l], *bn = p.b[l + 1];
    const T om = p.omega;
    int c = 0;
    for (int k = 0; k < p.nu_pre; ++k) {
        T *ui = u[c], *uo = u[c ^ 1];
        const int zero = k == 0;
        each(L.nv, [&](int64_t v) { cg_jacobi_at<DIM, T>(L, ui, b, uo, om, zero, v); });
        c ^= 1;
        sync();
    }
    if (p.nu_pre == 0) {
        T *u0 = u[0];
        each(L.nv, [&](int64_t v) { u0[v] = T(0); });
        sync();
    }
    T *uc = u[c];
    each(L.nv, [&](int64_t v) { cg_residual_at<DIM, T>(L, uc, b, r, v); });
    sync();
    const int64_t ncv = DIM == 3 ? (int64_t)L.mc[0] * L.mc[1] * L.mc[2] : (int64_t)L.mc[0] * L.mc[1];
    each(ncv, [&](int64_t V) { h_restrict_at<DIM, T>(L, r, bn, V); });
    sync();
}

// Up the cycle on level l: add the prolongated correction ec of level l + 1,
// nu_post Jacobi steps; returns the level's result, u[(nu_pre + nu_post) & 1].
template <int DIM, typename T, typename Each, typename Sync>
__device__ __forceinline__ const T *q1_up(const Q1Plan<T> &p, int l, const T *ec, const Each &each, Sync &sync) {
    const CGLevelDev<T> &L = p.L[l];
    T *u[2] = {p.u0[l], p.u1[l]};
    T *b = p.b[l];
    const T om = p.omega;
    int c = p.nu_pre & 1;
    T *uc = u[c];
    each(L.nv, [&](int64_t v) { h_prolong_at<DIM, T>(L, ec, uc, v); });
    sync();
    for (int k = 0; k < p.nu_post; ++k) {
        T *ui = u[c], *uo = u[c ^ 1];
        each(L.nv, [&](int64_t v) { cg_jacobi_at<DIM, T>(L, ui, b, uo, om, 0, v); });
        c ^= 1;
        sync();
    }
    return u[c];
}

// The levels from p.local_from down (small enough for one block: the
// threshold is lower in FP64, whose FMA throughput per SM is low) and the
// coarsest solve run in block 0 alone, separated by block barriers; the larger
// levels use the whole grid.
template <int DIM, typename T, int TPB>
__global__ void __launch_bounds__(TPB) k_q1_cycle(const Q1Plan<T> *__restrict__ P, unsigned long long *bar) {
    if (*(volatile unsigned long long *)&g_q1_barrier_timeouts != 0) return;
    const Q1Plan<T> &p = *P;
    // the finest level's stencil is first read after the zero-guess Jacobi step:
    // every block requests its share into L2 now (a hint; 16-byte pieces)
    if (threadIdx.x == 0 && p.nlev > 0) {
        const uint64_t bytes = (uint64_t)(DIM == 3 ? 27 : 9) * p.L[0].nv * sizeof(T);
        const uint64_t chunk = ((bytes + gridDim.x - 1) / gridDim.x + 15) / 16 * 16;
        const uint64_t off = (uint64_t)blockIdx.x * chunk;
        const unsigned char *base = reinterpret_cast<const unsigned char *>(p.L[0].st);
        if (off < bytes && (reinterpret_cast<uintptr_t>(base) & 15) == 0) {
            const uint64_t n = (bytes - off < chunk ? bytes - off : chunk) / 16 * 16;
            if (n > 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base + off), "r"((unsigned)n)
                             : "memory");
        }
    }
    const int nl = p.nlev, ls = p.local_from;
    GridSync grid{bar, 0ull, 0u};
    const GridEach on_grid;
    const int lg = ls < nl - 1 ? ls : nl - 1;   // levels [0, lg) go down on the whole grid
    for (int l = 0; l < lg; ++l) q1_down<DIM, T>(p, l, on_grid, grid);
    const T *ec;
    const T *rc = p.b[nl - 1];
    T *e = p.u0[nl - 1];
    const int64_t nc = p.ncoarse;
    const double *Ainv = p.Ainv;
    if (ls < nl) {
        if (blockIdx.x == 0) {
            BlockSync block;
            const BlockEach on_block;
            for (int l = ls; l < nl - 1; ++l) q1_down<DIM, T>(p, l, on_block, block);
            on_block(nc, [&](int64_t i) { coarse_row<T>(nc, Ainv, rc, e, i); });
            block();
            const T *el = e;
            for (int l = nl - 2; l >= ls; --l) el = q1_up<DIM, T>(p, l, el, on_block, block);
        }
        grid();
        ec = ls == nl - 1 ? e : p.u0[ls];
        if (ls < nl - 1 && ((p.nu_pre + p.nu_post) & 1)) ec = p.u1[ls];
    } else {
        on_grid(nc, [&](int64_t i) { coarse_row<T>(nc, Ainv, rc, e, i); });
        grid();
        ec = e;
    }
    for (int l = lg - 1; l >= 0; --l) ec = q1_up<DIM, T>(p, l, ec, on_grid, grid);
}

// ---- batched forms: work item k covers vertices [v0, v0 + BATCH_VERTS) of
// descriptor map[k].desc (one level of one instance); all instances share one
// persistent launch per stage, whose CTAs stride through the nb work items.
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_corner_gather_batch(const BatchCG<T> *__restrict__ D,
                                                                     const VertMap *__restrict__ map, int nb) {
    for (int k = blockIdx.x; k < nb; k += gridDim.x) {
        const VertMap m = map[k];
        const BatchCG<T> &d = D[m.desc];
        corner_gather_at<DIM, T>(d.n[0], d.n[1], d.n[2], d.corners, d.b, (int64_t)m.v0 + threadIdx.x);
    }
}
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_cg_jacobi_batch(const BatchCG<T> *__restrict__ D,
                                                                 const VertMap *__restrict__ map, int nb, T omega,
                                                                 int zero_guess, int cur) {
    for (int k = blockIdx.x; k < nb; k += gridDim.x) {
        const VertMap m = map[k];
        const BatchCG<T> &d = D[m.desc];
        cg_jacobi_at<DIM, T>(d.L, d.u[cur], d.b, d.u[cur ^ 1], omega, zero_guess, (int64_t)m.v0 + threadIdx.x);
    }
}
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_cg_residual_batch(const BatchCG<T> *__restrict__ D,
                                                                   const VertMap *__restrict__ map, int nb, int cur) {
    for (int k = blockIdx.x; k < nb; k += gridDim.x) {
        const VertMap m = map[k];
        const BatchCG<T> &d = D[m.desc];
        cg_residual_at<DIM, T>(d.L, d.u[cur], d.b, d.r, (int64_t)m.v0 + threadIdx.x);
    }
}
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_h_restrict_batch(const BatchCG<T> *__restrict__ D,
                                                                  const VertMap *__restrict__ map, int nb) {
    for (int k = blockIdx.x; k < nb; k += gridDim.x) {
        const VertMap m = map[k];
        const BatchCG<T> &d = D[m.desc];
        h_restrict_at<DIM, T>(d.L, d.r, d.b_next, (int64_t)m.v0 + threadIdx.x);
    }
}
template <int DIM, typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_h_prolong_batch(const BatchCG<T> *__restrict__ D,
                                                                 const VertMap *__restrict__ map, int nb, int cur) {
    for (int k = blockIdx.x; k < nb; k += gridDim.x) {
        const VertMap m = map[k];
        const BatchCG<T> &d = D[m.desc];
        h_prolong_at<DIM, T>(d.L, d.e_next, d.u[cur], (int64_t)m.v0 + threadIdx.x);
    }
}
template <typename T>
__global__ void __launch_bounds__(BATCH_VERTS) k_coarse_solve_batch(const BatchCG<T> *__restrict__ D,
                                                                    const VertMap *__restrict__ map, int nb) {
    for (int k = blockIdx.x; k < nb; k += gridDim.x) {
        const VertMap m = map[k];
        const BatchCG<T> &d = D[m.desc];
        coarse_row<T>(d.L.nv, d.Ainv, d.b, d.u[0], (int64_t)m.v0 + threadIdx.x);
    }
}

inline unsigned persistent_blocks(const void *fn, int threads, int nb) { return persistent_grid(fn, threads, 0, nb); }

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

}  // namespace

// the kernel of precision T, dimension dim, 256 or (wide, FP32) 512 threads
template <typename T>
const void *q1_cycle_fn(int dim, bool wide) {
    if (wide && sizeof(T) == 4)
        return dim == 3 ? (const void *)k_q1_cycle<3, T, Q1_TPB_WIDE> : (const void *)k_q1_cycle<2, T, Q1_TPB_WIDE>;
    return dim == 3 ? (const void *)k_q1_cycle<3, T, Q1_TPB> : (const void *)k_q1_cycle<2, T, Q1_TPB>;
}

template <typename T>
cudaError_t launch_q1_cycle(int dim, const Q1Plan<T> *plan, unsigned long long *bar, int blocks, bool wide,
                            cudaStream_t s) {
    const bool w = wide && sizeof(T) == 4;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(w ? Q1_TPB_WIDE : Q1_TPB);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident: the grid barrier cannot wait on an unscheduled block
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launches(1);
    if (w) {
        if (dim == 3) return cudaLaunchKernelEx(&cfg, k_q1_cycle<3, T, Q1_TPB_WIDE>, plan, bar);
        return cudaLaunchKernelEx(&cfg, k_q1_cycle<2, T, Q1_TPB_WIDE>, plan, bar);
    }
    if (dim == 3) return cudaLaunchKernelEx(&cfg, k_q1_cycle<3, T, Q1_TPB>, plan, bar);
    return cudaLaunchKernelEx(&cfg, k_q1_cycle<2, T, Q1_TPB>, plan, bar);
}

template <typename T>
int q1_cycle_max_blocks(int dim, bool wide) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    const int tpb = wide && sizeof(T) == 4 ? Q1_TPB_WIDE : Q1_TPB;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, q1_cycle_fn<T>(dim, wide), tpb, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // up to two blocks per SM: warps to hide the load latency of the vertex
    // loops; more would add arrivals at the grid barrier
    return per > 0 ? sms * (per < 2 ? per : 2) : 0;
}

cudaError_t q1_barrier_timeouts(unsigned long long *count) {
    return cudaMemcpyFromSymbol(count, g_q1_barrier_timeouts, sizeof(*count));
}
cudaError_t q1_barrier_timeouts_addr(unsigned long long **ptr) {
    return cudaGetSymbolAddress((void **)ptr, g_q1_barrier_timeouts);
}


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
        k_corner_gather_batch<3, T><<<persistent_blocks((const void *)k_corner_gather_batch<3, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(D, map, nb);
    else
        k_corner_gather_batch<2, T><<<persistent_blocks((const void *)k_corner_gather_batch<2, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(D, map, nb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_jacobi_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, T omega,
                                   bool zero_guess, int cur, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_cg_jacobi_batch<3, T><<<persistent_blocks((const void *)k_cg_jacobi_batch<3, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(
            D, map, nb, omega, zero_guess ? 1 : 0, cur);
    else
        k_cg_jacobi_batch<2, T><<<persistent_blocks((const void *)k_cg_jacobi_batch<2, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(
            D, map, nb, omega, zero_guess ? 1 : 0, cur);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_residual_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, int cur,
                                     cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_cg_residual_batch<3, T><<<persistent_blocks((const void *)k_cg_residual_batch<3, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(
            D, map, nb, cur);
    else
        k_cg_residual_batch<2, T><<<persistent_blocks((const void *)k_cg_residual_batch<2, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(
            D, map, nb, cur);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_h_restrict_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_h_restrict_batch<3, T><<<persistent_blocks((const void *)k_h_restrict_batch<3, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(
            D, map, nb);
    else
        k_h_restrict_batch<2, T><<<persistent_blocks((const void *)k_h_restrict_batch<2, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(
            D, map, nb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_h_prolong_batch(int dim, const BatchCG<T> *D, const VertMap *map, int nb, int cur,
                                   cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    if (dim == 3)
        k_h_prolong_batch<3, T><<<persistent_blocks((const void *)k_h_prolong_batch<3, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(
            D, map, nb, cur);
    else
        k_h_prolong_batch<2, T><<<persistent_blocks((const void *)k_h_prolong_batch<2, T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(
            D, map, nb, cur);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve_batch(const BatchCG<T> *D, const VertMap *map, int nb, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    count_launches(1);
    k_coarse_solve_batch<T><<<persistent_blocks((const void *)k_coarse_solve_batch<T>, BATCH_VERTS, nb), BATCH_VERTS, 0, s>>>(D, map, nb);
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

template cudaError_t launch_q1_cycle<double>(int, const Q1Plan<double> *, unsigned long long *, int, bool,
                                              cudaStream_t);
template cudaError_t launch_q1_cycle<float>(int, const Q1Plan<float> *, unsigned long long *, int, bool,
                                             cudaStream_t);
template int q1_cycle_max_blocks<double>(int, bool);
template int q1_cycle_max_blocks<float>(int, bool);

}  // namespace dgmg
