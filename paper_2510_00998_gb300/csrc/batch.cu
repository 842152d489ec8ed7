// Batched solves: many independent problems share one kernel launch per stage.
// Each problem is solved by the method of dgmg_solve (the hp cycle of Sec. 5.1
// and 5.2 with the single-touch smoothing step of Alg. 4); batching itself has
// no counterpart in the paper.
//
// dgmg_batch_create builds one ordinary hierarchy per problem (all of the
// set-up is the single-problem code), then lays the problems out for batched
// launches:
//  * DG level: problems of equal degree form a group. Their DG vectors are
//    concatenated (each problem starts at a multiple of 32 cells); every stage
//    of the group (projection, smoothing step, residual + p-restriction) is one
//    launch whose CTAs map, through a table, to (problem, first cell), and each
//    CTA runs the single-problem kernel body on its problem's slice with that
//    problem's constants and arrays.
//  * Q1 levels: one launch per stage for all problems (all degrees); a
//    problem's levels end at its own coarsest level, where the batched dense
//    solve takes it, while deeper problems continue the h-cycle.
// The outer iteration is FP64 preconditioned conjugate gradients with the
// batched V-cycle, one recurrence per problem (per-problem dot products, alpha
// and beta, from segmented kernels over the batch vectors): every problem
// follows exactly its own PCG, and a problem that met ||b_i - A_i x_i|| <=
// rtol ||b_i|| is frozen on the device while the others continue. In mixed
// precision the recurrences run in FP32 (FP32 V-cycle and operator) and the
// FP64 solution and true residuals are refreshed at reliable updates of the
// whole batch. One
// iteration of the whole batch is captured in a CUDA graph at its second use
// and replayed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "ctx.h"

using namespace dgmg;

namespace {

constexpr int BATCH_ALIGN_CELLS = 32;   // one CTA of the one-thread-per-cell smoother

// Per-problem CG: every problem runs its own conjugate-gradient recurrence
// (its own alpha and beta); a problem whose residual met its bound is frozen
// (active = 0) and its x, r and p are left untouched.
constexpr int SEG_BLOCKS = 16;   // CTAs per problem of the segmented kernels

// part[i][blockIdx.x] = partial sum of a*b over problem i = blockIdx.y
template <typename T>
__global__ void k_seg_dot_partial(const int64_t *__restrict__ off, const int64_t *__restrict__ len,
                                  const T *__restrict__ a, const T *__restrict__ b, double *__restrict__ part) {
    __shared__ double red[256];
    const int i = blockIdx.y;
    const int64_t o = off[i], n = len[i];
    double s = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        s += (double)a[o + k] * (double)b[o + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)i * SEG_BLOCKS + blockIdx.x] = red[0];
}

// out[i] = sum of the SEG_BLOCKS partials of problem i (fixed order)
__global__ void k_seg_dot_final(int count, const double *__restrict__ part, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double s = 0.0;
    for (int k = 0; k < SEG_BLOCKS; ++k) s += part[(int64_t)i * SEG_BLOCKS + k];
    out[i] = s;
}

// active problems: beta = <r,z>_new / <r,z>; <r,z> <- <r,z>_new
__global__ void k_seg_beta(int count, const int *__restrict__ active, double *__restrict__ rz,
                           const double *__restrict__ rzn, double *__restrict__ beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (!active[i]) {
        beta[i] = 0.0;
        return;
    }
    beta[i] = rzn[i] / rz[i];
    rz[i] = rzn[i];
}

// active problems, flexible (Polak-Ribiere) form for the FP32 V-cycle:
// beta = (<r,z>_new - <r_old,z>) / <r,z>; <r,z> <- <r,z>_new
__global__ void k_seg_beta_flex(int count, const int *__restrict__ active, double *__restrict__ rz,
                                const double *__restrict__ rzn, const double *__restrict__ rzo,
                                double *__restrict__ beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (!active[i]) {
        beta[i] = 0.0;
        return;
    }
    beta[i] = (rzn[i] - rzo[i]) / rz[i];
    rz[i] = rzn[i];
}

// active problems: p = z + beta p
template <typename T>
__global__ void k_seg_update_p(const int64_t *__restrict__ off, const int64_t *__restrict__ len,
                               const int *__restrict__ active, const double *__restrict__ beta, T *__restrict__ p,
                               const T *__restrict__ z) {
    const int i = blockIdx.y;
    if (!active[i]) return;
    const int64_t o = off[i], n = len[i];
    const T bt = (T)beta[i];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        p[o + k] = z[o + k] + bt * p[o + k];
}

// active problems: alpha = <r,z> / <p,q>; x += alpha p; r -= alpha q
__global__ void k_seg_update_xr(const int64_t *__restrict__ off, const int64_t *__restrict__ len,
                                const int *__restrict__ active, const double *__restrict__ rz,
                                const double *__restrict__ pq, double *__restrict__ x, double *__restrict__ r,
                                const double *__restrict__ p, const double *__restrict__ q) {
    const int i = blockIdx.y;
    if (!active[i]) return;
    const int64_t o = off[i], n = len[i];
    const double alpha = rz[i] / pq[i];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        x[o + k] += alpha * p[o + k];
        r[o + k] -= alpha * q[o + k];
    }
}

// Mixed precision (reliable updates), active problems: alpha = <r,z> / <p,q>;
// xs += alpha p; r_old = r; r -= alpha q, all FP32
__global__ void k_seg_update_xr32(const int64_t *__restrict__ off, const int64_t *__restrict__ len,
                                  const int *__restrict__ active, const double *__restrict__ rz,
                                  const double *__restrict__ pq, float *__restrict__ xs, float *__restrict__ r,
                                  float *__restrict__ rold, const float *__restrict__ p,
                                  const float *__restrict__ q) {
    const int i = blockIdx.y;
    if (!active[i]) return;
    const int64_t o = off[i], n = len[i];
    const float alpha = (float)(rz[i] / pq[i]);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float ri = r[o + k];
        rold[o + k] = ri;
        xs[o + k] += alpha * p[o + k];
        r[o + k] = ri - alpha * q[o + k];
    }
}

// x += xs (FP64 accumulation of the FP32 correction), xs = 0, whole batch
__global__ void k_accumulate32(int64_t n, double *__restrict__ x, float *__restrict__ xs) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        x[k] += (double)xs[k];
        xs[k] = 0.f;
    }
}

// active[i] = ||r_i||^2 > rtol^2 ||b_i||^2 (and finite)
__global__ void k_seg_flags(int count, const double *__restrict__ rr, const double *__restrict__ bb, double rtol2,
                            int *__restrict__ active) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double v = rr[i];
    active[i] = (v > rtol2 * bb[i] && v == v) ? 1 : 0;
}

}  // namespace

struct dgmg_batch {
    int count = 0, dim = 0;
    dgmg_opts opts;
    std::vector<dgmg_ctx *> inst;
    std::vector<int> depth;                  // Q1 levels per problem
    struct Group {
        int q = 0;
        std::vector<int> members;            // problem indices
        int64_t cells = 0;                   // padded cells
        int64_t dof0 = 0;                    // first DoF in the batch vectors
        // per precision of the hierarchy (FP64; FP32 for the mixed V-cycle):
        // descriptors (one per member), cells per CTA of projection, smoothing
        // (0: one thread per cell), residual, and the CTA tables
        template <typename T>
        struct Prec {
            BatchDG<T> *D = nullptr;
            int tile[3] = {0, 0, 0};
            BlockMap *map[3] = {nullptr, nullptr, nullptr};
            int nblocks[3] = {0, 0, 0};
        };
        Prec<double> p64;
        Prec<float> p32;
        template <typename T>
        Prec<T> &prec() {
            if constexpr (std::is_same<T, float>::value)
                return p32;
            else
                return p64;
        }
    };
    std::vector<Group> groups;
    bool mixed = false;                      // FP32 V-cycle inside the FP64 CG recurrences
    BatchCG<double> *C = nullptr;            // device, (problem, level) in order
    BatchCG<float> *C32 = nullptr;           // the same levels in FP32 (mixed)
    template <typename T>
    const BatchCG<T> *cg() const {
        if constexpr (std::is_same<T, float>::value)
            return C32;
        else
            return C;
    }
    // mixed precision: reliable-update CG with FP32 recurrences (r32, z32, p32,
    // q32, the correction xs32 since the last FP64 update, the previous
    // residual rold32) and FP64 x and true residuals at the updates
    float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *xs32 = nullptr, *rold32 = nullptr;
    double *rzo = nullptr;                   // <r_old, z>
    struct LevelMaps {
        VertMap *fine = nullptr, *next = nullptr, *coarse = nullptr;
        int nfine = 0, nnext = 0, ncoarse = 0;
    };
    std::vector<LevelMaps> lm;
    VertMap *gather = nullptr;
    int ngather = 0, maxdepth = 0;
    int64_t ndof = 0;
    double *x = nullptr, *b = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    std::vector<int64_t> dof_off, dof_len;
    int64_t *d_off = nullptr, *d_len = nullptr;
    double *d_norm = nullptr, *h_norm = nullptr;   // [count] device, pinned host
    double *d_bb = nullptr;                        // ||b_i||^2 (zero b: 1)
    double *rz = nullptr, *rzn = nullptr, *pq = nullptr, *beta = nullptr, *part = nullptr;
    int *active = nullptr;
    cudaEvent_t ev = nullptr;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;
    int graph_uses = 0;
    long long kernels_per_iteration = 0;
    std::vector<void *> allocs;
    size_t bytes = 0;

    template <typename T>
    int alloc(T **ptr, size_t n) {
        *ptr = nullptr;
        if (n == 0) n = 1;
        cudaError_t e = cudaMalloc((void **)ptr, n * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(DGMG_ENOMEM, "batch: cudaMalloc failed");
        }
        allocs.push_back(*ptr);
        bytes += n * sizeof(T);
        return DGMG_OK;
    }
    template <typename T>
    int upload(T **ptr, const std::vector<T> &h) {
        RC(alloc(ptr, h.size()));
        if (!h.empty()) LC(cudaMemcpy(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
        return DGMG_OK;
    }
    ~dgmg_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        if (ev) cudaEventDestroy(ev);
        if (h_norm) cudaFreeHost(h_norm);
        for (void *ptr : allocs) cudaFree(ptr);
        for (dgmg_ctx *c : inst)
            if (c) dgmg_destroy(c);
    }
};

namespace {

// result vector of Q1 level l of problem i after its part of the h-cycle
template <typename T>
const T *level_result(const dgmg_batch &B, int i, int l) {
    const auto &lv = cgl<T>(*B.inst[i]);
    const CGDev<T> &L = lv[l];
    if (l == B.depth[i] - 1) return L.u[0];
    return L.u[(B.opts.nu_pre + B.opts.nu_post) & 1];
}

template <typename T>
bool cells_apply(const dgmg_batch &B, int q) {
    return B.dim == 3 && q <= (std::is_same<T, float>::value ? 5 : 4) && B.opts.block_inverse == DGMG_BLOCK_EXACT;
}

// The one-thread-per-cell kernel for stage `stage` of precision T: the smoothing
// step, and the residual where the level carries the exact blocks' factors (the
// FP64 level of a mixed batch only applies the operator and has none).
template <typename T>
bool cells_stage(const dgmg_batch &B, int q, int stage) {
    if (!cells_apply<T>(B, q)) return false;
    if (stage == TILE_SMOOTH) return true;
    return stage == TILE_RESIDUAL && !(std::is_same<T, double>::value && B.mixed);
}

template <typename T>
int build_block_map(dgmg_batch &B, dgmg_batch::Group &grp, int stage) {
    auto &g = grp.prec<T>();
    const int nf = (int)(B.inst[grp.members[0]]->nloc / grp.q);
    int tile = g.tile[stage];
    if (tile <= 0) {
        // the one-thread-per-cell smoother where it applies, else ~128 threads
        const bool cells = cells_stage<T>(B, grp.q, stage);
        if (cells) {
            tile = BATCH_ALIGN_CELLS;
        } else {
            tile = std::max(1, 128 / nf);
            while (tile > 1 && tile * nf > 256) --tile;
            g.tile[stage] = tile;
        }
    }
    std::vector<BlockMap> m;
    for (size_t k = 0; k < grp.members.size(); ++k) {
        const int64_t nc = B.inst[grp.members[k]]->ncell;
        for (int64_t c0 = 0; c0 < nc; c0 += tile) m.push_back(BlockMap{(int)k, (int)c0});
    }
    g.nblocks[stage] = (int)m.size();
    return B.upload(&g.map[stage], m);
}

// Tile autotuning of a group's DG-level launches (opts.autotune): every
// candidate cells-per-CTA value (and, for the smoothing step, the
// one-thread-per-cell kernel) is timed on the batch's own buffers, one warm-up
// and three timed launches; the fastest is kept.
template <typename T>
int tune_group(dgmg_batch &B, dgmg_batch::Group &grp, T *u, T *bv, cudaStream_t s) {
    auto &g = grp.prec<T>();
    const int nf = (int)(B.inst[grp.members[0]]->nloc / grp.q);
    const int exact = B.opts.block_inverse == DGMG_BLOCK_EXACT ? 1 : 0;
    std::vector<int> cand;
    for (int c = 1; c <= 64; c *= 2)
        if (c * nf >= 32 && c * nf <= 256) cand.push_back(c);
    if (cand.empty()) cand.push_back(std::max(1, 128 / nf));
    cudaEvent_t e0, e1;
    LC(cudaEventCreate(&e0));
    LC(cudaEventCreate(&e1));
    u += grp.dof0;
    bv += grp.dof0;
    for (int st = 0; st < 3; ++st) {
        // mixed precision: the FP64 level only applies the operator (its problems
        // carry no FP64 block-inverse factors), so its smoothing step is never run
        if (std::is_same<T, double>::value && B.mixed && st == TILE_SMOOTH) continue;
        std::vector<int> cs = cand;
        if (cells_stage<T>(B, grp.q, st)) cs.insert(cs.begin(), 0);
        int best = cs[0];
        float best_ms = 1e30f;
        for (int c : cs) {
            g.tile[st] = c;
            RC(build_block_map<T>(B, grp, st));
            auto launch = [&]() -> cudaError_t {
                if (st == TILE_PROJECT)
                    return launch_project_batch<T>(B.dim, grp.q, g.D, g.map[st], g.nblocks[st], g.tile[st], u, 0, s);
                if (st == TILE_SMOOTH)
                    return launch_smooth_batch<T>(B.dim, grp.q, g.D, g.map[st], g.nblocks[st], g.tile[st], exact, u,
                                                  bv, 0, s);
                return launch_residual_batch<T>(B.dim, grp.q, g.D, g.map[st], g.nblocks[st], g.tile[st],
                                                RES_HAS_B | RES_CORNERS, u, bv, nullptr, 0, s);
            };
            float ms = 1e30f;
            if (launch() == cudaSuccess) {
                cudaEventRecord(e0, s);
                bool ok = true;
                for (int k = 0; k < 3 && ok; ++k) ok = launch() == cudaSuccess;
                cudaEventRecord(e1, s);
                if (ok && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            }
            cudaGetLastError();
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        g.tile[st] = best;
        RC(build_block_map<T>(B, grp, st));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LC(cudaStreamSynchronize(s));
    return DGMG_OK;
}

void push_verts(std::vector<VertMap> &m, int desc, int64_t n) {
    for (int64_t v0 = 0; v0 < n; v0 += BATCH_VERTS) m.push_back(VertMap{desc, (int)v0});
}

// ---- batched stages
int batch_apply(dgmg_batch &B, const double *u, const double *bvec, double *out, cudaStream_t s) {
    const int mode = bvec ? (RES_HAS_B | RES_WRITE_R) : (RES_WRITE_R | RES_NEGATE);
    for (auto &grp : B.groups) {
        auto &g = grp.p64;
        LC(launch_project_batch<double>(B.dim, grp.q, g.D, g.map[TILE_PROJECT], g.nblocks[TILE_PROJECT],
                                        g.tile[TILE_PROJECT], const_cast<double *>(u) + grp.dof0, 0, s));
        LC(launch_residual_batch<double>(B.dim, grp.q, g.D, g.map[TILE_RESIDUAL], g.nblocks[TILE_RESIDUAL],
                                         g.tile[TILE_RESIDUAL], mode, u + grp.dof0, bvec ? bvec + grp.dof0 : nullptr,
                                         out + grp.dof0, 0, s));
    }
    return DGMG_OK;
}

// out = A u with the FP32 operator of every problem (projection + residual
// with b = 0, sign flipped), all groups
int batch_apply32(dgmg_batch &B, const float *u, float *out, cudaStream_t s) {
    for (auto &grp : B.groups) {
        auto &g = grp.p32;
        LC(launch_project_batch<float>(B.dim, grp.q, g.D, g.map[TILE_PROJECT], g.nblocks[TILE_PROJECT],
                                       g.tile[TILE_PROJECT], const_cast<float *>(u) + grp.dof0, 0, s));
        LC(launch_residual_batch<float>(B.dim, grp.q, g.D, g.map[TILE_RESIDUAL], g.nblocks[TILE_RESIDUAL],
                                        g.tile[TILE_RESIDUAL], RES_WRITE_R | RES_NEGATE | RES_DIRECT, u + grp.dof0,
                                        nullptr, out + grp.dof0, 0, s));
    }
    return DGMG_OK;
}

template <typename T>
int batch_cg_cycle(dgmg_batch &B, int l, cudaStream_t s) {
    const auto &m = B.lm[l];
    const BatchCG<T> *C = B.cg<T>();
    const T om = (T)B.opts.omega_cg;
    LC(launch_coarse_solve_batch<T>(C, m.coarse, m.ncoarse, s));
    if (m.nfine == 0) return DGMG_OK;
    int cur = 0;
    for (int k = 0; k < B.opts.nu_pre; ++k) {
        LC(launch_cg_jacobi_batch<T>(B.dim, C, m.fine, m.nfine, om, k == 0, cur, s));
        cur ^= 1;
    }
    LC(launch_cg_residual_batch<T>(B.dim, C, m.fine, m.nfine, cur, s));
    LC(launch_h_restrict_batch<T>(B.dim, C, m.next, m.nnext, s));
    RC(batch_cg_cycle<T>(B, l + 1, s));
    LC(launch_h_prolong_batch<T>(B.dim, C, m.fine, m.nfine, cur, s));
    for (int k = 0; k < B.opts.nu_post; ++k) {
        LC(launch_cg_jacobi_batch<T>(B.dim, C, m.fine, m.nfine, om, false, cur, s));
        cur ^= 1;
    }
    return DGMG_OK;
}

// z = V(r) for every problem at once (zero initial guess), in precision T
template <typename T>
int batch_vcycle(dgmg_batch &B, const T *r, T *z, cudaStream_t s) {
    const int exact = B.opts.block_inverse == DGMG_BLOCK_EXACT ? 1 : 0;
    LC(cudaMemsetAsync(z, 0, sizeof(T) * B.ndof, s));
    for (auto &grp : B.groups)
        LC(launch_zero_traces_batch<T>(B.dim, grp.q, grp.prec<T>().D, (int)grp.members.size(), s));
    auto smooth = [&](int k) -> int {
        for (auto &grp : B.groups) {
            auto &g = grp.prec<T>();
            LC(launch_smooth_batch<T>(B.dim, grp.q, g.D, g.map[TILE_SMOOTH], g.nblocks[TILE_SMOOTH],
                                      g.tile[TILE_SMOOTH], exact, z + grp.dof0, r + grp.dof0, k & 1, s));
        }
        return DGMG_OK;
    };
    for (int k = 0; k < B.opts.nu_pre; ++k) RC(smooth(k));
    for (auto &grp : B.groups) {
        auto &g = grp.prec<T>();
        LC(launch_residual_batch<T>(B.dim, grp.q, g.D, g.map[TILE_RESIDUAL], g.nblocks[TILE_RESIDUAL],
                                    g.tile[TILE_RESIDUAL], RES_HAS_B | RES_CORNERS, z + grp.dof0, r + grp.dof0,
                                    nullptr, B.opts.nu_pre & 1, s));
    }
    LC(launch_corner_gather_batch<T>(B.dim, B.cg<T>(), B.gather, B.ngather, s));
    RC(batch_cg_cycle<T>(B, 0, s));
    for (auto &grp : B.groups) {
        auto &g = grp.prec<T>();
        LC(launch_project_batch<T>(B.dim, grp.q, g.D, g.map[TILE_PROJECT], g.nblocks[TILE_PROJECT],
                                   g.tile[TILE_PROJECT], z + grp.dof0, 1, s));
    }
    for (int k = 0; k < B.opts.nu_post; ++k) RC(smooth(k));
    return DGMG_OK;
}

unsigned small_grid(int count) { return (unsigned)((count + 127) / 128); }

// out[i] = <a_i, b_i> for every problem (deterministic: fixed partial order; FP64 sums)
template <typename T>
int seg_dot(dgmg_batch &B, const T *a, const T *b, double *out, cudaStream_t s) {
    count_launches(2);
    k_seg_dot_partial<T><<<dim3(SEG_BLOCKS, B.count), 256, 0, s>>>(B.d_off, B.d_len, a, b, B.part);
    k_seg_dot_final<<<small_grid(B.count), 128, 0, s>>>(B.count, B.part, out);
    LC(cudaGetLastError());
    return DGMG_OK;
}

// ||v_i||^2 of every problem to the host (pinned) and the active flags
int batch_norms(dgmg_batch &B, const double *v, cudaStream_t s) {
    RC(seg_dot(B, v, v, B.d_norm, s));
    count_launches(1);
    k_seg_flags<<<small_grid(B.count), 128, 0, s>>>(B.count, B.d_norm, B.d_bb, B.opts.rtol * B.opts.rtol, B.active);
    LC(cudaGetLastError());
    LC(cudaMemcpyAsync(B.h_norm, B.d_norm, sizeof(double) * B.count, cudaMemcpyDeviceToHost, s));
    return DGMG_OK;
}

// FP64: alpha step of every active problem: q = A p, <p,q>, x += alpha p,
// r -= alpha q, then ||r_i||^2 and the flags
int alpha_step(dgmg_batch &B, cudaStream_t s) {
    RC(batch_apply(B, B.p, nullptr, B.q, s));
    RC(seg_dot<double>(B, B.p, B.q, B.pq, s));
    count_launches(1);
    k_seg_update_xr<<<dim3(SEG_BLOCKS * 4, B.count), 256, 0, s>>>(B.d_off, B.d_len, B.active, B.rz, B.pq, B.x,
                                                                    B.r, B.p, B.q);
    LC(cudaGetLastError());
    return batch_norms(B, B.r, s);
}

// One iteration of every active problem. FP64: z = V(r), beta, p = z + beta p,
// the alpha step. Mixed precision (FP32 recurrences of the reliable-update CG):
// z = V(r) in FP32, flexible (Polak-Ribiere) beta, p = z + beta p, q = A p with
// the FP32 operator, xs += alpha p, r -= alpha q, and ||r_i||^2 of the FP32
// recursive residuals to the host (no flags: those follow the FP64 updates).
int batch_iteration(dgmg_batch &B, cudaStream_t s) {
    if (!B.mixed) {
        RC(batch_vcycle<double>(B, B.r, B.z, s));
        RC(seg_dot<double>(B, B.r, B.z, B.rzn, s));
        count_launches(2);
        k_seg_beta<<<small_grid(B.count), 128, 0, s>>>(B.count, B.active, B.rz, B.rzn, B.beta);
        k_seg_update_p<double><<<dim3(SEG_BLOCKS * 4, B.count), 256, 0, s>>>(B.d_off, B.d_len, B.active, B.beta,
                                                                              B.p, B.z);
        LC(cudaGetLastError());
        return alpha_step(B, s);
    }
    RC(batch_vcycle<float>(B, B.r32, B.z32, s));
    RC(seg_dot<float>(B, B.r32, B.z32, B.rzn, s));
    RC(seg_dot<float>(B, B.rold32, B.z32, B.rzo, s));
    count_launches(2);
    k_seg_beta_flex<<<small_grid(B.count), 128, 0, s>>>(B.count, B.active, B.rz, B.rzn, B.rzo, B.beta);
    k_seg_update_p<float><<<dim3(SEG_BLOCKS * 4, B.count), 256, 0, s>>>(B.d_off, B.d_len, B.active, B.beta, B.p32,
                                                                         B.z32);
    LC(cudaGetLastError());
    RC(batch_apply32(B, B.p32, B.q32, s));
    RC(seg_dot<float>(B, B.p32, B.q32, B.pq, s));
    count_launches(1);
    k_seg_update_xr32<<<dim3(SEG_BLOCKS * 4, B.count), 256, 0, s>>>(B.d_off, B.d_len, B.active, B.rz, B.pq,
                                                                      B.xs32, B.r32, B.rold32, B.p32, B.q32);
    LC(cudaGetLastError());
    RC(seg_dot<float>(B, B.r32, B.r32, B.d_norm, s));
    LC(cudaMemcpyAsync(B.h_norm, B.d_norm, sizeof(double) * B.count, cudaMemcpyDeviceToHost, s));
    return DGMG_OK;
}

// Mixed precision, reliable update of every problem: x += xs (FP64), xs = 0,
// r = b - A x with the FP64 operator, ||r_i||^2 and the flags (a problem that
// met its bound is frozen), r32 = r.
int reliable_update(dgmg_batch &B, cudaStream_t s) {
    count_launches(1);
    k_accumulate32<<<608, 256, 0, s>>>(B.ndof, B.x, B.xs32);
    LC(cudaGetLastError());
    RC(batch_apply(B, B.x, B.b, B.r, s));
    RC(batch_norms(B, B.r, s));
    LC(launch_cast_d2f(B.ndof, B.r, B.r32, s));
    return DGMG_OK;
}

// the steady-state iteration as one CUDA graph (captured at its second use)
int run_iteration(dgmg_batch &B, cudaStream_t s) {
    if (B.graph_uses++ == 0) {
        const long long before = g_kernel_launches.load();
        RC(batch_iteration(B, s));
        B.kernels_per_iteration = g_kernel_launches.load() - before;
        return DGMG_OK;
    }
    if (!B.exec) {
        const long long before = g_kernel_launches.load();
        LC(cudaStreamBeginCapture(B.capture_stream, cudaStreamCaptureModeRelaxed));
        const int rc = batch_iteration(B, B.capture_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(B.capture_stream, &graph);
        B.graph_kernels = g_kernel_launches.load() - before;
        g_kernel_launches.fetch_sub(B.graph_kernels);
        if (rc != DGMG_OK || e != cudaSuccess || cudaGraphInstantiate(&B.exec, graph, 0) != cudaSuccess) {
            // capture not possible now (e.g. invalidated from another thread): run eagerly
            if (graph) cudaGraphDestroy(graph);
            B.exec = nullptr;
            cudaGetLastError();
            B.graph_uses = 1;
            return batch_iteration(B, s);
        }
        cudaGraphDestroy(graph);
    }
    LC(cudaGraphLaunch(B.exec, s));
    count_launches((int)B.graph_kernels);
    return DGMG_OK;
}

// DG descriptors of a group in precision T (FP32 from the problems' FP32 hierarchies)
template <typename T>
std::vector<BatchDG<T>> group_descriptors(const dgmg_batch &B, const dgmg_batch::Group &grp) {
    std::vector<BatchDG<T>> D;
    int64_t cells = 0;
    for (int i : grp.members) {
        dgmg_ctx *c = B.inst[i];
        const DGDev<T> &dg = dgmg::dg<T>(*c);
        BatchDG<T> d{};
        d.c = dg.c;
        d.off = cells;
        d.kappa = dg.kappa;
        d.fd = dg.fd;
        d.fdr = dg.fdr;
        d.linv = dg.linv;
        d.tr[0] = dg.tr[0];
        d.tr[1] = dg.tr[1];
        d.corners = dg.corners;
        d.e0 = cgl<T>(*c).empty() ? nullptr : level_result<T>(B, i, 0);
        D.push_back(d);
        cells += (c->ncell + BATCH_ALIGN_CELLS - 1) / BATCH_ALIGN_CELLS * BATCH_ALIGN_CELLS;
    }
    return D;
}

// Q1 descriptors of every (problem, level) in precision T
template <typename T>
std::vector<BatchCG<T>> level_descriptors(const dgmg_batch &B) {
    std::vector<BatchCG<T>> C;
    for (int i = 0; i < B.count; ++i) {
        dgmg_ctx *c = B.inst[i];
        const auto &lv = cgl<T>(*c);
        for (int l = 0; l < B.depth[i]; ++l) {
            const CGDev<T> &L = lv[l];
            BatchCG<T> e{};
            e.L = L.L;
            e.u[0] = L.u[0];
            e.u[1] = L.u[1];
            e.b = L.b;
            e.r = L.r;
            const bool last = l == B.depth[i] - 1;
            e.b_next = last ? nullptr : lv[l + 1].b;
            e.e_next = last ? nullptr : level_result<T>(B, i, l + 1);
            e.Ainv = last ? c->coarse_inv : nullptr;
            for (int a = 0; a < 3; ++a) e.n[a] = c->n[a];
            e.corners = dgmg::dg<T>(*c).corners;
            C.push_back(e);
        }
    }
    return C;
}

}  // namespace

extern "C" {

int dgmg_batch_create(int count, const dgmg_mesh *meshes, const int *p, const double *const *kappa,
                      const dgmg_opts *opts, dgmg_batch **out) {
    if (!out) return fail(DGMG_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1) return fail(DGMG_EINVAL, "count must be >= 1");
    if (!meshes || !p) return fail(DGMG_EINVAL, "meshes and p must not be NULL");
    dgmg_opts o;
    dgmg_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != DGMG_FP64 && o.precision != DGMG_MIXED_FP32) return fail(DGMG_EINVAL, "unknown precision");
    if (o.nu_pre < 1) return fail(DGMG_EINVAL, "batched solves need nu_pre >= 1");
    if (o.p_coarsening != 0) return fail(DGMG_EINVAL, "batched solves coarsen p directly to Q1 (p_coarsening 0)");
    if (o.basis != DGMG_BASIS_GLL) return fail(DGMG_EINVAL, "batched solves use the GLL basis");
    if (o.recompute_block != 0) return fail(DGMG_EINVAL, "batched solves use the precomputed block factors");
    for (int i = 0; i < count; ++i)
        if (meshes[i].dim != meshes[0].dim) return fail(DGMG_EINVAL, "all meshes of a batch have one dimension");
    const bool trace = std::getenv("DGMG_TRACE_SETUP") != nullptr;
    auto tmark = std::chrono::steady_clock::now();
    auto phase = [&](const char *what) {
        if (!trace) return;
        const auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "dgmg batch setup %-18s %9.3f ms\n", what,
                     std::chrono::duration<double, std::milli>(now - tmark).count());
        tmark = now;
    };
    std::unique_ptr<dgmg_batch> B(new dgmg_batch());
    B->count = count;
    B->dim = meshes[0].dim;
    dgmg_opts oi = o;
    oi.outer = DGMG_OUTER_PCG;
    oi.autotune = 0;
    B->opts = oi;
    B->mixed = o.precision == DGMG_MIXED_FP32;
    // one hierarchy per problem, built on a few host threads (without the parts
    // the batch does not use)
    const int flags = CREATE_NO_SOLVER | (B->mixed ? CREATE_NO_FP64_SMOOTHER | CREATE_NO_FP64_Q1 : 0);
    B->inst.assign(count, nullptr);
    std::vector<int> rcs(count, DGMG_OK);
    std::vector<std::string> errs(count);
    {
        const int nt = std::max(1, std::min(count, 8));
        std::vector<std::thread> th;
        int dev = 0;
        cudaGetDevice(&dev);
        for (int t = 0; t < nt; ++t)
            th.emplace_back([&, t]() {
                cudaSetDevice(dev);
                for (int i = t; i < count; i += nt) {
                    rcs[i] = create_ctx(&meshes[i], p[i], kappa ? kappa[i] : nullptr, &oi, flags, &B->inst[i]);
                    if (rcs[i] != DGMG_OK) errs[i] = dgmg_last_error();
                }
            });
        for (auto &x : th) x.join();
    }
    for (int i = 0; i < count; ++i)
        if (rcs[i] != DGMG_OK) return fail(rcs[i], "batch problem " + std::to_string(i) + ": " + errs[i]);
    phase("hierarchies");
    for (int i = 0; i < count; ++i)
        B->depth.push_back((int)(B->mixed ? B->inst[i]->cg32.size() : B->inst[i]->cg64.size()));

    // DG groups by degree; each problem starts at a multiple of 32 cells
    for (int i = 0; i < count; ++i) {
        const int q = B->inst[i]->q;
        auto it = std::find_if(B->groups.begin(), B->groups.end(), [q](const dgmg_batch::Group &g) { return g.q == q; });
        if (it == B->groups.end()) {
            B->groups.emplace_back();
            B->groups.back().q = q;
            it = B->groups.end() - 1;
        }
        it->members.push_back(i);
    }
    B->dof_off.assign(count, 0);
    B->dof_len.assign(count, 0);
    int64_t dof = 0;
    for (auto &g : B->groups) {
        g.dof0 = dof;
        int64_t cells = 0;
        for (int i : g.members) {
            dgmg_ctx *c = B->inst[i];
            B->dof_off[i] = g.dof0 + cells * c->nloc;
            B->dof_len[i] = c->ndof;
            cells += (c->ncell + BATCH_ALIGN_CELLS - 1) / BATCH_ALIGN_CELLS * BATCH_ALIGN_CELLS;
        }
        g.cells = cells;
        dof += cells * B->inst[g.members[0]]->nloc;
        RC(B->upload(&g.p64.D, group_descriptors<double>(*B, g)));
        g.p64.tile[TILE_SMOOTH] = 0;
        for (int st = 0; st < 3; ++st) RC(build_block_map<double>(*B, g, st));
        if (B->mixed) {
            RC(B->upload(&g.p32.D, group_descriptors<float>(*B, g)));
            g.p32.tile[TILE_SMOOTH] = 0;
            for (int st = 0; st < 3; ++st) RC(build_block_map<float>(*B, g, st));
        }
    }
    B->ndof = dof;
    phase("dg descriptors");

    // Q1 levels of all problems (the same order in both precisions)
    std::vector<std::vector<int>> desc(count);
    {
        int k = 0;
        for (int i = 0; i < count; ++i) {
            for (int l = 0; l < B->depth[i]; ++l) desc[i].push_back(k++);
            B->maxdepth = std::max(B->maxdepth, B->depth[i]);
        }
    }
    if (B->mixed)
        RC(B->upload(&B->C32, level_descriptors<float>(*B)));
    else
        RC(B->upload(&B->C, level_descriptors<double>(*B)));
    {
        std::vector<VertMap> gm;
        for (int i = 0; i < count; ++i) push_verts(gm, desc[i][0], B->inst[i]->lv[0].nv);
        B->ngather = (int)gm.size();
        RC(B->upload(&B->gather, gm));
    }
    B->lm.resize(B->maxdepth);
    for (int l = 0; l < B->maxdepth; ++l) {
        std::vector<VertMap> fine, next, coarse;
        for (int i = 0; i < count; ++i) {
            if (l >= B->depth[i]) continue;
            const int64_t nv = B->inst[i]->lv[l].nv;
            if (l == B->depth[i] - 1) {
                push_verts(coarse, desc[i][l], nv);
            } else {
                push_verts(fine, desc[i][l], nv);
                push_verts(next, desc[i][l], B->inst[i]->lv[l + 1].nv);
            }
        }
        auto &m = B->lm[l];
        m.nfine = (int)fine.size();
        m.nnext = (int)next.size();
        m.ncoarse = (int)coarse.size();
        RC(B->upload(&m.fine, fine));
        RC(B->upload(&m.next, next));
        RC(B->upload(&m.coarse, coarse));
    }

    // batch vectors (padding stays zero), per-problem slices, scalars
    for (double **v : {&B->x, &B->b, &B->r, &B->z, &B->p, &B->q}) {
        RC(B->alloc(v, B->ndof));
        LC(cudaMemset(*v, 0, sizeof(double) * B->ndof));
    }
    RC(B->upload(&B->d_off, B->dof_off));
    RC(B->upload(&B->d_len, B->dof_len));
    for (double **v : {&B->d_norm, &B->d_bb, &B->rz, &B->rzn, &B->pq, &B->beta}) RC(B->alloc(v, count));
    RC(B->alloc(&B->part, (size_t)count * SEG_BLOCKS));
    RC(B->alloc(&B->active, count));
    if (B->mixed) {
        for (float **v : {&B->r32, &B->z32, &B->p32, &B->q32, &B->xs32, &B->rold32}) {
            RC(B->alloc(v, B->ndof));
            LC(cudaMemset(*v, 0, sizeof(float) * B->ndof));
        }
        RC(B->alloc(&B->rzo, count));
    }
    LC(cudaMallocHost((void **)&B->h_norm, sizeof(double) * count));
    LC(cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming));
    LC(cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking));
    for (dgmg_ctx *c : B->inst) B->bytes += c->bytes;
    LC(cudaDeviceSynchronize());
    phase("q1 descriptors");
    if (o.autotune) {
        for (auto &g : B->groups) {
            RC(tune_group<double>(*B, g, B->z, B->r, B->capture_stream));   // mixed: the FP64 apply only
            if (B->mixed) RC(tune_group<float>(*B, g, B->z32, B->r32, B->capture_stream));
        }
        phase("autotune");
    }
    *out = B.release();
    return DGMG_OK;
}

int dgmg_batch_info(const dgmg_batch *B, dgmg_batch_info_t *info) {
    if (!B || !info) return fail(DGMG_EINVAL, "batch and info must not be NULL");
    std::memset(info, 0, sizeof(*info));
    info->count = B->count;
    info->groups = (int)B->groups.size();
    info->ndof = B->ndof;
    info->device_bytes = B->bytes;
    info->max_levels = B->maxdepth;
    info->kernels_per_iteration = B->kernels_per_iteration;
    for (size_t k = 0; k < B->groups.size() && k < 4; ++k) {
        info->group_q[k] = B->groups[k].q;
        for (int st = 0; st < 3; ++st)
            info->group_tiles[k][st] = B->mixed ? B->groups[k].p32.tile[st] : B->groups[k].p64.tile[st];
    }
    return DGMG_OK;
}

int dgmg_batch_solve(dgmg_batch *B, const double *const *b, double *const *x, dgmg_stats *stats, void *stream) {
    if (!B) return fail(DGMG_EINVAL, "batch is NULL");
    if (!b || !x) return fail(DGMG_EINVAL, "b and x must not be NULL");
    for (int i = 0; i < B->count; ++i)
        if (!b[i] || !x[i]) return fail(DGMG_EINVAL, "b[i] and x[i] must not be NULL");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    const int n = B->count;
    for (int i = 0; i < n; ++i) {
        LC(cudaMemcpyAsync(B->b + B->dof_off[i], b[i], sizeof(double) * B->dof_len[i], cudaMemcpyDeviceToDevice, s));
        LC(cudaMemcpyAsync(B->x + B->dof_off[i], x[i], sizeof(double) * B->dof_len[i], cudaMemcpyDeviceToDevice, s));
    }
    std::vector<double> bn(n), rel(n);
    RC(seg_dot<double>(*B, B->b, B->b, B->d_norm, s));
    LC(cudaMemcpyAsync(B->h_norm, B->d_norm, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    LC(cudaStreamSynchronize(s));
    std::vector<double> bb(n);
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(B->h_norm[i])) return fail(DGMG_ENONFINITE, "||b|| is not finite");
        bn[i] = B->h_norm[i] > 0 ? std::sqrt(B->h_norm[i]) : 1.0;
        bb[i] = bn[i] * bn[i];
    }
    LC(cudaMemcpyAsync(B->d_bb, bb.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    auto converged = [&]() {
        double worst = 0.0;
        for (int i = 0; i < n; ++i) {
            rel[i] = std::sqrt(B->h_norm[i]) / bn[i];
            worst = std::max(worst, std::isfinite(rel[i]) ? rel[i] : INFINITY);
        }
        return worst;
    };
    RC(batch_apply(*B, B->x, B->b, B->r, s));   // r = b - A x
    RC(batch_norms(*B, B->r, s));
    LC(cudaStreamSynchronize(s));
    double worst = converged();
    int status = DGMG_OK, it = 0;
    std::vector<int> its(n, -1);              // iteration at which each problem met its bound
    auto mark = [&]() {
        for (int i = 0; i < n; ++i)
            if (its[i] < 0 && rel[i] <= B->opts.rtol) its[i] = it;
    };
    mark();
    int fp64_applies = 2;                     // the initial and the final true residuals
    if (worst > B->opts.rtol && B->mixed) {
        // reliable-update CG: FP32 recurrences, FP64 x and true residuals at the
        // updates. An update of the whole batch runs when half of the active
        // problems have reduced their recursive residual by `delta` since their
        // last update, when all of them are below the tolerance, or every
        // RELIABLE_MAX_GAP iterations; it freezes the problems that met their bound.
        constexpr int RELIABLE_MAX_GAP = 10;
        std::vector<double> rel_upd(rel);
        LC(launch_cast_d2f(B->ndof, B->r, B->r32, s));
        RC(batch_vcycle<float>(*B, B->r32, B->z32, s));
        RC(seg_dot<float>(*B, B->r32, B->z32, B->rz, s));
        LC(cudaMemcpyAsync(B->p32, B->z32, sizeof(float) * B->ndof, cudaMemcpyDeviceToDevice, s));
        RC(batch_apply32(*B, B->p32, B->q32, s));
        RC(seg_dot<float>(*B, B->p32, B->q32, B->pq, s));
        count_launches(1);
        k_seg_update_xr32<<<dim3(SEG_BLOCKS * 4, n), 256, 0, s>>>(B->d_off, B->d_len, B->active, B->rz, B->pq,
                                                                    B->xs32, B->r32, B->rold32, B->p32, B->q32);
        LC(cudaGetLastError());
        RC(seg_dot<float>(*B, B->r32, B->r32, B->d_norm, s));
        LC(cudaMemcpyAsync(B->h_norm, B->d_norm, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        std::vector<int> act(n);
        for (int i = 0; i < n; ++i) act[i] = rel[i] > B->opts.rtol;
        it = 1;
        int gap = 1;
        for (;;) {
            LC(cudaEventRecord(B->ev, s));
            LC(cudaEventSynchronize(B->ev));
            int nact = 0, due = 0, below = 0;
            for (int i = 0; i < n; ++i) {
                if (!act[i]) continue;
                ++nact;
                const double rr = std::sqrt(B->h_norm[i]) / bn[i];
                if (!std::isfinite(rr) || rr <= B->opts.delta * rel_upd[i]) ++due;
                if (rr <= B->opts.rtol) ++below;
            }
            if (2 * due >= nact || below == nact || gap >= RELIABLE_MAX_GAP) {
                RC(reliable_update(*B, s));
                ++fp64_applies;
                LC(cudaStreamSynchronize(s));
                worst = converged();
                mark();
                for (int i = 0; i < n; ++i) {
                    rel_upd[i] = rel[i];
                    act[i] = rel[i] > B->opts.rtol;
                }
                gap = 0;
                if (!std::isfinite(worst)) {
                    status = fail(DGMG_ENONFINITE, "residual norm is not finite");
                    break;
                }
                if (worst <= B->opts.rtol) break;
            }
            if (it >= B->opts.maxit) {
                status = fail(DGMG_ENOTCONVERGED, "maxit reached");
                break;
            }
            RC(run_iteration(*B, s));
            ++it;
            ++gap;
        }
        count_launches(1);
        k_accumulate32<<<608, 256, 0, s>>>(B->ndof, B->x, B->xs32);   // the correction since the last update
        LC(cudaGetLastError());
    } else if (worst > B->opts.rtol) {
        RC(batch_vcycle<double>(*B, B->r, B->z, s));
        RC(seg_dot<double>(*B, B->r, B->z, B->rz, s));
        LC(cudaMemcpyAsync(B->p, B->z, sizeof(double) * B->ndof, cudaMemcpyDeviceToDevice, s));
        RC(alpha_step(*B, s));
        ++fp64_applies;
        it = 1;
        for (;;) {
            LC(cudaEventRecord(B->ev, s));
            LC(cudaEventSynchronize(B->ev));
            worst = converged();
            mark();
            if (!std::isfinite(worst)) {
                status = fail(DGMG_ENONFINITE, "residual norm is not finite");
                break;
            }
            if (worst <= B->opts.rtol) break;
            if (it >= B->opts.maxit) {
                status = fail(DGMG_ENOTCONVERGED, "maxit reached");
                break;
            }
            RC(run_iteration(*B, s));
            ++it;
            ++fp64_applies;
        }
    }
    // true residuals of the returned iterates
    RC(batch_apply(*B, B->x, B->b, B->r, s));
    RC(batch_norms(*B, B->r, s));
    for (int i = 0; i < n; ++i)
        LC(cudaMemcpyAsync(x[i], B->x + B->dof_off[i], sizeof(double) * B->dof_len[i], cudaMemcpyDeviceToDevice, s));
    LC(cudaStreamSynchronize(s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats)
        for (int i = 0; i < n; ++i) {
            const double recursive = rel[i];
            std::memset(&stats[i], 0, sizeof(stats[i]));
            stats[i].iterations = its[i] >= 0 ? its[i] : it;
            stats[i].rel_residual = std::sqrt(B->h_norm[i]) / bn[i];
            stats[i].rel_residual_recursive = recursive;
            stats[i].seconds = secs;
            stats[i].fp64_applies = fp64_applies;
        }
    return status;
}

int dgmg_batch_destroy(dgmg_batch *B) {
    delete B;
    return DGMG_OK;
}

}  // extern "C"
