// Internal definition of the libdgmg context (shared by ctx.cu, solver.cu and
// server.cu; not part of the C ABI).
#pragma once

#include <chrono>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace dgmg {

// --------------------------------------------------------------- Q1 levels
// One continuous Q1 level on the host: stencils (SoA [3^d][nv]) and the
// per-axis transfer tables to the next coarser level.
struct CGLevelHost {
    int n[3] = {1, 1, 1};   // cells per axis
    int m[3] = {1, 1, 1};   // interior vertices per axis
    int64_t nv = 0;
    std::vector<double> st;
    // transfer to the next level (empty on the coarsest)
    int mc[3] = {1, 1, 1};
    std::vector<int> pl_lo[3], pl_hi[3], rs_start[3], rs_cnt[3];
    std::vector<double> pl_wlo[3], pl_whi[3], rs_w[3];
};


}  // namespace dgmg

using namespace dgmg;

// ---------------------------------------------------------------- context
template <typename T>
struct DGDev {
    DGConst<T> c;
    T *kappa = nullptr, *fd = nullptr, *tr[2] = {nullptr, nullptr}, *corners = nullptr;
    T *linv = nullptr;   // per-node omega / (sum of the cell's eigenvalues); FP64 only
    T *fdr = nullptr;    // the residual's factors [S^T M | lambda] per cell and axis
    T *kfac = nullptr;   // facet coefficients [cell][face]
};

template <typename T>
struct CGDev {
    CGLevelDev<T> L;
    T *st = nullptr;
    T *u[2] = {nullptr, nullptr}, *b = nullptr, *r = nullptr;
    int *itab = nullptr;
    T *wtab = nullptr;
};

// Per-stage device time, recorded with CUDA events on the launching stream
// around every stage launch while profiling is on (dgmg_profile).
enum { ST_PROJECT = 0, ST_SMOOTH = 1, ST_RESIDUAL = 2, ST_CG = 3, ST_VECTOR = 4, ST_N = 5 };
enum { TILE_PROJECT = 0, TILE_SMOOTH = 1, TILE_RESIDUAL = 2 };
struct StageProfiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;        // pairs: 2k start, 2k+1 stop
    std::vector<int> stage;
    size_t used = 0;
    double ms[ST_N] = {0};
    long long cnt[ST_N] = {0};
    int open_stage = -1;
    void begin(int st, cudaStream_t s) {
        if (!on) return;
        if (2 * used + 2 > ev.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            ev.push_back(a);
            ev.push_back(b);
            stage.push_back(st);
        }
        stage[used] = st;
        cudaEventRecord(ev[2 * used], s);
        open_stage = st;
    }
    void end(cudaStream_t s) {
        if (!on || open_stage < 0) return;
        cudaEventRecord(ev[2 * used + 1], s);
        ++used;
        open_stage = -1;
    }
    void collect() {
        for (size_t k = 0; k < used; ++k) {
            cudaEventSynchronize(ev[2 * k + 1]);
            float m = 0.f;
            cudaEventElapsedTime(&m, ev[2 * k], ev[2 * k + 1]);
            ms[stage[k]] += m;
            cnt[stage[k]] += 1;
        }
        used = 0;
    }
    void reset() {
        collect();
        for (int i = 0; i < ST_N; ++i) {
            ms[i] = 0;
            cnt[i] = 0;
        }
    }
    ~StageProfiler() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

// A DG space of the hierarchy: degree, nodes per axis, 1D reference element
// and the degree whose penalty its facets use (the finest degree on every
// level of a gradual p-hierarchy, which makes each level the Galerkin product
// of the one above).
struct DGSpace {
    int p = 0, q = 0, penalty_p = 0;
    int64_t nloc = 0, ndof = 0;
    RefElem1D re;
    FDInput fdin{};          // input of the factor kernel (kept for recompute_block)
};

// A lower DG level of a gradual p-hierarchy (levels 1 .. L-1; level 0 is the
// finest, held in dgmg_ctx::d64 / d32): its operator data, its iterate,
// right-hand side and residual, and the interpolation up to the next finer level.
template <typename T>
struct DGLevelDev {
    DGDev<T> D;
    T *z = nullptr, *b = nullptr, *r = nullptr;
    DGInterp<T> P;
};

struct dgmg_ctx {
    int dim = 0, p = 0, q = 0;
    int n[3] = {1, 1, 1};
    int64_t ncell = 0, ndof = 0, nloc = 0;
    dgmg_opts opts;
    RefElem1D re;
    int cpb = 8;                                  // heuristic cells per CTA
    // cells per CTA in use, [FP64, FP32][TILE_PROJECT, TILE_SMOOTH, TILE_RESIDUAL];
    // 0 = the launcher's own choice (the one-thread-per-cell FP32 smoother where it applies)
    int tile[2][3] = {{8, 8, 8}, {8, 8, 8}};
    template <typename T>
    int tile_of(int stage) const {
        return tile[std::is_same<T, float>::value ? 1 : 0][stage];
    }
    std::vector<CGLevelHost> lv;
    int64_t ncoarse = 0;
    double *coarse_inv = nullptr;
    // the Q1 cycle as one cooperative launch (q1_blocks > 0): per precision its
    // plan and two barrier words; q1_blocks = 0 keeps the launch per step
    Q1Plan<double> *q1plan64 = nullptr;
    Q1Plan<float> *q1plan32 = nullptr;
    unsigned long long *q1bar = nullptr;          // arrival counters [FP64, FP32]
    int q1_blocks = 0;
    int q1_blocks_t[2] = {0, 0};                   // blocks of the cycle per precision [FP64, FP32]
    bool q1_wide = true;                           // FP32 cycle in 512-thread blocks
    DGDev<double> d64;
    DGDev<float> d32;
    std::vector<CGDev<double>> cg64;
    std::vector<CGDev<float>> cg32;
    // DG spaces of the hierarchy ([0] = finest); more than one with gradual
    // p-coarsening, whose lower levels live in lvl64 / lvl32 ([0] unused)
    std::vector<DGSpace> dgs;
    std::vector<DGLevelDev<double>> lvl64;
    std::vector<DGLevelDev<float>> lvl32;
    double *res64 = nullptr;                      // finest-level residual before its restriction
    float *res32 = nullptr;
    // work vectors
    float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *xs32 = nullptr, *rold32 = nullptr;
    double *w_r = nullptr, *w_z = nullptr, *w_p = nullptr, *w_q = nullptr, *w_rold = nullptr;
    double *w_b = nullptr, *w_x = nullptr;        // dgmg_solve_host staging
    double *scal = nullptr, *partials = nullptr;  // device scalars
    // the volume-term A/B entry (dgmg_volume_residual_f32), built at its first
    // call: E in the swizzled operand layout, and the shared 1D factors P | P^T | L
    float *vol_esw = nullptr;
    float vol_fac[165] = {};
    double *host_scal = nullptr;                  // pinned: S_NSCAL scalars, then the wait-counter snapshots
    // device addresses of the bounded-wait counters (FP32 and FP64 DG kernels,
    // Q1 grid barrier) on the ctx's device
    unsigned long long *tmo_dev[3] = {nullptr, nullptr, nullptr};
    double *quad_x1 = nullptr, *quad_V = nullptr, *quad_w = nullptr;
    std::vector<void *> allocs;
    size_t bytes = 0;
    StageProfiler prof;
    cudaEvent_t ev = nullptr;                     // completion of the scalars copied to host_scal
    cudaStream_t setup_stream = nullptr;          // allocations, uploads and frees of this ctx
    // CUDA graphs of the CG iteration chunks (captured on capture_stream at the
    // second use, replayed with one launch; not used while profiling)
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        const void *key = nullptr;                // user pointer the captured work depends on
        long long kernels = 0;                    // kernels inside (for the launch counter)
        int uses = 0;
        int q1_off = 0;                           // g_q1_one_launch_off when captured
    };
    Graph g_iter, g_body;
    cudaStream_t capture_stream = nullptr;
    bool use_graphs = true;

    // Device memory of the context: buffers are carved (256-byte aligned) out of
    // chunks of at least ARENA_CHUNK bytes, each one stream-ordered allocation
    // on the context's own stream (no device-wide synchronisation with solves
    // running on other streams); a buffer larger than a chunk gets its own.
    // A context makes a handful of allocation calls instead of one per buffer.
    // `bytes` counts the buffers themselves (what dgmg_estimate_bytes predicts).
    static constexpr size_t ARENA_CHUNK = 8u << 20, ARENA_ALIGN = 256;
    char *arena_ptr = nullptr;
    size_t arena_left = 0;
    template <typename T>
    int alloc(T **ptr, size_t count) {
        *ptr = nullptr;
        if (count == 0) count = 1;
        const size_t need = (count * sizeof(T) + ARENA_ALIGN - 1) / ARENA_ALIGN * ARENA_ALIGN;
        if (need > arena_left) {
            const size_t chunk = need > ARENA_CHUNK / 2 ? need : ARENA_CHUNK;
            void *p = nullptr;
            cudaError_t e = cudaMallocAsync(&p, chunk, setup_stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(DGMG_ENOMEM, std::string("cudaMalloc of ") + std::to_string(chunk) +
                                             " bytes failed: " + cudaGetErrorString(e));
            }
            allocs.push_back(p);
            if (chunk == need) {       // a buffer of its own; the open chunk stays open
                *ptr = reinterpret_cast<T *>(p);
                bytes += count * sizeof(T);
                return DGMG_OK;
            }
            arena_ptr = reinterpret_cast<char *>(p);
            arena_left = chunk;
        }
        *ptr = reinterpret_cast<T *>(arena_ptr);
        arena_ptr += need;
        arena_left -= need;
        bytes += count * sizeof(T);
        return DGMG_OK;
    }
    template <typename T>
    int upload(T **ptr, const std::vector<T> &h) {
        int rc = alloc(ptr, h.size());
        if (rc) return rc;
        if (!h.empty())
            DG_CUDA(cudaMemcpyAsync(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, setup_stream));
        return DGMG_OK;
    }
    ~dgmg_ctx() {
        for (Graph *g : {&g_iter, &g_body})
            if (g->exec) cudaGraphExecDestroy(g->exec);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        for (void *p : allocs) cudaFreeAsync(p, setup_stream);
        if (setup_stream) {
            cudaStreamSynchronize(setup_stream);
            cudaStreamDestroy(setup_stream);
        }
        if (host_scal) cudaFreeHost(host_scal);
        if (ev) cudaEventDestroy(ev);
    }
};

// slots of ctx->scal
enum { S_RZ = 0, S_PQ = 1, S_BETA = 2, S_RR = 3, S_RZN = 4, S_RZO = 5, S_BB = 6, S_ZZ = 7, S_ZZ0 = 8, S_XX = 9,
       S_NSCAL = 16 };
// pinned host slots after the scalars: wait-counter snapshots [start 3 | end 3]
enum { S_TMO = S_NSCAL, S_HOST = S_NSCAL + 6 };


#define RC(x)                           \
    do {                                \
        int rc_ = (x);                  \
        if (rc_ != DGMG_OK) return rc_; \
    } while (0)

#define LC(x)                                            \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
    } while (0)

namespace dgmg {

int check_ctx(const dgmg_ctx *C);
int exact_block(const dgmg_ctx &C);
// the level's per-cell factors when they factor the exact diagonal blocks A_KK
// (the one-thread-per-cell residual forms A_KK u from them), else null
template <typename T>
inline const T *exact_fd(const dgmg_ctx &C, const DGDev<T> &D) {
    return exact_block(C) ? D.fdr : nullptr;
}
// y = A u (b == NULL) or out = b - A u, FP64
int apply64(dgmg_ctx &C, const double *u, const double *b, double *out, cudaStream_t s);
// y = A u in FP32
int apply32(dgmg_ctx &C, const float *u, float *y, cudaStream_t s);
// z = V(r): FP64 interface (FP32 cycle inside in mixed precision)
int vcycle64(dgmg_ctx &C, const double *r, double *z, cudaStream_t s);
// z = V(r) on the DG level in precision T (zero initial guess)
template <typename T>
int dg_vcycle(dgmg_ctx &C, const T *r, T *z, cudaStream_t s);

// One solve as a non-blocking state machine (solver.cu). advance() queues the
// next stretch of device work on the run's stream and returns without waiting;
// it returns 1 once the solve has finished (status and stats final), 0 while it
// waits for device scalars or has more work to queue.
template <typename T>
inline std::vector<DGLevelDev<T>> &dglevels(dgmg_ctx &C) {
    if constexpr (std::is_same<T, float>::value)
        return C.lvl32;
    else
        return C.lvl64;
}

inline DGSpace finest_space(const dgmg_ctx &C) {
    DGSpace S;
    S.p = C.p;
    S.q = C.q;
    S.penalty_p = C.p;
    S.nloc = C.nloc;
    S.ndof = C.ndof;
    S.re = C.re;
    return S;
}

// the DG level and the Q1 levels of ctx in precision T
template <typename T>
inline DGDev<T> &dg(dgmg_ctx &C) {
    if constexpr (std::is_same<T, float>::value)
        return C.d32;
    else
        return C.d64;
}
template <typename T>
inline const DGDev<T> &dg(const dgmg_ctx &C) {
    if constexpr (std::is_same<T, float>::value)
        return C.d32;
    else
        return C.d64;
}
template <typename T>
inline Q1Plan<T> *&q1plan(dgmg_ctx &C) {
    if constexpr (std::is_same<T, float>::value)
        return C.q1plan32;
    else
        return C.q1plan64;
}
template <typename T>
inline std::vector<CGDev<T>> &cgl(dgmg_ctx &C) {
    if constexpr (std::is_same<T, float>::value)
        return C.cg32;
    else
        return C.cg64;
}
template <typename T>
inline const std::vector<CGDev<T>> &cgl(const dgmg_ctx &C) {
    if constexpr (std::is_same<T, float>::value)
        return C.cg32;
    else
        return C.cg64;
}

// dgmg_create with parts left out for contexts that only serve a batch:
// no solver workspace (work vectors, scalars, quadrature tables); no FP64
// block-inverse factors (the FP64 level only applies the operator); no FP64 Q1
// levels (the V-cycle runs in FP32). CREATE_SHARED_GPU (solve server): the Q1
// cycle's cooperative launch in 256-thread blocks, one per SM, which fit beside
// the kernels of concurrent solves.
enum { CREATE_NO_SOLVER = 1, CREATE_NO_FP64_SMOOTHER = 2, CREATE_NO_FP64_Q1 = 4, CREATE_SHARED_GPU = 8 };
int create_ctx(const dgmg_mesh *mesh, int p, const double *kappa, const dgmg_opts *opts, int flags, dgmg_ctx **out);

int mg_cycle64(dgmg_ctx &C, double *x, const double *b, double *r, cudaStream_t s);
int project64(dgmg_ctx &C, double *x, cudaStream_t s);

struct SolveRun {
    dgmg_ctx *C = nullptr;
    const double *b = nullptr;
    double *x = nullptr;
    cudaStream_t s = nullptr;
    int state = 0, it = 0, status = DGMG_OK, nres = 0;
    double bb = 0, bn = 1, rr = 0, relrec = 0, rel_true = 0, rnorm_upd = 0, zz0 = 0, zz = 0;
    bool need_accumulate = false;
    std::chrono::steady_clock::time_point t0;
    dgmg_stats stats{};
    void start(dgmg_ctx *ctx, const double *b_, double *x_, cudaStream_t s_);
    int advance(bool blocking);
    int pcg_chunk(bool update_dir, cudaStream_t st);
    int mg_chunk(cudaStream_t st);
    double dd1 = 0;                               // MGMult: ||x_1 - x_0||^2
    int reliable_chunk(bool update_dir, cudaStream_t st);
};

}  // namespace dgmg
