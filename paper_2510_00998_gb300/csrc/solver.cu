// The outer iterations of dgmg_solve as a non-blocking state machine:
//
//  * FP64 preconditioned CG (DGMG_OUTER_PCG): one FP64 apply per iteration, the
//    V-cycle (FP64 or FP32) as preconditioner, flexible Polak-Ribiere form when
//    the V-cycle runs in FP32.
//  * Reliable-update CG (DGMG_OUTER_RELIABLE, mixed precision): the
//    recurrences in FP32 (FP32 apply and V-cycle, dot products accumulated in
//    FP64), the solution accumulated in FP64, and the true residual b - A x
//    recomputed in FP64 whenever the FP32 residual has fallen by `delta`
//    since the last FP64 evaluation, and before stopping.
//
// Device work is queued on the run's stream; the scalars the host decides on
// (residual norms) come back through pinned memory and an event, so a
// scheduler can advance many runs on different streams without blocking.
#include <cmath>
#include <cstring>

#include "ctx.h"

namespace dgmg {

namespace {

// beta of the CG direction update (Fletcher-Reeves, or Polak-Ribiere for the
// flexible variant) and the shift of <r,z>, on the device
__global__ void k_scalar_beta(double *scal, int flexible) {
    const double rzn = scal[S_RZN];
    scal[S_BETA] = flexible ? (rzn - scal[S_RZO]) / scal[S_RZ] : rzn / scal[S_RZ];
    scal[S_RZ] = rzn;
}

int launch_beta(dgmg_ctx *C, int flexible, cudaStream_t s) {
    count_launches(1);
    k_scalar_beta<<<1, 1, 0, s>>>(C->scal, flexible);
    LC(cudaGetLastError());
    return DGMG_OK;
}

// queue the copy of the whole scalar block to pinned host memory + the event
int copy_scalars(dgmg_ctx *C, cudaStream_t s) {
    LC(cudaMemcpyAsync(C->host_scal, C->scal, sizeof(double) * S_NSCAL, cudaMemcpyDeviceToHost, s));
    return DGMG_OK;
}

int post_scalars(dgmg_ctx *C, cudaStream_t s) {
    RC(copy_scalars(C, s));
    LC(cudaEventRecord(C->ev, s));
    return DGMG_OK;
}

// Stream-ordered snapshot of the bounded-wait counters (FP32 and FP64 DG
// kernels, Q1 grid barrier) into pinned slot `at` (0 start, 1 end of a run).
int snapshot_timeouts(dgmg_ctx *C, int at, cudaStream_t s) {
    for (int k = 0; k < 3; ++k)
        LC(cudaMemcpyAsync(C->host_scal + S_TMO + 3 * at + k, C->tmo_dev[k], sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
    return DGMG_OK;
}

unsigned long long snapshot_value(const dgmg_ctx *C, int slot) {
    unsigned long long v;
    std::memcpy(&v, C->host_scal + S_TMO + slot, sizeof(v));
    return v;
}

// End of a run: the counters again (the stream is idle once the final
// scalars have arrived, so the wait is a few microseconds). A wait that ran
// out during the run makes it fail with DGMG_ETIMEOUT; a grid-barrier one
// also switches the process to the launch per step of the Q1 levels.
int check_timeouts(dgmg_ctx *C, cudaStream_t s) {
    RC(snapshot_timeouts(C, 1, s));
    LC(cudaStreamSynchronize(s));
    bool grew = false;
    for (int k = 0; k < 3; ++k) grew = grew || snapshot_value(C, 3 + k) != snapshot_value(C, k);
    if (!grew) return DGMG_OK;
    if (snapshot_value(C, 5) != snapshot_value(C, 2)) g_q1_one_launch_off.store(1);
    return fail(DGMG_ETIMEOUT,
                "a bounded device-side wait ran out during the solve (bulk-copy mbarrier or Q1 grid barrier); "
                "the result is not to be trusted");
}

// Queue the work of `enqueue(stream)` on s. With graphs enabled (and profiling
// off) the work is captured once into a CUDA graph at its second use and then
// replayed with a single launch; `key` is the user pointer the work depends
// on (a different key re-captures).
template <typename F>
int run_chunk(dgmg_ctx *C, dgmg_ctx::Graph &g, const void *key, cudaStream_t s, F enqueue) {
    if (!C->use_graphs || C->prof.on || g.uses++ == 0) return enqueue(s);
    const int q1_off = g_q1_one_launch_off.load();
    if (!g.exec || g.key != key || g.q1_off != q1_off) {
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        // A capture can be invalidated from outside (another thread of the
        // process synchronising the whole device while it runs): then nothing
        // was queued, so this ctx stops using graphs and queues the work eagerly.
        auto eager = [&]() {
            cudaGetLastError();
            C->use_graphs = false;
            return enqueue(s);
        };
        const long long before = g_kernel_launches.load();
        if (cudaStreamBeginCapture(C->capture_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return eager();
        const int rc = enqueue(C->capture_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(C->capture_stream, &graph);
        g.kernels = g_kernel_launches.load() - before;
        g_kernel_launches.fetch_sub(g.kernels);   // capturing launched nothing
        if (rc != DGMG_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (e == cudaErrorStreamCaptureInvalidated || e == cudaErrorStreamCaptureUnsupported ||
                e == cudaErrorStreamCaptureImplicit || (rc != DGMG_OK && e != cudaSuccess))
                return eager();
            if (rc != DGMG_OK) return rc;
            return cuda_fail(e, "cudaStreamEndCapture");
        }
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            g.exec = nullptr;
            return eager();
        }
        g.key = key;
        g.q1_off = q1_off;
    }
    LC(cudaGraphLaunch(g.exec, s));
    count_launches((int)g.kernels);
    return DGMG_OK;
}

// 1 if the posted scalars have arrived, 0 if not yet; <0 on error
int scalars_ready(dgmg_ctx *C, bool blocking) {
    cudaError_t e = blocking ? cudaEventSynchronize(C->ev) : cudaEventQuery(C->ev);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    return cuda_fail(e, "cudaEventQuery");
}

enum {
    P_START, P_WAITX, P_WAIT0, P_WAIT1, P_ITER, P_WAIT_RR, P_FINAL, P_WAIT_FINAL,   // FP64 PCG
    R_START, R_WAITX, R_WAIT0, R_ITER, R_WAIT_RR, R_WAIT_UPD, R_CONT, R_FINAL, R_WAIT_FIN,   // reliable updates
    M_START, M_WAIT0, M_ITER, M_WAIT,                                              // MGMult
    S_DONE
};

}  // namespace

// y = A u in FP32 (warm-up projection + cell equation on the FP32 hierarchy).
// The operator of the FP32 CG recurrences forms A_KK u in the direct
// sum-factorised form (one thread per cell where that kernel applies, no
// factors passed): forming it through the eigenbasis of the fast-diagonalisation
// factors, in FP32, cost the 64^3 p = 4 lognormal solve five more iterations
// (42 instead of 37); the V-cycle's residual, a preconditioner step, keeps the
// eigenbasis kernel, which is faster.
int apply32(dgmg_ctx &C, const float *u, float *y, cudaStream_t s) {
    DGDev<float> &D = C.d32;
    C.prof.begin(ST_PROJECT, s);
    LC(launch_project<float>(C.dim, C.q, D.c, C.tile[1][TILE_PROJECT], const_cast<float *>(u), nullptr, D.tr[0], s));
    C.prof.end(s);
    C.prof.begin(ST_RESIDUAL, s);
    LC(launch_residual<float>(C.dim, C.q, D.c, C.tile[1][TILE_RESIDUAL], RES_WRITE_R | RES_NEGATE, u, nullptr, D.kappa, D.tr[0], y,
                              nullptr, nullptr, s));
    C.prof.end(s);
    return DGMG_OK;
}

void SolveRun::start(dgmg_ctx *ctx, const double *b_, double *x_, cudaStream_t s_) {
    C = ctx;
    b = b_;
    x = x_;
    s = s_;
    it = 0;
    status = DGMG_OK;
    nres = 0;
    need_accumulate = false;
    zz0 = zz = 0;
    t0 = std::chrono::steady_clock::now();
    dd1 = 0;
    const int o = C->opts.outer;
    state = o == DGMG_OUTER_RELIABLE ? R_START : (o == DGMG_OUTER_MGMULT || o == DGMG_OUTER_MGMULT_PREC) ? M_START
                                                                                                          : P_START;
}

#define ADV_FAIL(code, msg)               \
    do {                                  \
        status = fail(code, msg);         \
        state = S_DONE;                   \
        return 1;                         \
    } while (0)

#define ADV(x)                            \
    do {                                  \
        int rc_ = (x);                    \
        if (rc_ != DGMG_OK) {             \
            status = rc_;                 \
            state = S_DONE;               \
            return 1;                     \
        }                                 \
    } while (0)

#define ADV_CUDA(x)                                          \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) ADV(cuda_fail(e_, #x));      \
    } while (0)

// One PCG iteration's device work: (when `update_dir`) z = V(r), beta, p = z + beta p;
// then q = A p, alpha, x += alpha p, r -= alpha q, ||r||^2, scalars to the host.
int SolveRun::pcg_chunk(bool update_dir, cudaStream_t st) {
    const int64_t n = C->ndof;
    const bool flexible = C->opts.precision == DGMG_MIXED_FP32;
    double *r = C->w_r, *z = C->w_z, *p = C->w_p, *q = C->w_q, *rold = C->w_rold;
    if (update_dir) {
        RC(vcycle64(*C, r, z, st));
        C->prof.begin(ST_VECTOR, st);
        if (flexible)
            LC(launch_dot2(n, r, z, rold, C->partials, C->scal + S_RZN, C->scal + S_RZO, st));
        else
            LC(launch_dot(n, r, z, C->partials, C->scal + S_RZN, st));
        RC(launch_beta(C, flexible ? 1 : 0, st));
        LC(launch_pcg_update_p(n, p, z, C->scal, st));
        C->prof.end(st);
    }
    RC(apply64(*C, p, nullptr, q, st));                         // q = A p
    C->prof.begin(ST_VECTOR, st);
    LC(launch_dot(n, p, q, C->partials, C->scal + S_PQ, st));
    if (flexible) LC(cudaMemcpyAsync(rold, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    LC(launch_pcg_update_xr(n, x, r, p, q, C->scal, st));      // alpha = rz / pq
    LC(launch_dot(n, r, r, C->partials, C->scal + S_RR, st));
    C->prof.end(st);
    return copy_scalars(C, st);
}

// One reliable-update CG iteration's FP32 work: (when `update_dir`) z = V(r),
// beta, p = z + beta p; then q = A p, alpha, xs += alpha p, r -= alpha q,
// ||r||^2, scalars to the host.
int SolveRun::reliable_chunk(bool update_dir, cudaStream_t st) {
    const int64_t n = C->ndof;
    float *r32 = C->r32, *z32 = C->z32, *p32 = C->p32, *q32 = C->q32, *xs = C->xs32, *rold32 = C->rold32;
    if (update_dir) {
        RC(dg_vcycle<float>(*C, r32, z32, st));
        C->prof.begin(ST_VECTOR, st);
        LC(launch_dot2f(n, r32, z32, rold32, C->partials, C->scal + S_RZN, C->scal + S_RZO, st));
        RC(launch_beta(C, 1, st));
        LC(launch_update_p_f(n, p32, z32, C->scal, st));
        C->prof.end(st);
    }
    RC(apply32(*C, p32, q32, st));
    C->prof.begin(ST_VECTOR, st);
    LC(launch_dotf(n, p32, q32, C->partials, C->scal + S_PQ, st));
    LC(launch_update_xr_dot_f(n, xs, r32, rold32, p32, q32, C->scal, C->partials, C->scal + S_RR, st));
    C->prof.end(st);
    return copy_scalars(C, st);
}

// One MGMult cycle's device work (Alg. 7): x_old = x, one cycle on A x = b (b
// copied to w_rold at the start, so the captured graph does not depend on the
// caller's b), r = b - A x, ||r||^2 and ||x - x_old||^2, scalars to the host.
int SolveRun::mg_chunk(cudaStream_t st) {
    const int64_t n = C->ndof;
    double *xold = C->w_p, *dx = C->w_q, *r = C->w_r, *bc = C->w_rold;
    C->prof.begin(ST_VECTOR, st);
    LC(cudaMemcpyAsync(xold, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    C->prof.end(st);
    RC(mg_cycle64(*C, x, bc, r, st));
    C->prof.begin(ST_VECTOR, st);
    LC(launch_dot(n, r, r, C->partials, C->scal + S_RR, st));
    LC(launch_sub(n, x, xold, dx, st));
    LC(launch_dot(n, dx, dx, C->partials, C->scal + S_ZZ, st));
    C->prof.end(st);
    return copy_scalars(C, st);
}

int SolveRun::advance(bool blocking) {
    const int64_t n = C->ndof;
    const double rtol = C->opts.rtol;
    double *r = C->w_r, *z = C->w_z, *p = C->w_p;
    float *r32 = C->r32, *z32 = C->z32, *p32 = C->p32, *xs = C->xs32;
    for (;;) {
        switch (state) {
            // ------------------------------------------------ FP64 PCG
            // The initial residual: r = b when the initial guess is zero (the
            // host reads ||x||^2 first), else the FP64 apply r = b - A x.
            case P_START:
            case R_START:
                ADV(snapshot_timeouts(C, 0, s));
                ADV_CUDA(launch_dot(n, b, b, C->partials, C->scal + S_BB, s));
                ADV_CUDA(launch_dot(n, x, x, C->partials, C->scal + S_XX, s));
                ADV(post_scalars(C, s));
                state = state == P_START ? P_WAITX : R_WAITX;
                break;
            case P_WAITX:
            case R_WAITX: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                if (C->host_scal[S_XX] == 0.0) {
                    C->prof.begin(ST_VECTOR, s);
                    ADV_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                    C->prof.end(s);
                } else {
                    ADV(apply64(*C, x, b, r, s));
                    ++nres;
                }
                C->prof.begin(ST_VECTOR, s);
                ADV_CUDA(launch_dot(n, r, r, C->partials, C->scal + S_RR, s));
                if (state == R_WAITX) ADV_CUDA(launch_cast_d2f(n, r, r32, s));
                C->prof.end(s);
                ADV(post_scalars(C, s));
                state = state == P_WAITX ? P_WAIT0 : R_WAIT0;
                break;
            }
            case P_WAIT0: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                bb = C->host_scal[S_BB];
                rr = C->host_scal[S_RR];
                if (!std::isfinite(bb)) ADV_FAIL(DGMG_ENONFINITE, "||b|| is not finite");
                if (!std::isfinite(rr)) ADV_FAIL(DGMG_ENONFINITE, "initial residual is not finite");
                bn = std::sqrt(bb) > 0 ? std::sqrt(bb) : 1.0;
                relrec = std::sqrt(rr) / bn;
                if (relrec <= rtol) {
                    state = P_FINAL;
                    break;
                }
                ADV(vcycle64(*C, r, z, s));
                ADV_CUDA(launch_dot(n, r, z, C->partials, C->scal + S_RZ, s));
                ADV_CUDA(launch_dot(n, z, z, C->partials, C->scal + S_ZZ0, s));
                ADV_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                it = 1;
                state = P_ITER;
                break;
            }
            case P_ITER:
                ADV(run_chunk(C, it == 1 ? C->g_iter : C->g_body, x, s, [&](cudaStream_t st) -> int {
                    return pcg_chunk(it > 1, st);
                }));
                ADV_CUDA(cudaEventRecord(C->ev, s));
                state = P_WAIT_RR;
                break;
            case P_WAIT_RR: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                rr = C->host_scal[S_RR];
                if (!std::isfinite(rr)) {
                    status = fail(DGMG_ENONFINITE, "residual norm is not finite");
                    state = P_FINAL;
                    break;
                }
                relrec = std::sqrt(rr) / bn;
                if (relrec <= rtol) {
                    state = P_FINAL;
                    break;
                }
                if (it >= C->opts.maxit) {
                    status = fail(DGMG_ENOTCONVERGED, "maxit reached");
                    state = P_FINAL;
                    break;
                }
                ++it;                                  // next chunk starts with V-cycle and direction update
                state = P_ITER;
                break;
            }
            case P_FINAL:
                ADV_CUDA(launch_dot(n, z, z, C->partials, C->scal + S_ZZ, s));
                ADV(apply64(*C, x, b, r, s));          // true residual of the returned x
                ++nres;
                ADV_CUDA(launch_dot(n, r, r, C->partials, C->scal + S_RR, s));
                ADV(post_scalars(C, s));
                state = P_WAIT_FINAL;
                break;
            case P_WAIT_FINAL: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                zz = C->host_scal[S_ZZ];
                zz0 = it > 0 ? C->host_scal[S_ZZ0] : 0.0;
                rel_true = std::sqrt(C->host_scal[S_RR]) / bn;
                stats.iterations = it;
                stats.rel_residual = rel_true;
                stats.rel_residual_recursive = relrec;
                stats.prec_residual = zz0 > 0 ? std::sqrt(zz / zz0) : 0.0;
                stats.fp64_applies = nres + it;
                stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                {
                    const int tr = check_timeouts(C, s);    // the root cause of any other failure
                    if (tr != DGMG_OK) status = tr;
                }
                state = S_DONE;
                return 1;
            }
            // ------------------------------------------------ reliable updates
            case R_WAIT0: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                bb = C->host_scal[S_BB];
                rr = C->host_scal[S_RR];
                if (!std::isfinite(bb)) ADV_FAIL(DGMG_ENONFINITE, "||b|| is not finite");
                if (!std::isfinite(rr)) ADV_FAIL(DGMG_ENONFINITE, "initial residual is not finite");
                bn = std::sqrt(bb) > 0 ? std::sqrt(bb) : 1.0;
                rel_true = relrec = std::sqrt(rr) / bn;
                rnorm_upd = std::sqrt(rr);
                if (rel_true <= rtol) {
                    state = R_FINAL;
                    break;
                }
                ADV_CUDA(cudaMemsetAsync(xs, 0, sizeof(float) * n, s));
                ADV(dg_vcycle<float>(*C, r32, z32, s));
                C->prof.begin(ST_VECTOR, s);
                ADV_CUDA(launch_dotf(n, r32, z32, C->partials, C->scal + S_RZ, s));
                ADV_CUDA(launch_dotf(n, z32, z32, C->partials, C->scal + S_ZZ0, s));
                ADV_CUDA(cudaMemcpyAsync(p32, z32, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
                C->prof.end(s);
                it = 1;
                state = R_ITER;
                break;
            }
            case R_ITER:
                ADV(run_chunk(C, it == 1 ? C->g_iter : C->g_body, nullptr, s, [&](cudaStream_t st) -> int {
                    return reliable_chunk(it > 1, st);
                }));
                ADV_CUDA(cudaEventRecord(C->ev, s));
                need_accumulate = true;
                state = R_WAIT_RR;
                break;
            case R_WAIT_RR: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                const double rr32 = C->host_scal[S_RR];
                if (!std::isfinite(rr32)) {
                    status = fail(DGMG_ENONFINITE, "residual norm is not finite");
                    state = R_FINAL;
                    break;
                }
                relrec = std::sqrt(rr32) / bn;
                if (relrec <= rtol || std::sqrt(rr32) < C->opts.delta * rnorm_upd) {
                    // reliable update: fold the FP32 correction into x, FP64 true residual
                    C->prof.begin(ST_VECTOR, s);
                    ADV_CUDA(launch_accumulate_f2d(n, x, xs, s));
                    C->prof.end(s);
                    need_accumulate = false;
                    ADV(apply64(*C, x, b, r, s));
                    ++nres;
                    C->prof.begin(ST_VECTOR, s);
                    ADV_CUDA(launch_dot(n, r, r, C->partials, C->scal + S_RR, s));
                    ADV_CUDA(launch_cast_d2f(n, r, r32, s));
                    C->prof.end(s);
                    ADV(post_scalars(C, s));
                    state = R_WAIT_UPD;
                    break;
                }
                state = R_CONT;
                break;
            }
            case R_WAIT_UPD: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                rr = C->host_scal[S_RR];
                if (!std::isfinite(rr)) {
                    status = fail(DGMG_ENONFINITE, "residual norm is not finite");
                    state = R_FINAL;
                    break;
                }
                rel_true = std::sqrt(rr) / bn;
                rnorm_upd = std::sqrt(rr);
                if (rel_true <= rtol) {
                    state = R_FINAL;
                    break;
                }
                state = R_CONT;
                break;
            }
            case R_CONT:
                if (it >= C->opts.maxit) {
                    status = fail(DGMG_ENOTCONVERGED, "maxit reached");
                    state = R_FINAL;
                    break;
                }
                ++it;                                  // next chunk starts with V-cycle and direction update
                state = R_ITER;
                break;
            case R_FINAL:
                if (need_accumulate) {
                    C->prof.begin(ST_VECTOR, s);
                    ADV_CUDA(launch_accumulate_f2d(n, x, xs, s));
                    C->prof.end(s);
                    need_accumulate = false;
                    ADV(apply64(*C, x, b, r, s));
                    ++nres;
                    ADV_CUDA(launch_dot(n, r, r, C->partials, C->scal + S_RR, s));
                }
                if (it > 0) ADV_CUDA(launch_dotf(n, z32, z32, C->partials, C->scal + S_ZZ, s));
                ADV(post_scalars(C, s));
                state = R_WAIT_FIN;
                break;
            case R_WAIT_FIN: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                rel_true = std::sqrt(C->host_scal[S_RR]) / bn;
                zz = it > 0 ? C->host_scal[S_ZZ] : 0.0;
                zz0 = it > 0 ? C->host_scal[S_ZZ0] : 0.0;
                stats.iterations = it;
                stats.rel_residual = rel_true;
                stats.rel_residual_recursive = relrec;
                stats.prec_residual = zz0 > 0 ? std::sqrt(zz / zz0) : 0.0;
                stats.fp64_applies = nres;
                stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                {
                    const int tr = check_timeouts(C, s);    // the root cause of any other failure
                    if (tr != DGMG_OK) status = tr;
                }
                state = S_DONE;
                return 1;
            }
            // ------------------------------------------------ MGMult (Alg. 7)
            case M_START:
                ADV(snapshot_timeouts(C, 0, s));
                ADV_CUDA(cudaMemcpyAsync(C->w_rold, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                ADV(project64(*C, x, s));              // projections of the initial guess
                ADV_CUDA(launch_dot(n, b, b, C->partials, C->scal + S_BB, s));
                ADV(post_scalars(C, s));
                state = M_WAIT0;
                break;
            case M_WAIT0: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                bb = C->host_scal[S_BB];
                if (!std::isfinite(bb)) ADV_FAIL(DGMG_ENONFINITE, "||b|| is not finite");
                bn = std::sqrt(bb) > 0 ? std::sqrt(bb) : 1.0;
                it = 0;
                state = M_ITER;
                break;
            }
            case M_ITER:
                ADV(run_chunk(C, C->g_body, x, s, [&](cudaStream_t st) -> int { return mg_chunk(st); }));
                ADV_CUDA(cudaEventRecord(C->ev, s));
                state = M_WAIT;
                break;
            case M_WAIT: {
                const int rdy = scalars_ready(C, blocking);
                if (rdy < 0) ADV(rdy);
                if (!rdy) return 0;
                ++it;
                rr = C->host_scal[S_RR];
                const double dd = C->host_scal[S_ZZ];
                if (it == 1) dd1 = dd;
                rel_true = relrec = std::sqrt(rr) / bn;
                const double prec = dd1 > 0 ? std::sqrt(dd / dd1) : 0.0;
                bool done = false;
                if (!std::isfinite(rr) || !std::isfinite(dd)) {
                    status = fail(DGMG_ENONFINITE, "residual norm is not finite");
                    done = true;
                } else if (C->opts.outer == DGMG_OUTER_MGMULT ? rel_true <= rtol : (it > 1 && prec <= rtol)) {
                    done = true;
                } else if (it >= C->opts.maxit) {
                    status = fail(DGMG_ENOTCONVERGED, "maxit reached");
                    done = true;
                }
                if (!done) {
                    state = M_ITER;
                    break;
                }
                stats.iterations = it;
                stats.rel_residual = rel_true;
                stats.rel_residual_recursive = relrec;
                stats.prec_residual = prec;
                stats.fp64_applies = 2 * it;
                stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                {
                    const int tr = check_timeouts(C, s);    // the root cause of any other failure
                    if (tr != DGMG_OK) status = tr;
                }
                state = S_DONE;
                return 1;
            }
            case S_DONE:
            default:
                return 1;
        }
    }
}

}  // namespace dgmg

extern "C" {

int dgmg_solve(dgmg_ctx *C, const double *b, double *x, dgmg_stats *stats, void *stream) {
    RC(check_ctx(C));
    if (!b || !x) return fail(DGMG_EINVAL, "b and x must not be NULL");
    if (b == x) return fail(DGMG_EINVAL, "b and x must not overlap");
    SolveRun run;
    run.start(C, b, x, (cudaStream_t)stream);
    while (!run.advance(true)) {
    }
    if (stats) *stats = run.stats;
    return run.status;
}

int dgmg_apply_f32(dgmg_ctx *C, const float *u, float *y, int form, void *stream) {
    RC(check_ctx(C));
    if (C->opts.precision != DGMG_MIXED_FP32) return fail(DGMG_EINVAL, "dgmg_apply_f32: needs a mixed-precision ctx");
    if (!u || !y) return fail(DGMG_EINVAL, "dgmg_apply_f32: NULL vector");
    if (u == y) return fail(DGMG_EINVAL, "dgmg_apply_f32: y must not alias u");
    if (form < 0 || form > 2) return fail(DGMG_EINVAL, "dgmg_apply_f32: form must be 0, 1 or 2");
    cudaStream_t s = (cudaStream_t)stream;
    if (form == 0) return dgmg::apply32(*C, u, y, s);
    DGDev<float> &D = C->d32;
    // form 2 forms A_KK u from the per-cell factors, which factor A_KK only with
    // exact blocks (with interior-only blocks they hold the interior cell's block)
    const float *fd = dgmg::exact_fd(*C, D);
    if (form == 2 && !fd) return fail(DGMG_EINVAL, "dgmg_apply_f32: form 2 needs exact per-cell blocks");
    C->prof.begin(ST_PROJECT, s);
    LC(dgmg::launch_project<float>(C->dim, C->q, D.c, C->tile[1][TILE_PROJECT], const_cast<float *>(u), nullptr,
                                   D.tr[0], s));
    C->prof.end(s);
    // form 1: the per-pencil kernel (a positive tile), form 2: one thread per
    // cell through the fast-diagonalisation factors
    const int tile = form == 1 ? std::max(1, 128 / (C->dim == 3 ? C->q * C->q : C->q)) : 0;
    C->prof.begin(ST_RESIDUAL, s);
    LC(dgmg::launch_residual<float>(C->dim, C->q, D.c, tile, dgmg::RES_WRITE_R | dgmg::RES_NEGATE, u, nullptr,
                                    D.kappa, D.tr[0], y, nullptr, form == 2 ? fd : nullptr, s));
    C->prof.end(s);
    return DGMG_OK;
}

int dgmg_solve_host(dgmg_ctx *C, const double *b_host, double *x_host, dgmg_stats *stats, void *stream) {
    RC(check_ctx(C));
    if (!b_host || !x_host) return fail(DGMG_EINVAL, "b_host and x_host must not be NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (!C->w_b) {
        RC(C->alloc(&C->w_b, C->ndof));
        RC(C->alloc(&C->w_x, C->ndof));
        LC(cudaStreamSynchronize(C->setup_stream));
    }
    const auto t0 = std::chrono::steady_clock::now();
    LC(cudaMemcpyAsync(C->w_b, b_host, sizeof(double) * C->ndof, cudaMemcpyHostToDevice, s));
    LC(cudaMemcpyAsync(C->w_x, x_host, sizeof(double) * C->ndof, cudaMemcpyHostToDevice, s));
    const int rc = dgmg_solve(C, C->w_b, C->w_x, stats, stream);
    if (rc != DGMG_OK && rc != DGMG_ENOTCONVERGED) return rc;
    LC(cudaMemcpyAsync(x_host, C->w_x, sizeof(double) * C->ndof, cudaMemcpyDeviceToHost, s));
    LC(cudaStreamSynchronize(s));
    if (stats) stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

}  // extern "C"
