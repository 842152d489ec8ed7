// Residual + p-restriction (the residual traversal of Alg. 6 with the
// restriction fused in, Sec. 5.1 "Restriction") that allocates nothing at call
// time; as an interface variant it has no counterpart in the paper.
//
// Who needs it: code that runs where device allocation is not allowed or not
// available -- real-time or embedded loops that forbid allocation after
// start-up, host applications that hand the library a fixed memory budget up
// front, and hosts without an allocator at the point of the call. Such callers still pass their own inputs and
// outputs; the only scratch the stage needs (2^d corner partial sums per
// cell) comes from the fixed array below, which every GPU that loads this
// library holds until the process exits.
#include <mutex>

#include "internal.h"

namespace {

// Maximum number of corner partial sums: 2^21 doubles = 16 MiB, enough for
// 262,144 hexahedra (a 64^3 mesh) or 524,288 quadrilaterals.
constexpr int64_t kCornerScratchMax = int64_t(1) << 21;
static __device__ __align__(256) double g_corner_scratch[kCornerScratchMax];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int dgmg_residual_restrict_noalloc(dgmg_ctx *ctx, const double *u, const double *b,
                                              const double *traces, double *r, double *rc, void *stream) {
    if (!ctx) return dgmg::fail(DGMG_EINVAL, "ctx is NULL");
    if (!u || !b || !traces) return dgmg::fail(DGMG_EINVAL, "u, b and traces must not be NULL");
    const int64_t need = dgmg::corner_scratch_count(ctx);
    if (need > kCornerScratchMax)
        return dgmg::fail(DGMG_EINVAL, "dgmg_residual_restrict_noalloc: mesh needs " + std::to_string(need) +
                                           " corner sums; the fixed scratch holds " +
                                           std::to_string(kCornerScratchMax));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dgmg::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return dgmg::fail(DGMG_EINVAL, "device ordinal out of range");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            // one-time set-up per device, with that device current: the device
            // address of the fixed array (its host-side name is not one)
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_corner_scratch);
            if (e != cudaSuccess) return dgmg::cuda_fail(e, "cudaGetSymbolAddress(g_corner_scratch)");
            g_scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    return dgmg::residual_restrict_with_scratch(ctx, u, b, traces, r, rc, scratch, (cudaStream_t)stream);
}
