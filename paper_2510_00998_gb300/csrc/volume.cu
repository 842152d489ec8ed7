// The volume term of the SIPG operator on its own, r = b - kappa_K E u_K for
// every cell (E: the unit-coefficient element stiffness matrix, the cell
// integral of Eq. weak_form_IP, shared by all cells of a uniform mesh), 3D,
// q = 5 (p = 4), FP32 vectors: two implementations of the same contraction, to
// measure whether the cell GEMM belongs on the tensor cores.
//
//  * Tensor cores (tcgen05, TF32 operands, FP32 accumulation in tensor memory):
//    D = U E^T for tiles of 128 cells (M = 128, N = K = 128: 125 nodes padded),
//    E resident in shared memory in the 128-byte swizzled K-major layout; one
//    persistent CTA per SM; the u tile arrives by a bulk copy and is laid out
//    (rounded to TF32) by the CTA's threads; 16 MMAs of K = 8 per tile, issued
//    by one thread, completion through tcgen05.commit on an mbarrier; the
//    epilogue reads its row of the accumulator with tcgen05.ld (warp w owns
//    TMEM lanes 32w..32w+31, i.e. cells 32w..32w+31 of the tile).
//  * Sum factorisation on the CUDA cores (FP32, one thread per cell): with the
//    generalised eigenvectors of the 1D pair, K_a V_a = M_a V_a L_a and
//    V_a^T M_a V_a = I, every 1D operator factors as K_a = P_a^T L_a P_a,
//    M_a = P_a^T P_a with P_a = V_a^T M_a, so E = (P^T)^(x3) (L_x + L_y + L_z)
//    P^(x3): six passes of q x q matrices shared by every cell.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "dg_kernels.cuh"

namespace dgmg {
namespace {

constexpr int VQ = 5, VNL = VQ * VQ * VQ;      // nodes per axis, per cell
constexpr int KP = 128;                        // K and N padded to 128
constexpr int TM = 128;                        // cells per tile (MMA M)
constexpr int TMEM_COLS = 128;                 // FP32 accumulator columns (N)
constexpr uint32_t KBLOCK = TM * 128;          // bytes of one 32-element K block of a 128-row operand
constexpr uint32_t OPERAND_BYTES = 4 * KBLOCK; // 64 KB per 128 x 128 TF32 operand
constexpr uint32_t STAGE_BYTES = TM * VNL * 4; // raw tile of 128 cells (64,000 bytes)
constexpr size_t TC_SMEM = 2 * OPERAND_BYTES + STAGE_BYTES + 64 + 1024;   // + barriers, TMEM slot, alignment

// Byte offset of element (row, k) of a 128-row K-major operand in the 128-byte
// swizzled layout: K in blocks of 32 elements (128 bytes); in a block, 8-row
// groups of 1024 bytes, row r at 128 (r mod 8) within its group, its 16-byte
// chunk c stored at chunk position c xor (r mod 8).
__host__ __device__ inline uint32_t sw128_offset(int row, int k) {
    return (uint32_t)(k >> 5) * KBLOCK + (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u +
           ((uint32_t)(((k & 31) >> 2) ^ (row & 7)) << 4) + (uint32_t)(k & 3) * 4u;
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzled
// layout: start address / 16 (bits 0-13), leading byte offset 16 / 16 (bits
// 16-29; not used by this layout), stride byte offset 1024 / 16 between 8-row
// groups (bits 32-45), descriptor version 1 (bits 46-47), base offset 0
// (the blocks are 1024-byte aligned), swizzle mode 2 = 128 bytes (bits 61-63).
__device__ inline uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of tcgen05.mma kind::tf32: D in FP32 (bits 4-5 = 1),
// A and B TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N / 8
// (bits 17-22), M / 16 (bits 24-28).
constexpr uint32_t IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(KP >> 3) << 17) |
                                ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(IDESC_TF32), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of the calling thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t *v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Bounded wait on phase `parity` of `bar` by every calling thread; a wait that
// runs out is counted and reported false.
__device__ __forceinline__ bool wait_all(uint64_t *bar, unsigned parity) {
    if (mbar_wait_bounded(bar, parity)) return true;
    atomicAdd(&g_wait_timeouts, 1ull);
    return false;
}

// r = b - kappa E u on the tensor cores. Esw: E (N = 128 rows of K = 128,
// zero-padded) in the swizzled layout above, 64 KB. One CTA of 128 threads per
// SM strides over the tiles of 128 cells.
__global__ void __launch_bounds__(128, 1) k_volume_tc(const float *__restrict__ Esw, const float *__restrict__ u,
                                                      const float *__restrict__ b, const double *__restrict__ kappa,
                                                      float *__restrict__ r, int64_t ncell) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned base (the swizzle atoms need it)
    const uint32_t raw = smem_addr(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    unsigned char *sB = base;                                  // E, resident
    unsigned char *sA = base + OPERAND_BYTES;                  // u tile, swizzled TF32
    float *stage = reinterpret_cast<float *>(base + 2 * OPERAND_BYTES);   // raw u, then b, then r
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + 2 * OPERAND_BYTES + STAGE_BYTES);   // E, u, b, mma
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], OPERAND_BYTES);
        bulk_load(sB, Esw, OPERAND_BYTES, &bars[0]);
    }
    const int64_t ntiles = (ncell + TM - 1) / TM;
    unsigned ph_copy = 0, ph_mma = 0;
    bool ok = true, e_ready = false;
    const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t c0 = tile * TM;
        const int nc = (int)min((int64_t)TM, ncell - c0);
        const bool full = nc == TM;
        // u of the tile into the stage
        if (full) {
            if (tid == 0) {
                mbar_arrive_expect_tx(&bars[1], STAGE_BYTES);
                bulk_load(stage, u + c0 * VNL, STAGE_BYTES, &bars[1]);
            }
            ok = wait_all(&bars[1], ph_copy) && ok;
        } else {
            for (int e = tid; e < nc * VNL; e += TM) stage[e] = u[c0 * VNL + e];
        }
        ok = __syncthreads_and(ok) != 0;
        // row tid of the A operand: u rounded to TF32, zero beyond the cell's nodes
        // and beyond the tile's cells
        {
            const int row = tid;
            const float *src = stage + row * VNL;
#pragma unroll 4
            for (int ch = 0; ch < KP / 4; ++ch) {
                float4 v;
                const int k = 4 * ch;
                v.x = (row < nc && k + 0 < VNL) ? to_tf32(src[k + 0]) : 0.f;
                v.y = (row < nc && k + 1 < VNL) ? to_tf32(src[k + 1]) : 0.f;
                v.z = (row < nc && k + 2 < VNL) ? to_tf32(src[k + 2]) : 0.f;
                v.w = (row < nc && k + 3 < VNL) ? to_tf32(src[k + 3]) : 0.f;
                *reinterpret_cast<float4 *>(sA + sw128_offset(row, k)) = v;
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        // b of the tile into the stage (the raw u is consumed)
        if (full) {
            if (tid == 0) {
                mbar_arrive_expect_tx(&bars[2], STAGE_BYTES);
                bulk_load(stage, b + c0 * VNL, STAGE_BYTES, &bars[2]);
            }
        } else {
            for (int e = tid; e < nc * VNL; e += TM) stage[e] = b[c0 * VNL + e];
        }
        // D = U E^T: 16 MMAs of K = 8, one thread
        if (!e_ready) {                        // E resident (every thread waits once)
            ok = wait_all(&bars[0], 0) && ok;
            e_ready = true;
        }
        if (tid == 0 && ok) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < KP / 8; ++s) {
                const uint32_t off = (uint32_t)(s >> 2) * KBLOCK + (uint32_t)(s & 3) * 32u;
                tc_mma_tf32(tmem, sw128_desc(a0 + off), sw128_desc(b0 + off), s > 0 ? 1u : 0u);
            }
            tc_commit(&bars[3]);
        }
        ok = wait_all(&bars[3], ph_mma) && ok;
        if (full) ok = wait_all(&bars[2], ph_copy) && ok;
        ok = __syncthreads_and(ok) != 0;   // the same outcome in every thread
        tc_fence_after();
        // epilogue: this thread's cell (TMEM lane tid), r = b - kappa (E u)
        {
            uint32_t acc[KP];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
            for (int j = 0; j < KP / 32; ++j) tc_ld32(taddr + 32u * j, acc + 32 * j);
            tc_wait_ld();
            const int row = tid;
            if (row < nc) {
                const float kK = (float)kappa[c0 + row];
                float *dst = stage + row * VNL;
#pragma unroll
                for (int k = 0; k < VNL; ++k) dst[k] = dst[k] - kK * __uint_as_float(acc[k]);
            }
        }
        tc_fence_before();
        fence_proxy_async_smem();
        __syncthreads();
        if (full) {
            if (tid == 0) {
                bulk_store(r + c0 * VNL, stage, STAGE_BYTES);
                bulk_commit();
                bulk_wait_read_all();
            }
        } else {
            for (int e = tid; e < nc * VNL; e += TM) r[c0 * VNL + e] = stage[e];
        }
        __syncthreads();
        ph_copy ^= full ? 1u : 0u;
        ph_mma ^= 1u;
    }
    if (!e_ready) wait_all(&bars[0], 0);   // E must land before the CTA ends
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Shared 1D factors of the sum-factorised form: P_a = V_a^T M_a (row-major),
// its transpose, and L_a, per axis.
struct VolConst {
    float P[3][VQ * VQ], Pt[3][VQ * VQ], L[3][VQ];
    int64_t ncell;
};

// r = b - kappa E u with one thread per cell (FP32): six passes of the shared
// factors (P along x, y, z; the eigenvalue sums; P^T along x, y, z). A CTA is
// one warp serving 32 consecutive cells; u and b arrive by bulk copies, r
// leaves by a bulk store (plain copies for the last, partial block).
__global__ void __launch_bounds__(32) k_volume_sf(const __grid_constant__ VolConst vc, const float *__restrict__ u,
                                                  const float *__restrict__ b, const double *__restrict__ kappa,
                                                  float *__restrict__ r) {
    constexpr int W = 32;
    __shared__ __align__(128) float sU[W * VNL];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ float sP[3][VQ * VQ], sPt[3][VQ * VQ], sL[3][VQ];
    const int lane = threadIdx.x;
    const int64_t cell0 = (int64_t)blockIdx.x * W;
    const int ncl = (int)min((int64_t)W, vc.ncell - cell0);
    const bool full = ncl == W, active = lane < ncl;
    cells_init_bars(bars, 2, lane, false);
    for (int e = lane; e < 3 * VQ * VQ; e += W) {
        sP[e / (VQ * VQ)][e % (VQ * VQ)] = vc.P[e / (VQ * VQ)][e % (VQ * VQ)];
        sPt[e / (VQ * VQ)][e % (VQ * VQ)] = vc.Pt[e / (VQ * VQ)][e % (VQ * VQ)];
    }
    for (int e = lane; e < 3 * VQ; e += W) sL[e / VQ][e % VQ] = vc.L[e / VQ][e % VQ];
    stage_bulk<float>(full, lane, &bars[0], sU, u + cell0 * VNL, W * VNL, ncl * VNL);
    bool ok = true;
    if (full)
        ok = warp_wait_copies(&bars[0], lane) && ok;
    else
        __syncwarp();
    float R[VNL];
#pragma unroll
    for (int e = 0; e < VNL; ++e) R[e] = active ? sU[lane * VNL + e] : 0.f;
    fence_proxy_async_smem();
    __syncwarp();
    stage_bulk<float>(full, lane, &bars[1], sU, b + cell0 * VNL, W * VNL, ncl * VNL);
    if (active) {
#pragma unroll 1
        for (int ax = 0; ax < 3; ++ax) {           // P along x, y, z
            float S[VQ * VQ];
#pragma unroll
            for (int e = 0; e < VQ * VQ; ++e) S[e] = sP[ax][e];
            pass_x<float, VQ>(S, R);
            rotate<float, VQ>(R);
        }
#pragma unroll
        for (int kz = 0; kz < VQ; ++kz) {          // the eigenvalue sums
            const float lz = sL[2][kz];
#pragma unroll
            for (int j = 0; j < VQ; ++j) {
                const float lyz = sL[1][j] + lz;
#pragma unroll
                for (int i = 0; i < VQ; ++i) R[i + VQ * (j + VQ * kz)] *= sL[0][i] + lyz;
            }
        }
#pragma unroll 1
        for (int ax = 0; ax < 3; ++ax) {           // P^T along x, y, z
            float S[VQ * VQ];
#pragma unroll
            for (int e = 0; e < VQ * VQ; ++e) S[e] = sPt[ax][e];
            pass_x<float, VQ>(S, R);
            rotate<float, VQ>(R);
        }
    }
    if (full)
        ok = warp_wait_copies(&bars[1], lane) && ok;
    else
        __syncwarp();
    if (active) {
        const float kK = (float)kappa[cell0 + lane];
        float *row = sU + lane * VNL;
#pragma unroll
        for (int e = 0; e < VNL; ++e) row[e] = row[e] - kK * R[e];
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (ok) {
        if (full) {
            if (lane == 0) {
                bulk_store(r + cell0 * VNL, sU, (unsigned)(W * VNL * sizeof(float)));
                bulk_commit();
            }
        } else {
            for (int e = lane; e < ncl * VNL; e += W) r[cell0 * VNL + e] = sU[e];
        }
    }
    bulk_wait_read_all();
}

// symmetric eigenproblem by cyclic Jacobi rotations (n small), A overwritten
// by its eigenvalues on the diagonal, V the eigenvectors (columns)
void jacobi_eigen(int n, std::vector<double> &A, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

// The ctx's shared data of both forms, built at its first call (kept in the
// ctx, freed with it): E swizzled on the device, the sum-factorised factors.
int vol_setup(dgmg_ctx &C, cudaStream_t s) {
    const DGConst<double> &c = C.d64.c;
    const int q = VQ;
    // E[n][k] = sum_a (K_a along a, M_b along the others), node i + q j + q^2 k
    std::vector<float> Esw(OPERAND_BYTES / 4, 0.f);
    for (int n = 0; n < VNL; ++n)
        for (int k = 0; k < VNL; ++k) {
            const int ni[3] = {n % q, (n / q) % q, n / (q * q)}, ki[3] = {k % q, (k / q) % q, k / (q * q)};
            double e = 0.0;
            for (int a = 0; a < 3; ++a) {
                double t = 1.0;
                for (int d = 0; d < 3; ++d) t *= (d == a ? c.K[d] : c.M[d])[ni[d] * q + ki[d]];
                e += t;
            }
            // TF32 (round to nearest, ties away: 10 mantissa bits kept)
            float f = (float)e;
            uint32_t bits;
            std::memcpy(&bits, &f, 4);
            bits = (bits + 0x1000u) & ~0x1FFFu;
            std::memcpy(&f, &bits, 4);
            Esw[sw128_offset(n, k) / 4] = f;
        }
    RC(C.upload(&C.vol_esw, Esw));
    // generalised eigenvectors per axis: M = L L^T, L^-1 K L^-T = Q Lam Q^T, V = L^-T Q
    for (int a = 0; a < 3; ++a) {
        std::vector<double> Mm(c.M[a], c.M[a] + q * q), Km(c.K[a], c.K[a] + q * q), Li(q * q);
        if (!cholesky_inverse_lower(q, Mm.data(), Li.data())) return fail(DGMG_EINVAL, "mass not SPD");
        std::vector<double> A(q * q, 0.0), Qv;
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                double sum = 0.0;
                for (int k = 0; k < q; ++k)
                    for (int l = 0; l < q; ++l) sum += Li[i * q + k] * Km[k * q + l] * Li[j * q + l];
                A[i * q + j] = sum;
            }
        jacobi_eigen(q, A, Qv);
        std::vector<double> Vm(q * q, 0.0);   // V = L^-T Q
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                double sum = 0.0;
                for (int k = 0; k < q; ++k) sum += Li[k * q + i] * Qv[k * q + j];
                Vm[i * q + j] = sum;
            }
        for (int m = 0; m < q; ++m) {
            C.vol_fac[150 + a * q + m] = (float)A[m * q + m];                 // L
            for (int n = 0; n < q; ++n) {
                double p = 0.0;   // P = V^T M
                for (int k = 0; k < q; ++k) p += Vm[k * q + m] * Mm[k * q + n];
                C.vol_fac[a * q * q + m * q + n] = (float)p;                  // P
                C.vol_fac[75 + a * q * q + n * q + m] = (float)p;             // P^T
            }
        }
    }
    DG_CUDA(cudaStreamSynchronize(C.setup_stream));
    (void)s;
    return DGMG_OK;
}

}  // namespace

cudaError_t wait_timeouts_volume(unsigned long long *count) { return read_wait_timeouts(count); }

}  // namespace dgmg

extern "C" int dgmg_volume_residual_f32(dgmg_ctx *C, const float *u, const float *b, float *r, int method,
                                        void *stream) {
    using namespace dgmg;
    RC(check_ctx(C));
    if (C->dim != 3 || C->q != VQ) return fail(DGMG_EINVAL, "dgmg_volume_residual_f32: 3D, p = 4 only");
    if (!u || !b || !r) return fail(DGMG_EINVAL, "dgmg_volume_residual_f32: NULL vector");
    if (method != 0 && method != 1) return fail(DGMG_EINVAL, "dgmg_volume_residual_f32: method must be 0 or 1");
    if (((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(r)) & 15) != 0)
        return fail(DGMG_EINVAL, "dgmg_volume_residual_f32: vectors must be 16-byte aligned");
    if (u == r || b == r) return fail(DGMG_EINVAL, "dgmg_volume_residual_f32: r must not alias u or b");
    cudaStream_t s = (cudaStream_t)stream;
    if (!C->vol_esw) RC(vol_setup(*C, s));
    if (C->ncell == 0) return DGMG_OK;
    if (method == 0) {
        VolConst vc;
        std::memcpy(vc.P, C->vol_fac, sizeof(vc.P));
        std::memcpy(vc.Pt, C->vol_fac + 75, sizeof(vc.Pt));
        std::memcpy(vc.L, C->vol_fac + 150, sizeof(vc.L));
        vc.ncell = C->ncell;
        const int64_t grid = (C->ncell + 31) / 32;
        count_launches(1);
        k_volume_sf<<<(unsigned)grid, 32, 0, s>>>(vc, u, b, C->d64.kappa, r);
        LC(cudaGetLastError());
        return DGMG_OK;
    }
    static bool attr = false;
    if (!attr) {
        LC(cudaFuncSetAttribute(k_volume_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        attr = true;
    }
    int dev = 0, sms = 0;
    LC(cudaGetDevice(&dev));
    LC(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t ntiles = (C->ncell + TM - 1) / TM;
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sms);
    count_launches(1);
    k_volume_tc<<<grid, TM, TC_SMEM, s>>>(C->vol_esw, u, b, C->d64.kappa, r, C->ncell);
    LC(cudaGetLastError());
    return DGMG_OK;
}
