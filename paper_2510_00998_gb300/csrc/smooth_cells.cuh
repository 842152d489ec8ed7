// Single-touch smoothing step (Algorithm 4, exact diagonal blocks) with one
// thread per cell, 3D: FP32 for q <= 5, FP64 for q <= 4 nodes per axis.
//
// Each thread keeps its whole cell (q^3 values) in registers, so the six
// tensor passes of the fast-diagonalisation inverse need no transposes through
// shared memory. A CTA is one warp serving 32 consecutive cells. Its inputs are
// staged in shared memory in the order they are consumed:
//   - b and the fast-diagonalisation factors: one bulk (TMA) copy each,
//     completing on an mbarrier;
//   - the neighbours' traces, face by face through two slots: every lane
//     fetches its neighbour's face with one bulk copy (faces are padded to
//     16 bytes in the trace buffers), the copies of a face completing on one
//     mbarrier whose byte count lane 0 posts;
//   - FP32: u of the previous iterate by a bulk copy into the slot area once
//     the faces are consumed, overlapping the inverse;
//   - FP64: the per-node table of inverse eigenvalue sums into the slot area
//     once the faces are consumed (FP64 division is a long sequence on the
//     FP64 pipe, which bounds the FP64 kernel), then u of the previous iterate
//     into the same area once the table is used, overlapping the last passes.
// The new u leaves through a bulk store; every lane writes its new traces into
// its face slots and stores each face with one bulk store. A lane reads its own cell with stride q^3 (odd for odd
// q, so a warp's 32 loads hit 32 banks).
//
// The split update of the exact block (u <- (1 - w) u + w A_KK^{-1}(b - N u_nb))
// needs only the neighbours' traces and b before the inverse, so u itself is
// read once, at the end.
#pragma once

#include <cstdint>

namespace dgmg {

// Waits in the kernels below that gave up (an mbarrier phase that did not
// complete within the iteration limit). Zero in every healthy run.
static __device__ unsigned long long g_wait_timeouts;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile(
        "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait on phase `parity`; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
    for (int it = 0; it < (1 << 20); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
// Set up the CTA's mbarriers (lane 0). `reuse`: a persistent CTA's next work
// item; every phase of the previous item has completed, so the objects are
// invalidated first, and every lane's accesses of the staging areas are
// ordered before the bulk copies of the new item.
__device__ __forceinline__ void cells_init_bars(uint64_t *bars, int count, int lane, bool reuse) {
    if (reuse) fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
        for (int i = 0; i < count; ++i) {
            if (reuse) mbar_inval(&bars[i]);
            mbar_init(&bars[i], 1);
        }
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncwarp();
}

// Lane 0 waits for phase `parity` of `bar`; the outcome is shared with the
// warp. A wait that runs out is counted, then waited for once more (the copies
// must land before the CTA's shared memory is released).
__device__ __forceinline__ bool warp_wait_phase(uint64_t *bar, unsigned parity, int lane) {
    int ok = 1;
    if (lane == 0) {
        if (!mbar_wait_bounded(bar, parity)) {
            atomicAdd(&g_wait_timeouts, 1ull);
            mbar_wait_bounded(bar, parity);
            ok = 0;
        }
    }
    __syncwarp();
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
__device__ __forceinline__ bool warp_wait_copies(uint64_t *bar, int lane) { return warp_wait_phase(bar, 0, lane); }

// Cell coordinates with 32-bit division (the one-thread-per-cell kernels run on
// meshes of fewer than 2^31 cells; the launchers check).
__device__ __forceinline__ void cell_coords32(int64_t cell, const int *n, int *ci) {
    const unsigned c = (unsigned)cell, n0 = (unsigned)n[0], n1 = (unsigned)n[1];
    const unsigned r = c / n0;
    ci[0] = (int)(c - r * n0);
    ci[1] = (int)(r % n1);
    ci[2] = (int)(r / n1);
}

template <typename T, int Q>
struct CellGeo {
    static constexpr int NL = Q * Q * Q, NF = Q * Q, FDS = Q * Q + Q;
    static constexpr int FS = trace_face_stride<T>(NF), TR = 6 * FS;   // trace values per face / cell
    static constexpr int W = 32;                       // cells per CTA (one per lane)
    // FP64 (LEAN): the kernel is bound by the FP64 pipe, not by memory, so the
    // neighbour faces, the table and the previous u are read straight from
    // global memory by each lane and the traces written the same way; only
    // area A is staged. That halves the shared memory per CTA, so more CTAs
    // are resident (a 32^3 mesh fits in one wave).
    static constexpr bool LEAN = sizeof(T) == 8;
    // shared memory (values of T), per cell. FP32 smoothing step: area A holds
    // b, then one neighbour-face slot (FS values) during the facet lifting, then
    // the previous u, then the new u, then one slot of new traces; area B holds
    // the other face slot, then the factors, then the other trace slot (8
    // one-warp CTAs fit per SM). FP64: area A holds b, then the factors, then the
    // new u.
    static constexpr int PA = LEAN ? (NL > 3 * FDS ? NL : 3 * FDS) : NL;
    static constexpr int PB = LEAN ? 0 : (FS > 3 * FDS ? FS : 3 * FDS);
    static constexpr size_t OFF_B = (size_t)W * PA;
    static constexpr size_t BYTES = (OFF_B + (size_t)W * PB) * sizeof(T);
    static_assert(LEAN || FS <= NL, "a face slot fits area A");
};

// Neighbour across face f (= 2 axis + side) of `cell`, -1 where face f is on the
// boundary (bit f of mask clear); s1, s2: the cell strides along y and z.
__device__ __forceinline__ int cell_neighbour(int f, int mask, int64_t cell, int s1, int s2) {
    if (!(mask & (1 << f))) return -1;
    const int s = f < 2 ? 1 : (f < 4 ? s1 : s2);
    return (int)cell + ((f & 1) ? s : -s);
}


// Stage face f of the lane's neighbour nb (the neighbour's face f^1) into the
// lane's part of a face slot: one bulk copy per lane that has a neighbour, all
// completing on `bar`, whose byte count lane 0 posts before any copy is issued.
// The caller has ended every read of the slot (proxy fence and warp barrier).
template <typename T, int Q>
__device__ __forceinline__ void stage_face(int f, int nb, int lane, const T *__restrict__ tr, T *slot, uint64_t *bar) {
    using G = CellGeo<T, Q>;
    const unsigned with = __ballot_sync(0xffffffffu, nb >= 0);
    if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)(__popc(with) * G::FS * (int)sizeof(T)));
    __syncwarp();
    if (nb >= 0)
        bulk_load(slot + lane * G::FS, tr + (int64_t)nb * G::TR + (f ^ 1) * G::FS, (unsigned)(G::FS * sizeof(T)), bar);
}

// The cell tensor R[x + q y + q^2 z] is kept in registers and only ever worked
// on along its first index; the other axes are brought there by rotating the
// tensor (one code path for all three axes, which keeps the kernel small
// enough for the instruction cache).
// rotate: new (x, y, z) = old (y, z, x).
template <typename T, int Q>
__device__ __forceinline__ void rotate(T *R) {
    T tmp[Q * Q * Q];
#pragma unroll
    for (int e = 0; e < Q * Q * Q; ++e) tmp[e] = R[e];
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
        for (int j = 0; j < Q; ++j)
#pragma unroll
            for (int i = 0; i < Q; ++i) R[j + Q * k + Q * Q * i] = tmp[i + Q * j + Q * Q * k];
}
// rotate_back: new (x, y, z) = old (z, x, y).
template <typename T, int Q>
__device__ __forceinline__ void rotate_back(T *R) {
    T tmp[Q * Q * Q];
#pragma unroll
    for (int e = 0; e < Q * Q * Q; ++e) tmp[e] = R[e];
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
        for (int j = 0; j < Q; ++j)
#pragma unroll
            for (int i = 0; i < Q; ++i) R[k + Q * i + Q * Q * j] = tmp[i + Q * j + Q * Q * k];
}

// Load a q x q matrix (row-major in shared memory) into registers, transposed if asked.
template <typename T, int Q, bool TRANSPOSE>
__device__ __forceinline__ void load_matrix(const T *src, T *S) {
    T v[Q * Q];
    if (sizeof(T) == 4) {                               // 8-byte loads (the matrix is 8-byte aligned)
#pragma unroll
        for (int e = 0; e < (Q * Q) / 2; ++e) {
            const float2 w = reinterpret_cast<const float2 *>(src)[e];
            v[2 * e] = (T)w.x;
            v[2 * e + 1] = (T)w.y;
        }
        if ((Q * Q) & 1) v[Q * Q - 1] = src[Q * Q - 1];
    } else {
#pragma unroll
        for (int e = 0; e < Q * Q; ++e) v[e] = src[e];
    }
#pragma unroll
    for (int m = 0; m < Q; ++m)
#pragma unroll
        for (int n = 0; n < Q; ++n) S[m * Q + n] = TRANSPOSE ? v[n * Q + m] : v[m * Q + n];
}

// Along x with packed pairs of pencils (FP32): outputs of pencils t and t + 1 by
// one two-lane FMA per term, the matrix entry duplicated in both lanes (the
// same roundings as the scalar form, half the issue slots).
template <int Q>
__device__ __forceinline__ void pass_x2(const float *A, float *R) {
#pragma unroll
    for (int t = 0; t + 1 < Q * Q; t += 2) {
        float2 x[Q];
#pragma unroll
        for (int n = 0; n < Q; ++n) x[n] = make_float2(R[n + Q * t], R[n + Q * (t + 1)]);
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            float2 s = __fmul2_rn(make_float2(A[m * Q], A[m * Q]), x[0]);
#pragma unroll
            for (int n = 1; n < Q; ++n) s = __ffma2_rn(make_float2(A[m * Q + n], A[m * Q + n]), x[n], s);
            R[m + Q * t] = s.x;
            R[m + Q * (t + 1)] = s.y;
        }
    }
    if ((Q * Q) & 1) {
        constexpr int t = Q * Q - 1;
        float x[Q];
#pragma unroll
        for (int n = 0; n < Q; ++n) x[n] = R[n + Q * t];
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            float s = 0.f;
#pragma unroll
            for (int n = 0; n < Q; ++n) s += A[m * Q + n] * x[n];
            R[m + Q * t] = s;
        }
    }
}

// Along x: R[., a, b] <- A R[., a, b] for every pencil (A row-major q x q).
template <typename T, int Q>
__device__ __forceinline__ void pass_x(const T *A, T *R) {
    if constexpr (sizeof(T) == 4) {
        pass_x2<Q>(reinterpret_cast<const float *>(A), reinterpret_cast<float *>(R));
    } else {
#pragma unroll
        for (int t = 0; t < Q * Q; ++t) {
            T x[Q];
#pragma unroll
            for (int n = 0; n < Q; ++n) x[n] = R[n + Q * t];
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                T s = T(0);
#pragma unroll
                for (int n = 0; n < Q; ++n) s += A[m * Q + n] * x[n];
                R[m + Q * t] = s;
            }
        }
    }
}

// r -= N u_nb for the face normal to the current x axis on side `side`, whose
// neighbour fields fld = [g | h] (q^2 each) are indexed sa * a + sb * b at the
// current tangential position (a, b) = (y, z). With G, H the fields after the
// tangential mass M_a (x) M_b (the 1D masses of the original axes now at y and
// z, applied in their rank-one form M = diag(w) - u u^T: 3q operations per
// pencil instead of q^2; wa, ua / wb, ub in shared memory):
//   low face:  N = kF [e_0 (x) (H/2 - gamma G) - d_0 (x) G/2],
//   high face: N = kF [e_p (x) (-H/2 - gamma G) + d_p (x) G/2].
// The two terms of G share one vector: the pencil at (a, b) takes
// G(a, b) c with c = sgn kF/2 d + kF gamma e_end, formed once per face.
template <typename T, int Q>
__device__ __forceinline__ void lift_x_face(int side, const T *fld, int sa, int sb, const T *wa, const T *ua,
                                            const T *wb, const T *ub, const T *dv, T gam, T kF, T *R) {
    constexpr int NF = Q * Q;
    const T wv = T(0.5) * kF;
    // value field: all layers += G c; derivative field: end layer -= sgn kF/2 H
    T cg[Q];
    {
        const T sw = side ? -wv : wv;
#pragma unroll
        for (int n = 0; n < Q; ++n) cg[n] = sw * dv[n];
        cg[side ? Q - 1 : 0] += kF * gam;
    }
#pragma unroll
    for (int comp = 0; comp < 2; ++comp) {
        const T *f = fld + comp * NF;
        T t1[NF];                                      // t1[a + q b] = (M_b f(a, .))[b]
        if constexpr (sizeof(T) == 4) {
            // rows a and a + 1 together by two-lane FMAs
#pragma unroll
            for (int a = 0; a + 1 < Q; a += 2) {
                float2 col[Q];
                float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int bb = 0; bb < Q; ++bb) {
                    col[bb] = make_float2((float)f[sa * a + sb * bb], (float)f[sa * (a + 1) + sb * bb]);
                    s2 = __ffma2_rn(make_float2((float)ub[bb], (float)ub[bb]), col[bb], s2);
                }
#pragma unroll
                for (int b = 0; b < Q; ++b) {
                    const float2 t = __ffma2_rn(make_float2(-(float)ub[b], -(float)ub[b]), s2,
                                                __fmul2_rn(make_float2((float)wb[b], (float)wb[b]), col[b]));
                    t1[a + Q * b] = (T)t.x;
                    t1[a + 1 + Q * b] = (T)t.y;
                }
            }
            if (Q & 1) {
                constexpr int a = Q - 1;
                T col[Q];
                T s = T(0);
#pragma unroll
                for (int bb = 0; bb < Q; ++bb) {
                    col[bb] = f[sa * a + sb * bb];
                    s += ub[bb] * col[bb];
                }
#pragma unroll
                for (int b = 0; b < Q; ++b) t1[a + Q * b] = wb[b] * col[b] - ub[b] * s;
            }
        } else {
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                T col[Q];
                T s = T(0);
#pragma unroll
                for (int bb = 0; bb < Q; ++bb) {
                    col[bb] = f[sa * a + sb * bb];
                    s += ub[bb] * col[bb];
                }
#pragma unroll
                for (int b = 0; b < Q; ++b) t1[a + Q * b] = wb[b] * col[b] - ub[b] * s;
            }
        }
        if constexpr (sizeof(T) == 4) {
            if (comp == 0) {
                T vv[NF];
#pragma unroll
                for (int b = 0; b < Q; ++b) {
                    T s = T(0);
#pragma unroll
                    for (int aa = 0; aa < Q; ++aa) s += ua[aa] * t1[aa + Q * b];
#pragma unroll
                    for (int a = 0; a < Q; ++a) vv[a + Q * b] = wa[a] * t1[a + Q * b] - ua[a] * s;
                }
                // pencils t, t + 1: pen[n] += v c[n] by two-lane FMAs
                float *Rf = reinterpret_cast<float *>(R);
#pragma unroll
                for (int t = 0; t < NF; t += 2) {
                    if (t + 1 < NF) {
                        const float2 v2 = make_float2((float)vv[t], (float)vv[t + 1]);
#pragma unroll
                        for (int n = 0; n < Q; ++n) {
                            float2 pp = make_float2(Rf[Q * t + n], Rf[Q * (t + 1) + n]);
                            pp = __ffma2_rn(v2, make_float2((float)cg[n], (float)cg[n]), pp);
                            Rf[Q * t + n] = pp.x;
                            Rf[Q * (t + 1) + n] = pp.y;
                        }
                    } else {
#pragma unroll
                        for (int n = 0; n < Q; ++n) R[Q * t + n] += vv[t] * cg[n];
                    }
                }
                continue;
            }
        }
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            T s = T(0);
#pragma unroll
            for (int aa = 0; aa < Q; ++aa) s += ua[aa] * t1[aa + Q * b];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const T v = wa[a] * t1[a + Q * b] - ua[a] * s;
                T *pen = R + Q * (a + Q * b);              // the pencil along x at (a, b)
                if (comp == 0) {
#pragma unroll
                    for (int n = 0; n < Q; ++n) pen[n] += v * cg[n];
                } else {
                    if (side) pen[Q - 1] += wv * v; else pen[0] -= wv * v;
                }
            }
        }
    }
}

// Traces of the face normal to the current x axis on side `side` into dst
// ([value q^2 | derivative q^2], indexed sa * a + sb * b).
template <typename T, int Q>
__device__ __forceinline__ void x_face_traces(int side, const T *R, const T *dv, int sa, int sb, T *dst) {
    constexpr int NF = Q * Q;
    if constexpr (sizeof(T) == 4) {
        // derivative traces of pencils t and t + 1 by two-lane FMAs
#pragma unroll
        for (int t = 0; t < NF; t += 2) {
            const int a0 = t % Q, b0 = t / Q;
            const float *p0 = reinterpret_cast<const float *>(R) + Q * t;
            if (t + 1 < NF) {
                const int a1 = (t + 1) % Q, b1 = (t + 1) / Q;
                const float *p1 = p0 + Q;
                float2 d = __fmul2_rn(make_float2((float)dv[0], (float)dv[0]), make_float2(p0[0], p1[0]));
#pragma unroll
                for (int n = 1; n < Q; ++n)
                    d = __ffma2_rn(make_float2((float)dv[n], (float)dv[n]), make_float2(p0[n], p1[n]), d);
                dst[sa * a0 + sb * b0] = side ? (T)p0[Q - 1] : (T)p0[0];
                dst[sa * a1 + sb * b1] = side ? (T)p1[Q - 1] : (T)p1[0];
                dst[NF + sa * a0 + sb * b0] = (T)d.x;
                dst[NF + sa * a1 + sb * b1] = (T)d.y;
            } else {
                T d = T(0);
#pragma unroll
                for (int n = 0; n < Q; ++n) d += dv[n] * R[Q * t + n];
                dst[sa * a0 + sb * b0] = side ? R[Q * t + Q - 1] : R[Q * t];
                dst[NF + sa * a0 + sb * b0] = d;
            }
        }
    } else {
#pragma unroll
        for (int b = 0; b < Q; ++b)
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const T *pen = R + Q * (a + Q * b);
                T d = T(0);
#pragma unroll
                for (int n = 0; n < Q; ++n) d += dv[n] * pen[n];
                dst[sa * a + sb * b] = side ? pen[Q - 1] : pen[0];
                dst[NF + sa * a + sb * b] = d;
            }
    }
}

// Traces of the cell tensor R (one per lane) to tr_out[cell][face][FS]: the
// faces normal to axis p, then rotate. FP32: every lane writes its two faces
// into its parts of two slots of shared memory (slot0, slot1: W x FS values
// each, free for the whole call) and stores each with one bulk store (a slot is
// rewritten once the lane's previous stores have read it); FP64 (LEAN):
// written per lane. R ends rotated. Only lanes with `write` store.
template <typename T, int Q>
__device__ __forceinline__ void cells_write_traces(const DGConst<T> &c, T *R, int lane, bool write, int64_t cell,
                                                   T *slot0, T *slot1, T *__restrict__ tr_out) {
    using G = CellGeo<T, Q>;
    constexpr int FS = G::FS, TR = G::TR;
    // unrolled: the two rotations become register renames
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int sa = p == 1 ? Q : 1, sb = p == 1 ? 1 : Q;
        if (!G::LEAN && p > 0) bulk_wait_read_all();
        if (write) {
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {
                T dv[Q];
#pragma unroll
                for (int n = 0; n < Q; ++n) dv[n] = side ? c.dp[p][n] : c.d0[p][n];
                T *dst = G::LEAN ? tr_out + cell * TR + (2 * p + side) * FS : (side ? slot1 : slot0) + lane * FS;
                x_face_traces<T, Q>(side, R, dv, sa, sb, dst);
            }
            if (!G::LEAN) {
                fence_proxy_async_smem();
#pragma unroll
                for (int side = 0; side < 2; ++side)
                    bulk_store(tr_out + cell * TR + (2 * p + side) * FS, (side ? slot1 : slot0) + lane * FS,
                               (unsigned)(FS * sizeof(T)));
                bulk_commit();
            }
        }
        if (p < 2) rotate<T, Q>(R);
    }
    if (!G::LEAN) bulk_wait_read_all();
}

template <typename T>
__device__ __forceinline__ T div_approx(T a, T b);
template <>
__device__ __forceinline__ float div_approx<float>(float a, float b) { return __fdividef(a, b); }
template <>
__device__ __forceinline__ double div_approx<double>(double a, double b) { return a / b; }

// Divide the transformed cell tensor R[x + q y + q^2 z] by the eigenvalue sums
// lambda_x + lambda_y + lambda_z of the fast diagonalisation (fd: the cell's
// factors, axis a at a * (q^2 + q), lambda after S), or multiply it by the
// precomputed table of their inverses (li, q^3 values) when there is one.
template <typename T, int Q>
__device__ __forceinline__ void scale_inverse(T *R, const T *fd, const T *li) {
    constexpr int FDS = Q * Q + Q;
    if (li) {
#pragma unroll
        for (int e = 0; e < Q * Q * Q; ++e) R[e] *= li[e];
        return;
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const T lz = fd[2 * FDS + Q * Q + k];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const T lyz = fd[1 * FDS + Q * Q + j] + lz;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int e = i + Q * (j + Q * k);
                R[e] = div_approx<T>(R[e], fd[Q * Q + i] + lyz);
            }
        }
    }
}

// Bulk copy of `bytes` into shared memory on `bar` (lane 0 issues).
template <typename T>
__device__ __forceinline__ void stage_bulk(bool full, int lane, uint64_t *bar, T *dst, const T *src, int64_t count,
                                           int ncount) {
    if (full) {
        if (lane == 0) {
            mbar_arrive_expect_tx(bar, (unsigned)(count * sizeof(T)));
            bulk_load(dst, src, (unsigned)(count * sizeof(T)), bar);
        }
    } else {
        for (int e = lane; e < ncount; e += 32) dst[e] = src[e];
    }
}

template <typename T, int Q>
__device__ __forceinline__ void smooth_cells_body(const DGConst<T> &c, int64_t cell0, T *__restrict__ u, const T *__restrict__ b, const T *__restrict__ kappa, const T *__restrict__ fd, const T *__restrict__ linv, const T *__restrict__ tr_in, T *__restrict__ tr_out, bool reuse = false) {
    using G = CellGeo<T, Q>;
    constexpr int W = G::W, NL = G::NL, FDS = G::FDS, TR = G::TR, FS = G::FS;
    extern __shared__ __align__(128) unsigned char smem_c[];
    // area A: b -> face slot 1 (FP32) or the factors (FP64) -> previous u (FP32)
    //         -> new u -> trace slot 1
    // area B (FP32): face slot 0 -> factors -> trace slot 0
    T *sA = reinterpret_cast<T *>(smem_c);
    T *sB = sA + G::OFF_B;
    // mbarriers: 0 b, 1 previous u (FP32) / factors (FP64), 2 factors (FP32),
    // 4 face slot 0, 5 face slot 1 (phase k = the slot's k-th face)
    __shared__ __align__(8) uint64_t bars[6];
    __shared__ T sMw[3][Q], sMu[3][Q];
    const int lane = threadIdx.x;
    const int ncl = (int)min((int64_t)W, c.ncell - cell0);
    const bool full = ncl == W;                          // bulk copies of b, u, factors: whole 32-cell blocks
    const bool active = lane < ncl;
    const int64_t cell = cell0 + lane;
    const bool table = linv != nullptr;
    bool ok = true;                                      // false once a bounded wait ran out

    cells_init_bars(bars, 6, lane, reuse);
    for (int e = lane; e < 3 * Q; e += W) {
        sMw[e / Q][e % Q] = c.mw[e / Q][e % Q];
        sMu[e / Q][e % Q] = c.mu[e / Q][e % Q];
    }
    stage_bulk<T>(full, lane, &bars[0], sA, b + cell0 * NL, W * NL, ncl * NL);
    // neighbours of this lane's cell (a mask of interior faces and the strides);
    // the first neighbour face is requested at once
    int mask = 0;
    if (active) {
        int ci[3];
        cell_coords32(cell, c.n, ci);
        mask = interior_mask<3>(ci, c.n);
    }
    const int s1 = c.n[0], s2 = c.n[0] * c.n[1];
    if (!G::LEAN) stage_face<T, Q>(0, cell_neighbour(0, mask, cell, s1, s2), lane, tr_in, sB, &bars[4]);

    // r = b
    if (full)
        ok = warp_wait_copies(&bars[0], lane) && ok;
    else
        __syncwarp();
    T R[NL];
#pragma unroll
    for (int e = 0; e < NL; ++e) R[e] = active ? sA[lane * NL + e] : T(0);
    fence_proxy_async_smem();
    __syncwarp();
    // area A is free: FP32 the second neighbour face, FP64 the factors
    if (G::LEAN)
        stage_bulk<T>(full, lane, &bars[1], sA, fd + cell0 * 3 * FDS, W * 3 * FDS, ncl * 3 * FDS);
    else
        stage_face<T, Q>(1, cell_neighbour(1, mask, cell, s1, s2), lane, tr_in, sA, &bars[5]);

    // r -= N u_nb: the two faces normal to axis p, then rotate the next axis to x
#pragma unroll 1
    for (int p = 0; p < 3; ++p) {
        T dv[Q];
        const int ta = p == 2 ? 0 : p + 1, tb = p == 0 ? 2 : p - 1;
        const int sa = p == 1 ? Q : 1, sb = p == 1 ? 1 : Q;   // the y faces are stored transposed
        const T gam = c.gamma[p];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int f = 2 * p + side;
            const int nb = cell_neighbour(f, mask, cell, s1, s2);
            const T kF = nb >= 0 ? c.kfac[cell * 6 + f] : T(0);
            T *slot = side ? sA : sB;
            if (!G::LEAN) ok = warp_wait_phase(&bars[4 + side], (unsigned)(p & 1), lane) && ok;
            if (active && nb >= 0) {
#pragma unroll
                for (int n = 0; n < Q; ++n) dv[n] = side ? c.dp[p][n] : c.d0[p][n];
                const T *fld = G::LEAN ? tr_in + (int64_t)nb * TR + (f ^ 1) * FS : slot + lane * FS;
                lift_x_face<T, Q>(side, fld, sa, sb, sMw[ta], sMu[ta], sMw[tb], sMu[tb], dv, gam, kF, R);
            }
            if (!G::LEAN && f + 2 < 6) {
                fence_proxy_async_smem();
                __syncwarp();
                stage_face<T, Q>(f + 2, cell_neighbour(f + 2, mask, cell, s1, s2), lane, tr_in, slot,
                                 &bars[4 + side]);
            } else if (!G::LEAN && f == 4) {
                // area B is free after the last face of slot 0: the factors, whose copy
                // overlaps the lifting of face 5
                fence_proxy_async_smem();
                __syncwarp();
                stage_bulk<T>(full, lane, &bars[2], sB, fd + cell0 * 3 * FDS, W * 3 * FDS, ncl * 3 * FDS);
            }
        }
        rotate<T, Q>(R);
    }
    // FP32: the previous u into area A (face slot 1 is free now; u is first
    // needed after the inverse)
    if (!G::LEAN) {
        fence_proxy_async_smem();
        __syncwarp();
        stage_bulk<T>(full, lane, &bars[1], sA, u + cell0 * NL, W * NL, ncl * NL);
    }

    // A_KK^{-1} by fast diagonalisation: S^T along x, y, z; scale by the
    // inverse eigenvalue sums; S along x, y, z
    if (full)
        ok = warp_wait_copies(&bars[G::LEAN ? 1 : 2], lane) && ok;
    else
        __syncwarp();
    const T *myFD = (G::LEAN ? sA : sB) + lane * 3 * FDS;
    // (the tensor-product factors commute, so both halves take the axes in the
    // same order and one loop body serves all six passes)
#pragma unroll 1
    for (int k = 0; k < 6 && active; ++k) {
        if (k == 3) scale_inverse<T, Q>(R, myFD, table ? linv + cell * NL : nullptr);
        T S[Q * Q];
        if (k < 3)
            load_matrix<T, Q, true>(myFD + k * FDS, S);
        else
            load_matrix<T, Q, false>(myFD + (k - 3) * FDS, S);
        pass_x<T, Q>(S, R);
        rotate<T, Q>(R);
    }

    // u <- (1 - w) u + w y (w already in y when the inverse came from the table),
    // stored through area A (the barrier also ends every lane's reads of the
    // factors before area A (FP64) or B (FP32) is rewritten)
    if (!G::LEAN && full)
        ok = warp_wait_copies(&bars[1], lane) && ok;
    else
        __syncwarp();
    T *myU = sA + lane * NL;
    if (active) {
        const T om = c.omega, keep = T(1) - om;
        const T *uo = G::LEAN ? u + cell * NL : sA + lane * NL;
        if (table) {
#pragma unroll
            for (int e = 0; e < NL; ++e) R[e] = keep * uo[e] + R[e];
        } else {
#pragma unroll
            for (int e = 0; e < NL; ++e) R[e] = keep * uo[e] + om * R[e];
        }
#pragma unroll
        for (int e = 0; e < NL; ++e) myU[e] = R[e];
    }
    fence_proxy_async_smem();
    __syncwarp();
    // a launch whose wait ran out leaves u and the traces of its cells unchanged
    if (ok) {
        if (full) {
            if (lane == 0) {
                bulk_store(u + cell0 * NL, sA, (unsigned)(W * NL * sizeof(T)));
                bulk_commit();
                bulk_wait_read_all();                    // area A is read: trace slot 1
            }
        } else {
            for (int e = lane; e < ncl * NL; e += W) u[cell0 * NL + e] = sA[e];
        }
        __syncwarp();
        // traces of the new iterate (FP32: slots in areas B and A)
        cells_write_traces<T, Q>(c, R, lane, active, cell, sB, sA, tr_out);
    }
    bulk_wait_read_all();
}

// Warm-up projection (Alg. 4 preamble) with one thread per cell, 3D, GLL:
// optionally u += P e (the p-prolongation of the Q1 correction e, Sec. 5.1,
// trilinear hats of the cell's corner values at the GLL nodes), then the
// traces of every face. u arrives by a bulk copy; the updated u (with e)
// leaves by a bulk store, the traces as in the smoothing step.
template <typename T, int Q>
__device__ __forceinline__ void project_cells_body(const DGConst<T> &c, int64_t cell0, T *__restrict__ u,
                                                   const T *__restrict__ e0, T *__restrict__ tr) {
    using G = CellGeo<T, Q>;
    constexpr int W = G::W, NL = G::NL;
    extern __shared__ __align__(128) unsigned char smem_c[];
    T *sA = reinterpret_cast<T *>(smem_c);              // u
    T *sB = sA + G::OFF_B;                               // FP32: trace staging
    __shared__ __align__(8) uint64_t bars[1];
    const int lane = threadIdx.x;
    const int ncl = (int)min((int64_t)W, c.ncell - cell0);
    const bool full = ncl == W;
    const bool active = lane < ncl;
    const int64_t cell = cell0 + lane;
    if (full && lane == 0) {
        mbar_init(&bars[0], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    stage_bulk<T>(full, lane, &bars[0], sA, u + cell0 * NL, W * NL, ncl * NL);
    // the corner values of the correction (zero at boundary vertices)
    T ec[8];
    if (e0 != nullptr && active) {
        int ci[3];
        cell_coords<3>(cell, c.n, ci);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            bool interior = true;
            int64_t vid = 0, stride = 1;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int v = ci[a] + ((k >> a) & 1);
                interior = interior && v >= 1 && v <= c.n[a] - 1;
                vid += (int64_t)(v - 1) * stride;
                stride *= (c.n[a] - 1);
            }
            ec[k] = interior ? e0[vid] : T(0);
        }
    }
    if (full) {
        if (!warp_wait_copies(&bars[0], lane)) return;
    } else {
        __syncwarp();
    }
    T R[NL];
#pragma unroll
    for (int e = 0; e < NL; ++e) R[e] = active ? sA[lane * NL + e] : T(0);
    if (e0 != nullptr) {
        if (active) {
            // u(i,j,k) += sum over corners of e_c hat_cx(x_i) hat_cy(y_j) hat_cz(z_k), axis by axis
            T Z[4][Q];
#pragma unroll
            for (int cxy = 0; cxy < 4; ++cxy)
#pragma unroll
                for (int k = 0; k < Q; ++k) Z[cxy][k] = ec[cxy] * c.hat[0][k] + ec[cxy + 4] * c.hat[1][k];
#pragma unroll
            for (int k = 0; k < Q; ++k)
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    const T y0 = Z[0][k] * c.hat[0][j] + Z[2][k] * c.hat[1][j];   // cx = 0
                    const T y1 = Z[1][k] * c.hat[0][j] + Z[3][k] * c.hat[1][j];   // cx = 1
#pragma unroll
                    for (int i = 0; i < Q; ++i) R[i + Q * (j + Q * k)] += y0 * c.hat[0][i] + y1 * c.hat[1][i];
                }
#pragma unroll
            for (int e = 0; e < NL; ++e) sA[lane * NL + e] = R[e];
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (full) {
            if (lane == 0) {
                bulk_store(u + cell0 * NL, sA, (unsigned)(W * NL * sizeof(T)));
                bulk_commit();
            }
        } else {
            for (int e = lane; e < ncl * NL; e += W) u[cell0 * NL + e] = sA[e];
        }
    }
    // area A (u) becomes the second trace slot once its store has read it
    if (e0 != nullptr && full && lane == 0) bulk_wait_read_all();
    __syncwarp();
    cells_write_traces<T, Q>(c, R, lane, active, cell, sB, sA, tr);
    bulk_wait_read_all();
}

template <typename T, int Q>
__global__ void __launch_bounds__(32) k_project_cells(const __grid_constant__ DGConst<T> c, T *__restrict__ u,
                                                      const T *__restrict__ e0, T *__restrict__ tr) {
    project_cells_body<T, Q>(c, (int64_t)blockIdx.x * CellGeo<T, Q>::W, u, e0, tr);
}

// Kt_a of the cell along axis a (row-major q x q, GLL): kappa_K K_a plus the
// cell's own facet terms of the two faces normal to a (rows and columns 0 and
// q - 1); kF[f] is the facet coefficient of an interior face f (bit f of mask),
// a boundary face takes kappa_K with weight 1 (Nitsche). The same entries as the
// per-pencil kernels' block tables.
template <typename T, int Q, int A>
__device__ __forceinline__ void build_kt(const DGConst<T> &c, T kK, const T *kF, int mask, T *Kt) {
    const bool inL = mask & (1 << (2 * A)), inR = mask & (1 << (2 * A + 1));
    const T kL = inL ? kF[2 * A] : kK, wL = inL ? T(0.5) : T(1);
    const T kR = inR ? kF[2 * A + 1] : kK, wR = inR ? T(0.5) : T(1);
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            T v = kK * c.K[A][i * Q + j];
            if (i == 0 || j == 0) {
                if (i == 0 && j == 0)
                    v += kL * (T(2) * wL * c.d0[A][0] + c.gamma[A]);
                else
                    v += kL * wL * c.d0[A][i == 0 ? j : i];
            }
            if (i == Q - 1 || j == Q - 1) {
                if (i == Q - 1 && j == Q - 1)
                    v += kR * (c.gamma[A] - T(2) * wR * c.dp[A][Q - 1]);
                else
                    v -= kR * wR * c.dp[A][i == Q - 1 ? j : i];
            }
            Kt[i * Q + j] = v;
        }
}

// R = A_KK u in the direct sum-factorised form A_KK = sum_a Kt_a (x) M (x) M
// (the rounding of the per-pencil kernels, which the FP32 CG recurrences need),
// one thread per cell: u in the lane's part Y of shared memory (natural order
// x + q y + q^2 z), overwritten by the second intermediate. With the 1D masses
// in their rank-one form M x = w o x - mu (mu . x):
//   along z: R = M_z u, Y = Kt_z u;
//   along y: R <- M_y R, Y <- Kt_y R + M_y Y;
//   along x: R <- Kt_x R + M_x Y.
// Each pencil reads and writes only its own positions of Y, and the axes are
// fixed at compile time (no rotation of R).
template <typename T, int Q>
__device__ __forceinline__ void direct_volume(const DGConst<T> &c, T kK, const T *kF, int mask, T *Y, T *R) {
    T Kt[Q * Q];
    build_kt<T, Q, 2>(c, kK, kF, mask, Kt);
#pragma unroll
    for (int j = 0; j < Q; ++j)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T x[Q];
#pragma unroll
            for (int n = 0; n < Q; ++n) x[n] = Y[i + Q * j + Q * Q * n];
            T d = T(0);
#pragma unroll
            for (int n = 0; n < Q; ++n) d += c.mu[2][n] * x[n];
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                T sb = T(0);
#pragma unroll
                for (int n = 0; n < Q; ++n) sb += Kt[m * Q + n] * x[n];
                R[i + Q * j + Q * Q * m] = c.mw[2][m] * x[m] - c.mu[2][m] * d;
                Y[i + Q * j + Q * Q * m] = sb;
            }
            asm volatile("" ::: "memory");   // keeps later pencils' loads here (no spills)
        }
    build_kt<T, Q, 1>(c, kK, kF, mask, Kt);
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T xa[Q], xb[Q];
#pragma unroll
            for (int n = 0; n < Q; ++n) {
                xa[n] = R[i + Q * n + Q * Q * k];
                xb[n] = Y[i + Q * n + Q * Q * k];
            }
            T da = T(0), db = T(0);
#pragma unroll
            for (int n = 0; n < Q; ++n) {
                da += c.mu[1][n] * xa[n];
                db += c.mu[1][n] * xb[n];
            }
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                T se = c.mw[1][m] * xb[m] - c.mu[1][m] * db;
#pragma unroll
                for (int n = 0; n < Q; ++n) se += Kt[m * Q + n] * xa[n];
                R[i + Q * m + Q * Q * k] = c.mw[1][m] * xa[m] - c.mu[1][m] * da;
                Y[i + Q * m + Q * Q * k] = se;
            }
            asm volatile("" ::: "memory");
        }
    build_kt<T, Q, 0>(c, kK, kF, mask, Kt);
#pragma unroll
    for (int t = 0; t < Q * Q; ++t) {
        T xa[Q], xb[Q];
#pragma unroll
        for (int n = 0; n < Q; ++n) {
            xa[n] = R[n + Q * t];
            xb[n] = Y[n + Q * t];
        }
        T db = T(0);
#pragma unroll
        for (int n = 0; n < Q; ++n) db += c.mu[0][n] * xb[n];
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            T sy = c.mw[0][m] * xb[m] - c.mu[0][m] * db;
#pragma unroll
            for (int n = 0; n < Q; ++n) sy += Kt[m * Q + n] * xa[n];
            R[m + Q * t] = sy;
        }
        asm volatile("" ::: "memory");
    }
}

// Residual r = b - A u with one thread per cell, 3D, exact diagonal blocks
// (Alg. 2 stage 3; the residual of a V-cycle level and the operator apply),
// with A u = A_KK u + N u_nb. A_KK u from the cell's fast-diagonalisation
// factors: Kt_a S_a = M_a S_a Lambda_a with S_a^T M_a S_a = I gives
// A_KK = (M S)^(x3) (Lambda_x + Lambda_y + Lambda_z) (S^T M)^(x3), so A_KK u
// takes the six tensor passes of the smoother's inverse, with P_a = S_a^T M_a
// and its transpose, and a multiplication by the eigenvalue sums instead of a
// division. fd holds [P_a | Lambda_a] per cell and axis (computed once at
// set-up from the smoother's factors). Then b is added and the neighbour terms are lifted as in the
// smoothing step. Outputs as for k_residual: r (negated for y = A u) and the
// cell corner sums of the p-restriction.
// Staging: u and the factors by bulk copies; FP32: b into u's area once u is
// in registers, the neighbour faces through the slots once the factors are
// used; FP64 (LEAN): the factors into u's area, b and the faces read per lane.
// r leaves through area A by a bulk store.
// DIRECT (FP32, fd unused): A_KK u in the direct form (direct_volume) instead,
// for the operator of the FP32 CG recurrences; u stays in area A for the
// volume passes, the first neighbour face is staged into area B at once, b is
// read per lane.
template <typename T, int Q, bool DIRECT = false>
__device__ __forceinline__ void residual_cells_body(const DGConst<T> &c, int64_t cell0, int mode,
                                                    const T *__restrict__ u, const T *__restrict__ b,
                                                    const T *__restrict__ kappa, const T *__restrict__ fd,
                                                    const T *__restrict__ tr, T *__restrict__ rout,
                                                    T *__restrict__ corners, bool reuse = false) {
    using G = CellGeo<T, Q>;
    constexpr int W = G::W, NL = G::NL, FDS = G::FDS, TR = G::TR, FS = G::FS;
    extern __shared__ __align__(128) unsigned char smem_c[];
    T *sA = reinterpret_cast<T *>(smem_c);              // u -> b (FP32) or factors (FP64) -> face slot 1 -> r
    T *sB = sA + G::OFF_B;                               // FP32: factors -> face slot 0
    // mbarriers: 0 u, 1 b (FP32) / factors (FP64), 2 factors (FP32), 4 face
    // slot 0 (area B), 5 face slot 1 (area A) (FP32; phase k = the slot's k-th face)
    __shared__ __align__(8) uint64_t bars[6];
    __shared__ T sMw[3][Q], sMu[3][Q];
    const int lane = threadIdx.x;
    const int ncl = (int)min((int64_t)W, c.ncell - cell0);
    const bool full = ncl == W;
    const bool active = lane < ncl;
    const int64_t cell = cell0 + lane;
    const bool has_b = (mode & RES_HAS_B) != 0;

    cells_init_bars(bars, 6, lane, reuse);
    for (int e = lane; e < 3 * Q; e += W) {
        sMw[e / Q][e % Q] = c.mw[e / Q][e % Q];
        sMu[e / Q][e % Q] = c.mu[e / Q][e % Q];
    }
    bool ok = true;                                      // false once a bounded wait ran out
    static_assert(!DIRECT || !G::LEAN, "the direct form is the FP32 operator's");
    stage_bulk<T>(full, lane, &bars[0], sA, u + cell0 * NL, W * NL, ncl * NL);
    if (!G::LEAN && !DIRECT)
        stage_bulk<T>(full, lane, &bars[2], sB, fd + cell0 * 3 * FDS, W * 3 * FDS, ncl * 3 * FDS);
    int mask = 0;
    if (active) {
        int ci[3];
        cell_coords32(cell, c.n, ci);
        mask = interior_mask<3>(ci, c.n);
    }
    const int s1 = c.n[0], s2 = c.n[0] * c.n[1];
    if (DIRECT) stage_face<T, Q>(0, cell_neighbour(0, mask, cell, s1, s2), lane, tr, sB, &bars[4]);
    const T kK = active ? kappa[cell] : T(1);

    if (full)
        ok = warp_wait_copies(&bars[0], lane) && ok;
    else
        __syncwarp();
    T R[NL];
    if constexpr (DIRECT) {
        if (active) {
            T kF[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) kF[f] = c.kfac[cell * 6 + f];
            direct_volume<T, Q>(c, kK, kF, mask, sA + lane * NL, R);
            const T *bb = has_b ? b + cell * NL : nullptr;
#pragma unroll
            for (int e = 0; e < NL; ++e) R[e] = (bb ? bb[e] : T(0)) - R[e];
        } else {
#pragma unroll
            for (int e = 0; e < NL; ++e) R[e] = T(0);
        }
        fence_proxy_async_smem();
        __syncwarp();
        stage_face<T, Q>(1, cell_neighbour(1, mask, cell, s1, s2), lane, tr, sA, &bars[5]);
    } else {
#pragma unroll
        for (int e = 0; e < NL; ++e) R[e] = active ? sA[lane * NL + e] : T(0);
        fence_proxy_async_smem();
        __syncwarp();
        // area A: the factors (FP64) or b (FP32)
        if (G::LEAN)
            stage_bulk<T>(full, lane, &bars[1], sA, fd + cell0 * 3 * FDS, W * 3 * FDS, ncl * 3 * FDS);
        else if (has_b)
            stage_bulk<T>(full, lane, &bars[1], sA, b + cell0 * NL, W * NL, ncl * NL);
        const bool b_staged = !G::LEAN && has_b;

        // R = A_KK u: P along x, y, z; times the eigenvalue sums; P^T along x, y, z
        // (the tensor-product factors commute: one loop body for all six passes)
        if (full)
            ok = warp_wait_copies(&bars[G::LEAN ? 1 : 2], lane) && ok;
        else
            __syncwarp();
        const T *myFD = (G::LEAN ? sA : sB) + lane * 3 * FDS;
#pragma unroll 1
        for (int k = 0; k < 6 && active; ++k) {
            if (k == 3) {
#pragma unroll
                for (int kz = 0; kz < Q; ++kz) {
                    const T lz = myFD[2 * FDS + Q * Q + kz];
#pragma unroll
                    for (int j = 0; j < Q; ++j) {
                        const T lyz = myFD[1 * FDS + Q * Q + j] + lz;
#pragma unroll
                        for (int i = 0; i < Q; ++i) R[i + Q * (j + Q * kz)] *= myFD[Q * Q + i] + lyz;
                    }
                }
            }
            T P[Q * Q];
            const int ax = k < 3 ? k : k - 3;
            if (k < 3)
                load_matrix<T, Q, false>(myFD + ax * FDS, P);   // P_a = S_a^T M_a, precomputed per cell
            else
                load_matrix<T, Q, true>(myFD + ax * FDS, P);    // its transpose M_a S_a
            pass_x<T, Q>(P, R);
            rotate<T, Q>(R);
        }
        // R = b - A_KK u
        if (b_staged && full)
            ok = warp_wait_copies(&bars[1], lane) && ok;
        else
            __syncwarp();
        if (active) {
            const T *bb = has_b ? (G::LEAN ? b + cell * NL : sA + lane * NL) : nullptr;
#pragma unroll
            for (int e = 0; e < NL; ++e) R[e] = (bb ? bb[e] : T(0)) - R[e];
        }
        // FP32: the neighbour faces into the slots (every lane is done with the
        // factors in area B and with b in area A)
        if (!G::LEAN) {
            fence_proxy_async_smem();
            __syncwarp();
            stage_face<T, Q>(0, cell_neighbour(0, mask, cell, s1, s2), lane, tr, sB, &bars[4]);
            stage_face<T, Q>(1, cell_neighbour(1, mask, cell, s1, s2), lane, tr, sA, &bars[5]);
        }
    }
    // R -= N u_nb, face pair by face pair as in the smoothing step
#pragma unroll 1
    for (int p = 0; p < 3; ++p) {
        T dv[Q];
        const int ta = p == 2 ? 0 : p + 1, tb = p == 0 ? 2 : p - 1;
        const int sa = p == 1 ? Q : 1, sb = p == 1 ? 1 : Q;
        const T gam = c.gamma[p];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int f = 2 * p + side;
            const int nb = cell_neighbour(f, mask, cell, s1, s2);
            const T kF = nb >= 0 ? c.kfac[cell * 6 + f] : T(0);
            T *slot = side ? sA : sB;
            if (!G::LEAN) ok = warp_wait_phase(&bars[4 + side], (unsigned)(p & 1), lane) && ok;
            if (active && nb >= 0) {
#pragma unroll
                for (int n = 0; n < Q; ++n) dv[n] = side ? c.dp[p][n] : c.d0[p][n];
                const T *fld = G::LEAN ? tr + (int64_t)nb * TR + (f ^ 1) * FS : slot + lane * FS;
                lift_x_face<T, Q>(side, fld, sa, sb, sMw[ta], sMu[ta], sMw[tb], sMu[tb], dv, gam, kF, R);
            }
            if (!G::LEAN && f + 2 < 6) {
                fence_proxy_async_smem();
                __syncwarp();
                stage_face<T, Q>(f + 2, cell_neighbour(f + 2, mask, cell, s1, s2), lane, tr, slot, &bars[4 + side]);
            }
        }
        rotate<T, Q>(R);
    }
    if (mode & RES_NEGATE) {
#pragma unroll
        for (int e = 0; e < NL; ++e) R[e] = -R[e];
    }
    if ((mode & RES_WRITE_R) && ok) {
        __syncwarp();                                  // every lane is done with area A
        if (active) {
#pragma unroll
            for (int e = 0; e < NL; ++e) sA[lane * NL + e] = R[e];
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (full) {
            if (lane == 0) {
                bulk_store(rout + cell0 * NL, sA, (unsigned)(W * NL * sizeof(T)));
                bulk_commit();
            }
        } else {
            for (int e = lane; e < ncl * NL; e += W) rout[cell0 * NL + e] = sA[e];
        }
    }
    if ((mode & RES_CORNERS) && active && ok) {
        // corner (cx, cy, cz): sum over the nodes of hat_cx(x_i) hat_cy(y_j) hat_cz(z_k) r_ijk
        T X[2][Q * Q];
#pragma unroll
        for (int t = 0; t < Q * Q; ++t) {
            T s0 = T(0), s1 = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                s0 += c.hat[0][i] * R[i + Q * t];
                s1 += c.hat[1][i] * R[i + Q * t];
            }
            X[0][t] = s0;
            X[1][t] = s1;
        }
        T out[8];
#pragma unroll
        for (int cx = 0; cx < 2; ++cx)
#pragma unroll
            for (int cy = 0; cy < 2; ++cy) {
                T Y[Q];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    T sy = T(0);
#pragma unroll
                    for (int j = 0; j < Q; ++j) sy += c.hat[cy][j] * X[cx][j + Q * k];
                    Y[k] = sy;
                }
#pragma unroll
                for (int cz = 0; cz < 2; ++cz) {
                    T sz = T(0);
#pragma unroll
                    for (int k = 0; k < Q; ++k) sz += c.hat[cz][k] * Y[k];
                    out[cx | (cy << 1) | (cz << 2)] = sz;
                }
            }
#pragma unroll
        for (int k = 0; k < 8; ++k) corners[cell * 8 + k] = out[k];
    }
    bulk_wait_read_all();
}

template <typename T, int Q>
__global__ void __launch_bounds__(32) k_residual_cells(const __grid_constant__ DGConst<T> c, int mode,
                                                       const T *__restrict__ u, const T *__restrict__ b,
                                                       const T *__restrict__ kappa, const T *__restrict__ fd,
                                                       const T *__restrict__ tr, T *__restrict__ rout,
                                                       T *__restrict__ corners) {
    residual_cells_body<T, Q>(c, (int64_t)blockIdx.x * CellGeo<T, Q>::W, mode, u, b, kappa, fd, tr, rout, corners);
}

// The same output with A_KK u in the direct form (FP32 CG operator; no factors).
template <typename T, int Q>
__global__ void __launch_bounds__(32) k_residual_cells_direct(const __grid_constant__ DGConst<T> c, int mode,
                                                              const T *__restrict__ u, const T *__restrict__ b,
                                                              const T *__restrict__ kappa,
                                                              const T *__restrict__ tr, T *__restrict__ rout,
                                                              T *__restrict__ corners) {
    residual_cells_body<T, Q, true>(c, (int64_t)blockIdx.x * CellGeo<T, Q>::W, mode, u, b, kappa, nullptr, tr, rout,
                                    corners);
}

template <typename T, int Q>
__global__ void __launch_bounds__(32) k_smooth_cells(const __grid_constant__ DGConst<T> c, T *__restrict__ u,
                                                     const T *__restrict__ b, const T *__restrict__ kappa,
                                                     const T *__restrict__ fd, const T *__restrict__ linv,
                                                     const T *__restrict__ tr_in, T *__restrict__ tr_out) {
    smooth_cells_body<T, Q>(c, (int64_t)blockIdx.x * CellGeo<T, Q>::W, u, b, kappa, fd, linv, tr_in, tr_out);
}

// Host-side read of the timeout counter of this translation unit.
static inline cudaError_t read_wait_timeouts(unsigned long long *v) {
    return cudaMemcpyFromSymbol(v, g_wait_timeouts, sizeof(*v));
}

}  // namespace dgmg
