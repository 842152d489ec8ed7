// libdgmg context: hierarchy set-up on the host, device buffers, the stage
// entry points, the hp V-cycle and the FP64 preconditioned CG solve.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.h"

namespace dgmg {

std::atomic<long long> g_kernel_launches{0};
std::atomic<int> g_q1_one_launch_off{0};

unsigned persistent_grid(const void *fn, int threads, size_t smem, int64_t items) {
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> cap;
    if (items <= 0) return 0;
    int c = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cap.find({fn, smem});
        if (it != cap.end()) c = it->second;
    }
    if (c == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess) {
            cudaGetLastError();
            per = 1;
        }
        c = std::max(1, sms * std::max(per, 1));
        std::lock_guard<std::mutex> lk(mu);
        cap[{fn, smem}] = c;
    }
    return (unsigned)std::min<int64_t>(items, c);
}

// ------------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return DGMG_ECUDA;
}

// ------------------------------------------------------------ set-up trace
// With the environment variable DGMG_TRACE_SETUP set, dgmg_create prints the
// wall time of each set-up phase to stderr.
struct SetupTrace {
    bool on = std::getenv("DGMG_TRACE_SETUP") != nullptr;
    std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
    void mark(const char *what) {
        if (!on) return;
        const auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "dgmg setup %-14s %8.3f ms\n", what,
                     std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};

// ---------------------------------------------------------- host threading
template <typename F>
static void parallel_for(int64_t n, F f) {
    unsigned nt = std::thread::hardware_concurrency();
    // about 2048 items per thread: thread start-up costs tens of microseconds
    nt = (unsigned)std::max<int64_t>(1, std::min<int64_t>({(int64_t)nt, 64, n / 2048}));
    if (nt == 1) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    const int64_t chunk = (n + nt - 1) / nt;
    for (unsigned k = 0; k < nt; ++k) {
        const int64_t a = k * chunk, b = std::min(n, a + chunk);
        if (a >= b) break;
        th.emplace_back([=, &f]() {
            for (int64_t i = a; i < b; ++i) f(i);
        });
    }
    for (auto &t : th) t.join();
}

// --------------------------------------------------------------- Q1 levels
static std::vector<int> coarse_positions(int n, int f) {
    std::vector<int> pos;
    for (int i = 0; i < n; i += f) pos.push_back(i);
    pos.push_back(n);
    return pos;
}

static bool can_coarsen(int n, int f) { return n > f; }

// Per-axis nested Q1 interpolation tables between n fine cells and the coarse
// axis (coarse vertices at fine indices 0, f, 2f, ..., n).
static void axis_tables(int n, int f, CGLevelHost &L, int a, int &nc) {
    const int mf = n - 1;
    L.pl_lo[a].assign(mf, -1);
    L.pl_hi[a].assign(mf, -1);
    L.pl_wlo[a].assign(mf, 0.0);
    L.pl_whi[a].assign(mf, 0.0);
    if (!can_coarsen(n, f)) {
        nc = n;
        for (int i = 0; i < mf; ++i) {
            L.pl_lo[a][i] = i;
            L.pl_wlo[a][i] = 1.0;
        }
        L.rs_start[a].resize(mf);
        L.rs_cnt[a].assign(mf, 1);
        L.rs_w[a].assign(mf * 5, 0.0);
        for (int i = 0; i < mf; ++i) {
            L.rs_start[a][i] = i;
            L.rs_w[a][i * 5] = 1.0;
        }
        return;
    }
    const std::vector<int> pos = coarse_positions(n, f);
    nc = (int)pos.size() - 1;
    for (int i = 1; i < n; ++i) {           // fine interior vertex i
        int j = 0;
        while (!(pos[j] <= i && i < pos[j + 1])) ++j;
        const double wlo = double(pos[j + 1] - i) / double(pos[j + 1] - pos[j]);
        const double whi = double(i - pos[j]) / double(pos[j + 1] - pos[j]);
        if (j >= 1 && wlo != 0.0) {
            L.pl_lo[a][i - 1] = j - 1;
            L.pl_wlo[a][i - 1] = wlo;
        }
        if (j + 1 <= nc - 1 && whi != 0.0) {
            L.pl_hi[a][i - 1] = j;               // coarse vertex j+1 -> interior index j
            L.pl_whi[a][i - 1] = whi;
        }
    }
    const int mcv = nc - 1;
    L.rs_start[a].assign(mcv, 0);
    L.rs_cnt[a].assign(mcv, 0);
    L.rs_w[a].assign(mcv * 5, 0.0);
    for (int J = 1; J < nc; ++J) {
        const int lo = pos[J - 1], mid = pos[J], hi = pos[J + 1];
        L.rs_start[a][J - 1] = lo;              // fine vertex lo+1 -> interior index lo
        int k = 0;
        for (int i = lo + 1; i < hi; ++i, ++k) {
            const double w = i <= mid ? double(i - lo) / double(mid - lo) : double(hi - i) / double(hi - mid);
            L.rs_w[a][(J - 1) * 5 + k] = w;
        }
        L.rs_cnt[a][J - 1] = k;
    }
}

static int stencil_size(int dim) { return dim == 3 ? 27 : 9; }

// Level 0: the kappa-weighted Q1 stiffness on the interior vertices, which equals
// P^T A P for the SIPG operator A (all facet terms vanish on continuous functions
// that are zero on the boundary, Sec. 2.4). Element matrix per cell:
// sum over axes of K1 (x) M1 (x) M1 with K1 = (1/h)[1 -1; -1 1], M1 = (h/6)[2 1; 1 2].
static void build_level0(int dim, const int *n, const std::vector<double> &kappa, CGLevelHost &L) {
    const int NS = stencil_size(dim);
    for (int a = 0; a < 3; ++a) {
        L.n[a] = a < dim ? n[a] : 1;
        L.m[a] = a < dim ? n[a] - 1 : 1;
    }
    L.nv = (int64_t)L.m[0] * L.m[1] * L.m[2];
    L.st.assign((size_t)NS * L.nv, 0.0);
    const int nc = 1 << dim;
    double h[3] = {1.0 / n[0], 1.0 / n[1], dim == 3 ? 1.0 / n[2] : 1.0};
    std::vector<double> Ke(nc * nc, 0.0);
    for (int A = 0; A < nc; ++A)
        for (int B = 0; B < nc; ++B) {
            double s = 0.0;
            for (int k = 0; k < dim; ++k) {
                double t = 1.0;
                for (int a = 0; a < dim; ++a) {
                    const int ia = (A >> a) & 1, ib = (B >> a) & 1;
                    if (a == k)
                        t *= (ia == ib ? 1.0 : -1.0) / h[a];
                    else
                        t *= (ia == ib ? 2.0 : 1.0) * h[a] / 6.0;
                }
                s += t;
            }
            Ke[A * nc + B] = s;
        }
    // gather per vertex (no races): vertex v collects from its 2^d cells
    parallel_for(L.nv, [&](int64_t v) {
        int c[3] = {(int)(v % L.m[0]), (int)((v / L.m[0]) % L.m[1]), (int)(v / ((int64_t)L.m[0] * L.m[1]))};
        int vv[3] = {c[0] + 1, c[1] + 1, c[2] + 1};   // vertex index per axis
        for (int a = 0; a < nc; ++a) {
            // cell with lower corner vv - 1 + a; the vertex is its corner A = ~a
            int cc[3] = {0, 0, 0};
            for (int d = 0; d < dim; ++d) cc[d] = vv[d] - 1 + ((a >> d) & 1);
            const int64_t cell = cc[0] + (int64_t)n[0] * (cc[1] + (dim == 3 ? (int64_t)n[1] * cc[2] : 0));
            const int A = (~a) & (nc - 1);
            for (int B = 0; B < nc; ++B) {
                int w[3] = {1, 1, 1}, off[3] = {0, 0, 0};
                bool inside = true;
                for (int d = 0; d < dim; ++d) {
                    w[d] = cc[d] + ((B >> d) & 1);
                    off[d] = w[d] - vv[d];
                    inside = inside && w[d] >= 1 && w[d] <= n[d] - 1;
                }
                if (!inside) continue;
                const int k = (off[0] + 1) + 3 * (off[1] + 1) + (dim == 3 ? 9 * (off[2] + 1) : 0);
                L.st[(size_t)k * L.nv + v] += kappa[cell] * Ke[A * nc + B];
            }
        }
    });
}

// Galerkin coarsening A_c = P_h^T A_f P_h on stencils (row I of A_c gathered
// from the fine children of I; the coarse stencil stays 3^d-point).
static void build_coarse(int dim, CGLevelHost &F, CGLevelHost &C) {
    const int NS = stencil_size(dim);
    for (int a = 0; a < 3; ++a) {
        C.n[a] = a < dim ? F.mc[a] : 1;
        C.m[a] = a < dim ? F.mc[a] - 1 : 1;
    }
    C.nv = (int64_t)C.m[0] * C.m[1] * C.m[2];
    C.st.assign((size_t)NS * C.nv, 0.0);
    parallel_for(C.nv, [&](int64_t I) {
        int Ic[3] = {(int)(I % C.m[0]), (int)((I / C.m[0]) % C.m[1]), (int)(I / ((int64_t)C.m[0] * C.m[1]))};
        int st0[3], cnt[3];
        for (int a = 0; a < 3; ++a) {
            if (a < dim) {
                st0[a] = F.rs_start[a][Ic[a]];
                cnt[a] = F.rs_cnt[a][Ic[a]];
            } else {
                st0[a] = 0;
                cnt[a] = 1;
            }
        }
        double acc[27] = {0};
        for (int kz = 0; kz < cnt[2]; ++kz)
            for (int ky = 0; ky < cnt[1]; ++ky)
                for (int kx = 0; kx < cnt[0]; ++kx) {
                    const int fi[3] = {st0[0] + kx, st0[1] + ky, st0[2] + kz};
                    double wi = F.rs_w[0][Ic[0] * 5 + kx] * F.rs_w[1][Ic[1] * 5 + ky];
                    if (dim == 3) wi *= F.rs_w[2][Ic[2] * 5 + kz];
                    const int64_t iv = fi[0] + (int64_t)F.m[0] * (fi[1] + (int64_t)F.m[1] * fi[2]);
                    for (int s = 0; s < NS; ++s) {
                        const int so[3] = {s % 3 - 1, (s / 3) % 3 - 1, dim == 3 ? s / 9 - 1 : 0};
                        int fj[3];
                        bool inside = true;
                        for (int a = 0; a < 3; ++a) {
                            fj[a] = fi[a] + so[a];
                            if (a < dim) inside = inside && fj[a] >= 0 && fj[a] < F.m[a];
                        }
                        if (!inside) continue;
                        const double Aij = F.st[(size_t)s * F.nv + iv];
                        if (Aij == 0.0) continue;
                        // coarse parents of fine vertex j
                        int par[3][2];
                        double pw[3][2];
                        for (int a = 0; a < 3; ++a) {
                            if (a < dim) {
                                par[a][0] = F.pl_lo[a][fj[a]];
                                pw[a][0] = F.pl_wlo[a][fj[a]];
                                par[a][1] = F.pl_hi[a][fj[a]];
                                pw[a][1] = F.pl_whi[a][fj[a]];
                            } else {
                                par[a][0] = 0;
                                pw[a][0] = 1.0;
                                par[a][1] = -1;
                                pw[a][1] = 0.0;
                            }
                        }
                        for (int z = 0; z < 2; ++z) {
                            if (par[2][z] < 0) continue;
                            for (int y = 0; y < 2; ++y) {
                                if (par[1][y] < 0) continue;
                                for (int x = 0; x < 2; ++x) {
                                    if (par[0][x] < 0) continue;
                                    const int o[3] = {par[0][x] - Ic[0], par[1][y] - Ic[1], par[2][z] - Ic[2]};
                                    const int k = (o[0] + 1) + 3 * (o[1] + 1) + (dim == 3 ? 9 * (o[2] + 1) : 0);
                                    acc[k] += wi * Aij * pw[0][x] * pw[1][y] * pw[2][z];
                                }
                            }
                        }
                    }
                }
        for (int s = 0; s < NS; ++s) C.st[(size_t)s * C.nv + I] = acc[s];
    });
}

}  // namespace dgmg

namespace dgmg {

int exact_block(const dgmg_ctx &C) { return C.opts.block_inverse == DGMG_BLOCK_EXACT ? 1 : 0; }

template <typename T>
void fill_const(const dgmg_ctx &C, const DGSpace &S, DGConst<T> &c) {
    std::memset(&c, 0, sizeof(c));
    const int q = S.q;
    for (int a = 0; a < 3; ++a) c.n[a] = C.n[a];
    c.ncell = C.ncell;
    for (int a = 0; a < C.dim; ++a) {
        const double h = 1.0 / C.n[a];
        for (int i = 0; i < q * q; ++i) {
            c.M[a][i] = (T)(S.re.M[i] * h / 2.0);
            c.K[a][i] = (T)(S.re.K[i] * 2.0 / h);
        }
        for (int i = 0; i < q; ++i) {
            c.d0[a][i] = (T)(S.re.d0[i] * 2.0 / h);
            c.dp[a][i] = (T)(S.re.dp[i] * 2.0 / h);
        }
        c.gamma[a] = (T)(2.0 * S.penalty_p * (S.penalty_p + 1) / h);
    }
    for (int i = 0; i < q; ++i) {
        c.hat[0][i] = (T)((1.0 - S.re.nodes[i]) / 2.0);
        c.hat[1][i] = (T)((1.0 + S.re.nodes[i]) / 2.0);
        c.v0[i] = (T)S.re.e0[i];
        c.vp[i] = (T)S.re.ep[i];
    }
    c.gl = S.re.basis == DGMG_BASIS_GL ? 1 : 0;
    c.omega = (T)C.opts.omega_dg;
    // M_ref = diag(w) + sigma l l^T: w the row sums (the lumped quadrature
    // weights), l_i = 1 / prod_{m != i} (x_i - x_m) the leading coefficient of
    // the basis function l_i, sigma from the first entry (sigma <= 0)
    std::vector<double> w(q, 0.0), lc(q, 1.0);
    for (int i = 0; i < q; ++i) {
        for (int j = 0; j < q; ++j) w[i] += S.re.M[i * q + j];
        for (int m = 0; m < q; ++m)
            if (m != i) lc[i] /= S.re.nodes[i] - S.re.nodes[m];
    }
    const double sigma = std::min(0.0, (S.re.M[0] - w[0]) / (lc[0] * lc[0]));
    for (int a = 0; a < C.dim; ++a) {
        const double h = 1.0 / C.n[a];
        for (int i = 0; i < q; ++i) {
            c.mw[a][i] = (T)(w[i] * h / 2.0);
            c.mu[a][i] = (T)(std::sqrt(-sigma * h / 2.0) * lc[i]);
        }
    }
}

// Input of the device kernel that computes the per-cell fast-diagonalisation
// factors of the exact diagonal blocks (Kt_a = kappa_K K_a + the own-face terms
// of the two faces normal to axis a, Sec. 4.1; Kt_a S = M_a S diag(lambda),
// S^T M_a S = I): the h-scaled 1D data of space S per axis.
static int fd_input(const dgmg_ctx &C, const DGSpace &S, FDInput &in) {
    std::memset(&in, 0, sizeof(in));
    const int q = S.q;
    in.dim = C.dim;
    in.q = q;
    in.interior_only = C.opts.block_inverse == DGMG_BLOCK_INTERIOR_ONLY ? 1 : 0;
    for (int a = 0; a < 3; ++a) in.n[a] = C.n[a];
    for (int i = 0; i < q; ++i) {
        in.e0[i] = S.re.e0[i];
        in.ep[i] = S.re.ep[i];
    }
    for (int a = 0; a < C.dim; ++a) {
        const double h = 1.0 / C.n[a];
        double Mh[QMAX * QMAX];
        for (int i = 0; i < q * q; ++i) {
            Mh[i] = S.re.M[i] * h / 2.0;
            in.Kh[a][i] = S.re.K[i] * 2.0 / h;
        }
        for (int i = 0; i < q; ++i) {
            in.d0[a][i] = S.re.d0[i] * 2.0 / h;
            in.dp[a][i] = S.re.dp[i] * 2.0 / h;
        }
        in.gam[a] = 2.0 * S.penalty_p * (S.penalty_p + 1) / h;
        if (!cholesky_inverse_lower(q, Mh, in.Linv[a])) return fail(DGMG_EINVAL, "1D mass matrix not SPD");
    }
    return DGMG_OK;
}

template <typename T>
std::vector<T> convert(const std::vector<double> &v) {
    return std::vector<T>(v.begin(), v.end());
}

// The per-cell factors (and, FP64, the table of inverse eigenvalue sums) of
// level D from the FP64 kappa of the finest level, on the set-up stream.
// FP32 factors are the rounded FP64 ones when those exist (fd64).
template <typename T>
int compute_factors(dgmg_ctx &C, const DGSpace &S, DGDev<T> &D, const double *fd64 = nullptr) {
    // the residual's factors [S^T M | lambda], from the FP64 factors where there are some
    MassTables mt;
    std::memset(&mt, 0, sizeof(mt));
    for (int a = 0; a < C.dim; ++a) {
        const double h = 1.0 / C.n[a];
        for (int i = 0; i < S.q * S.q; ++i) mt.M[a][i] = S.re.M[i] * h / 2.0;
    }
    if (std::is_same<T, float>::value && fd64) {
        LC(launch_cast_d2f((int64_t)C.ncell * C.dim * (S.q * S.q + S.q), fd64, reinterpret_cast<float *>(D.fd),
                           C.setup_stream));
        if (D.fdr)
            LC((launch_residual_factors<double, float>(C.dim, S.q, C.ncell, fd64, mt,
                                                       reinterpret_cast<float *>(D.fdr), C.setup_stream)));
        return DGMG_OK;
    }
    FDInput in;
    RC(fd_input(C, S, in));
    const_cast<DGSpace &>(S).fdin = in;
    LC(launch_fd_factors<T>(in, C.d64.kappa, C.ncell, D.fd, C.setup_stream));
    if (sizeof(T) == sizeof(double))
        LC(launch_inverse_eigen_sums(C.dim, S.q, C.ncell, reinterpret_cast<const double *>(D.fd),
                                     C.opts.omega_dg, reinterpret_cast<double *>(D.linv), C.setup_stream));
    if (D.fdr) LC((launch_residual_factors<T, T>(C.dim, S.q, C.ncell, D.fd, mt, D.fdr, C.setup_stream)));
    return DGMG_OK;
}

// The "recompute" variant of the block inverse (Table 6, opts.recompute_block):
// the level's per-cell factors (and, FP64, the table of inverse eigenvalue
// sums) computed again on stream s, before a smoothing step, from the same
// input as at set-up; the residual's factors stay the set-up ones.
template <typename T>
int recompute_factors(dgmg_ctx &C, const DGSpace &S, DGDev<T> &D, cudaStream_t s) {
    if (!D.fd) return DGMG_OK;
    LC(launch_fd_factors<T>(S.fdin, C.d64.kappa, C.ncell, D.fd, s));
    if (sizeof(T) == sizeof(double) && D.linv)
        LC(launch_inverse_eigen_sums(C.dim, S.q, C.ncell, reinterpret_cast<const double *>(D.fd),
                                     C.opts.omega_dg, reinterpret_cast<double *>(D.linv), s));
    return DGMG_OK;
}

// One DG level in precision T: constants, kappa (uploaded, or shared with the
// finest level), the per-cell factors computed on the device from the FP64
// kappa of the finest level (C.d64.kappa, uploaded first), the FP64 table of
// inverse eigenvalue sums, traces and corner sums.
template <typename T>
int setup_dg(dgmg_ctx &C, const DGSpace &S, DGDev<T> &D, const std::vector<double> &kappa, bool smoother = true,
             const T *shared_kappa = nullptr, const double *fd64 = nullptr, const T *shared_kfac = nullptr) {
    fill_const(C, S, D.c);
    if (shared_kappa)
        D.kappa = const_cast<T *>(shared_kappa);
    else
        RC(C.upload(&D.kappa, convert<T>(kappa)));
    // facet coefficients (from the FP64 kappa of the finest level, uploaded first)
    if (shared_kfac) {
        D.kfac = const_cast<T *>(shared_kfac);
    } else {
        RC(C.alloc(&D.kfac, C.ncell * 2 * C.dim));
        LC(launch_facet_coefficients<T>(C.dim, C.n, C.ncell, C.d64.kappa, D.kfac, C.setup_stream));
    }
    D.c.kfac = D.kfac;
    const int64_t trn = C.ncell * 2 * C.dim * trace_face_stride<T>((int)(S.nloc / S.q));
    if (!smoother) {                  // operator only (projection, residual): no block-inverse factors
        RC(C.alloc(&D.tr[0], trn));
        RC(C.alloc(&D.tr[1], trn));
        RC(C.alloc(&D.corners, C.ncell * (1 << C.dim)));
        return DGMG_OK;
    }
    RC(C.alloc(&D.fd, (size_t)C.ncell * C.dim * (S.q * S.q + S.q)));
    RC(C.alloc(&D.fdr, (size_t)C.ncell * C.dim * (S.q * S.q + S.q)));
    if (sizeof(T) == sizeof(double)) RC(C.alloc(&D.linv, (size_t)S.ndof));
    RC(compute_factors<T>(C, S, D, fd64));
    RC(C.alloc(&D.tr[0], trn));
    RC(C.alloc(&D.tr[1], trn));
    RC(C.alloc(&D.corners, C.ncell * (1 << C.dim)));
    return DGMG_OK;
}

// The lower DG levels of a gradual p-hierarchy (degrees p-1 .. 1, finest
// penalty): fast-diagonalisation factors, constants, traces, the level's
// vectors and the interpolation up to the next finer level, in FP64 and (mixed
// precision) FP32; the finest residual scratch. dgs[0] (the finest space) is
// always set.
int setup_dg_levels(dgmg_ctx &C, const std::vector<double> &kap) {
    C.dgs.assign(1, finest_space(C));
    if (C.opts.p_coarsening == 0 || C.p < 2) return DGMG_OK;
    const bool mixed = C.opts.precision == DGMG_MIXED_FP32;
    for (int pc = C.p - 1; pc >= 1; --pc) {
        DGSpace S;
        S.p = pc;
        S.q = pc + 1;
        S.penalty_p = C.p;
        S.nloc = C.dim == 3 ? (int64_t)S.q * S.q * S.q : (int64_t)S.q * S.q;
        S.ndof = C.ncell * S.nloc;
        S.re = make_refelem(pc, C.opts.basis);
        C.dgs.push_back(S);
    }
    const int L = (int)C.dgs.size();
    C.lvl64.resize(L);
    if (mixed) C.lvl32.resize(L);
    for (int l = 1; l < L; ++l) {
        const DGSpace &S = C.dgs[l], &F = C.dgs[l - 1];
        // I[i][j] = l_j(x_i): this level's basis at the finer level's nodes
        std::vector<double> I((size_t)F.q * S.q), val(S.q);
        for (int i = 0; i < F.q; ++i) {
            lagrange_at(S.re.nodes, F.re.nodes[i], val.data(), nullptr);
            for (int j = 0; j < S.q; ++j) I[(size_t)i * S.q + j] = val[j];
        }
        auto level = [&](auto &lv, auto *kappa_dev, const double *fd64, decltype(kappa_dev) kfac_dev) -> int {
            using T = typename std::remove_pointer<decltype(kappa_dev)>::type;
            RC(setup_dg<T>(C, S, lv.D, kap, true, kappa_dev, fd64, kfac_dev));
            RC(C.alloc(&lv.z, S.ndof));
            RC(C.alloc(&lv.b, S.ndof));
            RC(C.alloc(&lv.r, S.ndof));
            std::memset(&lv.P, 0, sizeof(lv.P));
            for (size_t k = 0; k < I.size(); ++k) lv.P.I[k] = (T)I[k];
            return DGMG_OK;
        };
        RC(level(C.lvl64[l], C.d64.kappa, nullptr, C.d64.kfac));
        if (mixed) RC(level(C.lvl32[l], C.d32.kappa, C.lvl64[l].D.fd, C.d32.kfac));
    }
    RC(C.alloc(&C.res64, C.ndof));
    if (mixed) RC(C.alloc(&C.res32, C.ndof));
    return DGMG_OK;
}

template <typename T>
int setup_cg(dgmg_ctx &C, std::vector<CGDev<T>> &out) {
    const int nl = (int)C.lv.size();
    out.resize(nl);
    for (int l = 0; l < nl; ++l) {
        CGLevelHost &H = C.lv[l];
        CGDev<T> &D = out[l];
        std::memset(&D.L, 0, sizeof(D.L));
        for (int a = 0; a < 3; ++a) {
            D.L.m[a] = H.m[a];
            D.L.mc[a] = H.mc[a] > 0 ? H.mc[a] - 1 : 0;
        }
        D.L.nv = H.nv;
        RC(C.upload(&D.st, convert<T>(H.st)));
        D.L.st = D.st;
        RC(C.alloc(&D.u[0], H.nv));
        RC(C.alloc(&D.u[1], H.nv));
        RC(C.alloc(&D.b, H.nv));
        RC(C.alloc(&D.r, H.nv));
        if (l + 1 < nl) {
            std::vector<int> it;
            std::vector<double> wt;
            size_t off_i[3][4], off_w[3][3];
            for (int a = 0; a < C.dim; ++a) {
                off_i[a][0] = it.size();
                it.insert(it.end(), H.pl_lo[a].begin(), H.pl_lo[a].end());
                off_i[a][1] = it.size();
                it.insert(it.end(), H.pl_hi[a].begin(), H.pl_hi[a].end());
                off_i[a][2] = it.size();
                it.insert(it.end(), H.rs_start[a].begin(), H.rs_start[a].end());
                off_i[a][3] = it.size();
                it.insert(it.end(), H.rs_cnt[a].begin(), H.rs_cnt[a].end());
                off_w[a][0] = wt.size();
                wt.insert(wt.end(), H.pl_wlo[a].begin(), H.pl_wlo[a].end());
                off_w[a][1] = wt.size();
                wt.insert(wt.end(), H.pl_whi[a].begin(), H.pl_whi[a].end());
                off_w[a][2] = wt.size();
                wt.insert(wt.end(), H.rs_w[a].begin(), H.rs_w[a].end());
            }
            RC(C.upload(&D.itab, it));
            RC(C.upload(&D.wtab, convert<T>(wt)));
            for (int a = 0; a < C.dim; ++a) {
                D.L.pl_lo[a] = D.itab + off_i[a][0];
                D.L.pl_hi[a] = D.itab + off_i[a][1];
                D.L.rs_start[a] = D.itab + off_i[a][2];
                D.L.rs_cnt[a] = D.itab + off_i[a][3];
                D.L.pl_wlo[a] = D.wtab + off_w[a][0];
                D.L.pl_whi[a] = D.wtab + off_w[a][1];
                D.L.rs_w[a] = D.wtab + off_w[a][2];
            }
            for (int a = 0; a < 3; ++a) D.L.mc[a] = a < C.dim ? H.mc[a] - 1 : 1;
        }
    }
    return DGMG_OK;
}

// The Q1 levels for kappa: the Galerkin level-0 operator P^T A P and the
// coarsenings by factor f while some axis can be coarsened.
static void build_q1_levels(int dim, const int *n, int f, const std::vector<double> &kap,
                            std::vector<CGLevelHost> &lv) {
    lv.clear();
    lv.emplace_back();
    build_level0(dim, n, kap, lv[0]);
    for (;;) {
        CGLevelHost &F = lv.back();
        bool any = false;
        for (int a = 0; a < dim; ++a) any = any || can_coarsen(F.n[a], f);
        if (!any) break;
        for (int a = 0; a < dim; ++a) {
            int nc = 0;
            axis_tables(F.n[a], f, F, a, nc);
            F.mc[a] = nc;
        }
        CGLevelHost Cl;
        build_coarse(dim, F, Cl);
        lv.push_back(std::move(Cl));
    }
}

// dense inverse of the coarsest operator via Cholesky (FP64, host)
int coarse_inverse(dgmg_ctx &C, std::vector<double> &inv) {
    const CGLevelHost &L = C.lv.back();
    const int64_t nc = L.nv;
    if (nc > 4096) return fail(DGMG_EINVAL, "coarsest level has more than 4096 unknowns");
    C.ncoarse = nc;
    std::vector<double> A((size_t)nc * nc, 0.0);
    const int NS = stencil_size(C.dim);
    for (int64_t v = 0; v < nc; ++v) {
        int c[3] = {(int)(v % L.m[0]), (int)((v / L.m[0]) % L.m[1]), (int)(v / ((int64_t)L.m[0] * L.m[1]))};
        for (int s = 0; s < NS; ++s) {
            const int o[3] = {s % 3 - 1, (s / 3) % 3 - 1, C.dim == 3 ? s / 9 - 1 : 0};
            int w[3];
            bool inside = true;
            for (int a = 0; a < 3; ++a) {
                w[a] = c[a] + o[a];
                inside = inside && w[a] >= 0 && w[a] < L.m[a];
            }
            if (!inside) continue;
            const int64_t wi = w[0] + (int64_t)L.m[0] * (w[1] + (int64_t)L.m[1] * w[2]);
            A[v * nc + wi] += L.st[(size_t)s * L.nv + v];
        }
    }
    // Cholesky A = L L^T in place (lower)
    std::vector<double> Lc((size_t)nc * nc, 0.0);
    for (int64_t j = 0; j < nc; ++j) {
        double s = A[j * nc + j];
        for (int64_t k = 0; k < j; ++k) s -= Lc[j * nc + k] * Lc[j * nc + k];
        if (!(s > 0.0)) return fail(DGMG_EINVAL, "coarsest operator is not positive definite");
        Lc[j * nc + j] = std::sqrt(s);
        for (int64_t i = j + 1; i < nc; ++i) {
            double t = A[i * nc + j];
            for (int64_t k = 0; k < j; ++k) t -= Lc[i * nc + k] * Lc[j * nc + k];
            Lc[i * nc + j] = t / Lc[j * nc + j];
        }
    }
    // inverse column by column: solve L y = e_c, L^T x = y
    inv.assign((size_t)nc * nc, 0.0);
    std::vector<double> y(nc);
    for (int64_t c = 0; c < nc; ++c) {
        for (int64_t i = 0; i < nc; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int64_t k = 0; k < i; ++k) s -= Lc[i * nc + k] * y[k];
            y[i] = s / Lc[i * nc + i];
        }
        for (int64_t i = nc - 1; i >= 0; --i) {
            double s = y[i];
            for (int64_t k = i + 1; k < nc; ++k) s -= Lc[k * nc + i] * inv[k * nc + c];
            inv[i * nc + c] = s / Lc[i * nc + i];
        }
    }
    return DGMG_OK;
}

// ------------------------------------------------------------ V-cycle

// h-multigrid V-cycle on Q1 level l with zero initial guess; RHS in cg[l].b.
// Returns the buffer holding the result.
template <typename T>
int cg_vcycle(dgmg_ctx &C, int l, cudaStream_t s, T **result) {
    auto &lv = cgl<T>(C);
    CGDev<T> &L = lv[l];
    const T om = (T)C.opts.omega_cg;
    if (l == (int)lv.size() - 1) {
        LC(launch_coarse_solve<T>(L.L.nv, C.coarse_inv, L.b, L.u[0], s));
        *result = L.u[0];
        return DGMG_OK;
    }
    int cur = 0;
    bool zero = true;
    for (int k = 0; k < C.opts.nu_pre; ++k) {
        LC(launch_cg_jacobi<T>(C.dim, L.L, L.u[cur], L.b, L.u[cur ^ 1], om, zero, s));
        zero = false;
        cur ^= 1;
    }
    if (zero) {
        LC(cudaMemsetAsync(L.u[cur], 0, sizeof(T) * L.L.nv, s));
        zero = false;
    }
    LC(launch_cg_residual<T>(C.dim, L.L, L.u[cur], L.b, L.r, s));
    LC(launch_h_restrict<T>(C.dim, L.L, L.r, lv[l + 1].b, s));
    T *ec = nullptr;
    RC(cg_vcycle<T>(C, l + 1, s, &ec));
    LC(launch_h_prolong<T>(C.dim, L.L, ec, L.u[cur], s));
    for (int k = 0; k < C.opts.nu_post; ++k) {
        LC(launch_cg_jacobi<T>(C.dim, L.L, L.u[cur], L.b, L.u[cur ^ 1], om, false, s));
        cur ^= 1;
    }
    *result = L.u[cur];
    return DGMG_OK;
}

// The whole Q1 cycle from level 0 (RHS in cg[0].b) as one cooperative launch
// when the context has its plan; the launch per step otherwise.
template <typename T>
int q1_cycle(dgmg_ctx &C, cudaStream_t s, T **result) {
    auto &lv = cgl<T>(C);
    Q1Plan<T> *plan = q1plan<T>(C);
    if (!plan || C.q1_blocks <= 0 || g_q1_one_launch_off.load(std::memory_order_relaxed))
        return cg_vcycle<T>(C, 0, s, result);
    const int pi = std::is_same<T, float>::value ? 1 : 0;
    LC(launch_q1_cycle<T>(C.dim, plan, C.q1bar + pi, C.q1_blocks_t[pi], C.q1_wide, s));
    *result = lv.size() == 1 ? lv[0].u[0] : lv[0].u[(C.opts.nu_pre + C.opts.nu_post) & 1];
    return DGMG_OK;
}

// The cooperative Q1 cycle is used when the kernels of both precisions in use
// can be launched co-resident (> 0); each precision launches as many blocks as
// its kernel keeps co-resident (q1_blocks_t; every launch on a plan's arrival
// counter has the same block count); 0 where the launch is not possible.
static int q1_blocks_for(int dim, bool mixed) {
    int qb = q1_cycle_max_blocks<double>(dim, false);
    if (mixed) qb = std::min(qb, q1_cycle_max_blocks<float>(dim, false));
    return std::max(0, qb);
}

// Build the plan of q1_cycle for precision T. The cooperative launch is kept
// only if it can also be captured into a CUDA graph (the solve replays its
// iterations as graphs); otherwise the Q1 levels keep one launch per step.
template <typename T>
int setup_q1_plan(dgmg_ctx &C) {
    auto &lv = cgl<T>(C);
    const int nl = (int)lv.size();
    if (nl == 0 || nl > Q1_MAXLEV || C.q1_blocks <= 0) return DGMG_OK;
    Q1Plan<T> h;
    std::memset(&h, 0, sizeof(h));
    h.nlev = nl;
    h.nu_pre = C.opts.nu_pre;
    h.nu_post = C.opts.nu_post;
    h.omega = (T)C.opts.omega_cg;
    h.ncoarse = lv[nl - 1].L.nv;
    // the trailing levels small enough for one block: up to 512 vertices in
    // FP32; in FP64 (about 2 FMA per clock per SM) only a one-vertex coarsest
    // level (measured on the 32^3, p = 3 hierarchy: a 27-vertex level is
    // faster on the whole grid, 146 against 159 us per cycle)
    const int64_t local_max = std::is_same<T, float>::value ? 512 : 1;
    h.local_from = nl;
    while (h.local_from > 0 && lv[h.local_from - 1].L.nv <= local_max) --h.local_from;
    h.Ainv = C.coarse_inv;
    for (int l = 0; l < nl; ++l) {
        h.L[l] = lv[l].L;
        h.u0[l] = lv[l].u[0];
        h.u1[l] = lv[l].u[1];
        h.b[l] = lv[l].b;
        h.r[l] = lv[l].r;
    }
    Q1Plan<T> *d = nullptr;
    RC(C.upload(&d, std::vector<Q1Plan<T>>{h}));
    if (!C.q1bar) {
        RC(C.alloc(&C.q1bar, 2));
        DG_CUDA(cudaMemsetAsync(C.q1bar, 0, 2 * sizeof(unsigned long long), C.setup_stream));
    }
    static std::atomic<int> capture_ok{-1};   // per precision: unknown, no, yes
    if (capture_ok.load() < 0 && C.capture_stream) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        bool ok = cudaStreamBeginCapture(C.capture_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            const int pi = std::is_same<T, float>::value ? 1 : 0;
            const cudaError_t el =
                launch_q1_cycle<T>(C.dim, d, C.q1bar + pi, C.q1_blocks_t[pi], C.q1_wide, C.capture_stream);
            g_kernel_launches.fetch_sub(1);   // captured, not launched
            const cudaError_t ee = cudaStreamEndCapture(C.capture_stream, &graph);
            ok = el == cudaSuccess && ee == cudaSuccess && graph &&
                 cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        capture_ok.store(ok ? 1 : 0);
    }
    if (capture_ok.load() == 1) q1plan<T>(C) = d;   // else the plan stays unused
    return DGMG_OK;
}

// DG level l of the hierarchy in precision T (0 = the finest), and its tiles
// (the finest level's tuned ones; launcher defaults below).
template <typename T>
DGDev<T> &dg_level(dgmg_ctx &C, int l) {
    return l == 0 ? dg<T>(C) : dglevels<T>(C)[l].D;
}

template <typename T>
int level_smooth(dgmg_ctx &C, int l, T *z, const T *b, int cur, cudaStream_t s) {
    DGDev<T> &D = dg_level<T>(C, l);
    C.prof.begin(ST_SMOOTH, s);
    if (C.opts.recompute_block) RC(recompute_factors<T>(C, C.dgs[l], D, s));
    LC(launch_smooth<T>(C.dim, C.dgs[l].q, D.c, l == 0 ? C.tile_of<T>(TILE_SMOOTH) : 0, exact_block(C), z, b,
                        D.kappa, D.fd, D.linv, D.tr[cur], D.tr[cur ^ 1], s));
    C.prof.end(s);
    return DGMG_OK;
}

template <typename T>
int level_cycle(dgmg_ctx &C, int l, const T *b, T *z, cudaStream_t s);

// Coarse-grid correction of the iterate z of DG level l for the right-hand side
// b, whose projections are in tr[cur]: the residual is restricted to the next
// level (the next DG level, or the Q1 levels below the last one), solved there
// by one cycle with zero initial guess, and the correction is prolongated into
// z; the projections of the new z end in tr[0].
template <typename T>
int coarse_correction(dgmg_ctx &C, int l, T *z, const T *b, int cur, cudaStream_t s) {
    DGDev<T> &D = dg_level<T>(C, l);
    const DGSpace &S = C.dgs[l];
    const int tres = l == 0 ? C.tile_of<T>(TILE_RESIDUAL) : 0, tproj = l == 0 ? C.tile_of<T>(TILE_PROJECT) : 0;
    if (l == (int)C.dgs.size() - 1) {
        C.prof.begin(ST_RESIDUAL, s);
        LC(launch_residual<T>(C.dim, S.q, D.c, tres, RES_HAS_B | RES_CORNERS, z, b, D.kappa, D.tr[cur], nullptr,
                              D.corners, exact_fd(C, D), s));
        C.prof.end(s);
        auto &lv = cgl<T>(C);
        C.prof.begin(ST_CG, s);
        LC(launch_corner_gather<T>(C.dim, C.n, D.corners, lv[0].b, s));
        T *e0 = nullptr;
        RC(q1_cycle<T>(C, s, &e0));
        C.prof.end(s);
        C.prof.begin(ST_PROJECT, s);
        LC(launch_project<T>(C.dim, S.q, D.c, tproj, z, e0, D.tr[0], s));   // z += P e0
        C.prof.end(s);
        return DGMG_OK;
    }
    auto &lvl = dglevels<T>(C);
    DGLevelDev<T> &N = lvl[l + 1];
    T *res = l == 0 ? (std::is_same<T, float>::value ? (T *)C.res32 : (T *)C.res64) : lvl[l].r;
    C.prof.begin(ST_RESIDUAL, s);
    LC(launch_residual<T>(C.dim, S.q, D.c, tres, RES_HAS_B | RES_WRITE_R, z, b, D.kappa, D.tr[cur], res, nullptr,
                          exact_fd(C, D), s));
    C.prof.end(s);
    C.prof.begin(ST_CG, s);
    LC(launch_dg_transfer<T>(C.dim, S.q, false, C.ncell, N.P, res, N.b, s));
    C.prof.end(s);
    RC(level_cycle<T>(C, l + 1, N.b, N.z, s));
    C.prof.begin(ST_CG, s);
    LC(launch_dg_transfer<T>(C.dim, S.q, true, C.ncell, N.P, N.z, z, s));
    C.prof.end(s);
    C.prof.begin(ST_PROJECT, s);
    LC(launch_project<T>(C.dim, S.q, D.c, tproj, z, nullptr, D.tr[0], s));
    C.prof.end(s);
    return DGMG_OK;
}

// One V(nu_pre, nu_post) cycle from DG level l with zero initial guess.
template <typename T>
int level_cycle(dgmg_ctx &C, int l, const T *b, T *z, cudaStream_t s) {
    DGDev<T> &D = dg_level<T>(C, l);
    const DGSpace &S = C.dgs[l];
    const int64_t trn = C.ncell * 2 * C.dim * trace_face_stride<T>((int)(S.nloc / S.q));
    LC(cudaMemsetAsync(z, 0, sizeof(T) * S.ndof, s));
    LC(cudaMemsetAsync(D.tr[0], 0, sizeof(T) * trn, s));   // projections of z = 0
    int cur = 0;
    for (int k = 0; k < C.opts.nu_pre; ++k) {
        RC(level_smooth<T>(C, l, z, b, cur, s));
        cur ^= 1;
    }
    RC(coarse_correction<T>(C, l, z, b, cur, s));
    cur = 0;
    for (int k = 0; k < C.opts.nu_post; ++k) {
        RC(level_smooth<T>(C, l, z, b, cur, s));
        cur ^= 1;
    }
    return DGMG_OK;
}

// z = V(r) on the DG level in precision T (zero initial guess).
template <typename T>
int dg_vcycle(dgmg_ctx &C, const T *r, T *z, cudaStream_t s) {
    return level_cycle<T>(C, 0, r, z, s);
}

// One cycle of the stationary hp-multigrid iteration (Alg. 7, MGMult) in FP64:
// nu_pre block-Jacobi steps on A x = b, then the coarse-grid correction (Alg. 6:
// residual, p-restriction, one h-V-cycle on the Q1 levels, p-prolongation fused
// into the projection). D.tr[0] holds the projections of x on entry and of the
// new x on exit; r (if not NULL) receives b - A x of the new x.
int mg_cycle64(dgmg_ctx &C, double *x, const double *b, double *r, cudaStream_t s) {
    DGDev<double> &D = C.d64;
    int cur = 0;
    for (int k = 0; k < C.opts.nu_pre; ++k) {
        RC(level_smooth<double>(C, 0, x, b, cur, s));
        cur ^= 1;
    }
    RC(coarse_correction<double>(C, 0, x, b, cur, s));
    if (r) {
        C.prof.begin(ST_RESIDUAL, s);
        LC(launch_residual<double>(C.dim, C.q, D.c, C.tile[0][TILE_RESIDUAL], RES_HAS_B | RES_WRITE_R, x, b,
                                   D.kappa, D.tr[0], r, nullptr, exact_fd(C, D), s));
        C.prof.end(s);
    }
    return DGMG_OK;
}

// Projections of x into D.tr[0] (FP64), for a stationary cycle's first step.
int project64(dgmg_ctx &C, double *x, cudaStream_t s) {
    C.prof.begin(ST_PROJECT, s);
    LC(launch_project<double>(C.dim, C.q, C.d64.c, C.tile[0][TILE_PROJECT], x, nullptr, C.d64.tr[0], s));
    C.prof.end(s);
    return DGMG_OK;
}

int vcycle64(dgmg_ctx &C, const double *r, double *z, cudaStream_t s) {
    if (C.opts.precision == DGMG_MIXED_FP32) {
        C.prof.begin(ST_VECTOR, s);
        LC(launch_cast_d2f(C.ndof, r, C.r32, s));
        C.prof.end(s);
        RC(dg_vcycle<float>(C, C.r32, C.z32, s));
        C.prof.begin(ST_VECTOR, s);
        LC(launch_cast_f2d(C.ndof, C.z32, z, s));
        C.prof.end(s);
        return DGMG_OK;
    }
    return dg_vcycle<double>(C, r, z, s);
}

// y = A u (negate = false) or r = b - A u, FP64
int apply64(dgmg_ctx &C, const double *u, const double *b, double *out, cudaStream_t s) {
    DGDev<double> &D = C.d64;
    C.prof.begin(ST_PROJECT, s);
    LC(launch_project<double>(C.dim, C.q, D.c, C.tile[0][TILE_PROJECT], const_cast<double *>(u), nullptr, D.tr[0],
                              s));
    C.prof.end(s);
    const int mode = b ? (RES_HAS_B | RES_WRITE_R) : (RES_WRITE_R | RES_NEGATE);
    C.prof.begin(ST_RESIDUAL, s);
    LC(launch_residual<double>(C.dim, C.q, D.c, C.tile[0][TILE_RESIDUAL], mode, u, b, D.kappa, D.tr[0], out,
                               nullptr, exact_fd(C, D), s));
    C.prof.end(s);
    return DGMG_OK;
}

// ------------------------------------------------------------ tile autotuner
// For each DG-level kernel (projection, smoothing step, residual + restriction)
// and each precision the ctx runs, time the candidate cells-per-CTA values on
// the ctx's own buffers (one warm-up and three timed launches each, CUDA events
// on the set-up stream) and keep the fastest; for the FP32 smoothing step the
// one-thread-per-cell kernel (tile 0) competes with the pencil tiles. Results
// are cached per (dimension, degree, mesh, precision, block inverse) for the
// process, so a repeated shape is tuned once.
struct TileKey {
    int v[8];
    bool operator<(const TileKey &o) const { return std::lexicographical_compare(v, v + 8, o.v, o.v + 8); }
};
static std::mutex g_tile_mu;
static std::map<TileKey, std::array<int, 6>> g_tile_cache;

template <typename T>
static int tune_tiles(dgmg_ctx &C, T *u, T *b, int *tile, bool trace, bool smooth) {
    DGDev<T> &D = dg<T>(C);
    cudaStream_t s = C.setup_stream;
    const int nf = (int)(C.nloc / C.q);
    const int64_t trn = C.ncell * 2 * C.dim * trace_face_stride<T>(nf);
    std::vector<int> cand;
    for (int c = 1; c <= 64; c *= 2)
        if (c * nf >= 32 && c * nf <= 256) cand.push_back(c);
    // and the most cells whose pencils fit 256 threads (q = 5: 10 cells, 250
    // threads, the last warp nearly full; FP64 work of idle lanes is lost)
    if (nf <= 256 && 256 / nf * nf >= 32 && std::find(cand.begin(), cand.end(), 256 / nf) == cand.end())
        cand.push_back(256 / nf);
    if (cand.empty()) cand.push_back(C.cpb);
    DG_CUDA(cudaMemsetAsync(u, 0, sizeof(T) * C.ndof, s));
    DG_CUDA(cudaMemsetAsync(b, 0, sizeof(T) * C.ndof, s));
    DG_CUDA(cudaMemsetAsync(D.tr[0], 0, sizeof(T) * trn, s));
    DG_CUDA(cudaMemsetAsync(D.tr[1], 0, sizeof(T) * trn, s));
    cudaEvent_t e0, e1;
    DG_CUDA(cudaEventCreate(&e0));
    DG_CUDA(cudaEventCreate(&e1));
    const float INF = 1e30f;
    // milliseconds of three launches, INF if the shape cannot launch
    auto time_it = [&](auto launch) -> float {
        if (launch() != cudaSuccess) {
            cudaGetLastError();
            return INF;
        }
        cudaEventRecord(e0, s);
        for (int k = 0; k < 3; ++k)
            if (launch() != cudaSuccess) {
                cudaGetLastError();
                return INF;
            }
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return INF;
        float ms = INF;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    const char *tname = sizeof(T) == 8 ? "fp64" : "fp32";
    // the fastest candidate; the one-thread-per-cell kernel (tile 0) is kept
    // unless another tile is more than 3% faster, so that a near tie in the
    // three-launch timing does not flip the choice from run to run
    auto pick = [&](const char *stage, std::vector<int> cs, auto launch_with) {
        int best = cs[0];
        float best_ms = INF, ms0 = INF;
        for (int c : cs) {
            const float ms = time_it([&] { return launch_with(c); });
            if (trace) std::fprintf(stderr, "dgmg autotune %s %-9s tile %2d: %8.4f ms\n", tname, stage, c, ms / 3);
            if (c == 0) ms0 = ms;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        return ms0 < INF && ms0 <= 1.03f * best_ms ? 0 : best;
    };
    std::vector<int> cp = cand;
    if (C.dim == 3 && C.q <= (std::is_same<T, float>::value ? 5 : 4) && C.opts.basis == DGMG_BASIS_GLL)
        cp.insert(cp.begin(), 0);
    tile[TILE_PROJECT] = pick("project", cp, [&](int c) {
        return launch_project<T>(C.dim, C.q, D.c, c, u, nullptr, D.tr[0], s);
    });
    std::vector<int> cs = cand;
    if (C.dim == 3 && C.q <= (std::is_same<T, float>::value ? 5 : 4) && exact_block(C)) cs.insert(cs.begin(), 0);
    if (smooth)                     // (the FP64 smoother of a mixed-precision context never runs)
        tile[TILE_SMOOTH] = pick("smooth", cs, [&](int c) {
            return launch_smooth<T>(C.dim, C.q, D.c, c, exact_block(C), u, b, D.kappa, D.fd, D.linv, D.tr[0],
                                    D.tr[1], s);
        });
    std::vector<int> cr = cand;
    if (C.dim == 3 && C.q <= (std::is_same<T, float>::value ? 5 : 4) && exact_fd(C, D)) cr.insert(cr.begin(), 0);
    tile[TILE_RESIDUAL] = pick("residual", cr, [&](int c) {
        return launch_residual<T>(C.dim, C.q, D.c, c, RES_HAS_B | RES_CORNERS, u, b, D.kappa, D.tr[0], nullptr,
                                  D.corners, exact_fd(C, D), s);
    });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    DG_CUDA(cudaStreamSynchronize(s));
    return DGMG_OK;
}

static int autotune_tiles(dgmg_ctx &C) {
    const bool mixed = C.opts.precision == DGMG_MIXED_FP32;
    const TileKey key{{C.dim, C.q, C.n[0], C.n[1], C.n[2], C.opts.precision, C.opts.block_inverse, C.opts.basis}};
    {
        std::lock_guard<std::mutex> lk(g_tile_mu);
        auto it = g_tile_cache.find(key);
        if (it != g_tile_cache.end()) {
            for (int k = 0; k < 6; ++k) C.tile[k / 3][k % 3] = it->second[k];
            return DGMG_OK;
        }
    }
    const bool trace = std::getenv("DGMG_TRACE_SETUP") != nullptr;
    RC(tune_tiles<double>(C, C.w_z, C.w_r, C.tile[0], trace, !mixed));
    if (mixed) RC(tune_tiles<float>(C, C.z32, C.r32, C.tile[1], trace, true));
    std::array<int, 6> v;
    for (int k = 0; k < 6; ++k) v[k] = C.tile[k / 3][k % 3];
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tile_cache[key] = v;
    return DGMG_OK;
}

int check_ctx(const dgmg_ctx *C) {
    if (!C) return fail(DGMG_EINVAL, "ctx is NULL");
    return DGMG_OK;
}

template int dg_vcycle<double>(dgmg_ctx &, const double *, double *, cudaStream_t);
template int dg_vcycle<float>(dgmg_ctx &, const float *, float *, cudaStream_t);

}  // namespace dgmg

// ============================================================== C ABI
extern "C" {

const char *dgmg_version(void) { return "libdgmg 0.1 (sm_103a)"; }

const char *dgmg_last_error(void) { return g_last_error.c_str(); }

void dgmg_default_opts(dgmg_opts *o) {
    if (!o) return;
    o->omega_dg = 0.8;
    o->omega_cg = 0.8;
    o->nu_pre = 2;
    o->nu_post = 2;
    o->precision = DGMG_FP64;
    o->block_inverse = DGMG_BLOCK_EXACT;
    o->coarsening = 2;
    o->rtol = 1e-10;
    o->maxit = 200;
    o->outer = DGMG_OUTER_AUTO;
    o->delta = 0.01;
    o->autotune = 0;
    o->p_coarsening = 0;
    o->basis = DGMG_BASIS_GLL;
    o->recompute_block = 0;
}

int dgmg_create(const dgmg_mesh *mesh, int p, const double *kappa, const dgmg_opts *opts, dgmg_ctx **out) {
    return dgmg::create_ctx(mesh, p, kappa, opts, 0, out);
}

}  // extern "C"

namespace dgmg {

// Contexts allocate from the device's default stream-ordered memory pool
// (cudaMallocAsync on their set-up stream). By default the pool returns freed
// memory to the CUDA driver at every synchronisation, so a process that destroys
// and creates hierarchies (a server, a batch after a batch) pays for mapping
// the memory again on every allocation: the pool of the current device keeps
// what is freed instead (a property of this process's pool, not of the GPU).
static void keep_pool_memory() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.push_back(dev);
}

int create_ctx(const dgmg_mesh *mesh, int p, const double *kappa, const dgmg_opts *opts, int flags, dgmg_ctx **out) {
    if (!out) return fail(DGMG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mesh) return fail(DGMG_EINVAL, "mesh is NULL");
    if (mesh->dim != 2 && mesh->dim != 3) return fail(DGMG_EINVAL, "mesh->dim must be 2 or 3");
    if (p < 1 || p > PMAX) return fail(DGMG_EINVAL, "p must be in 1..6");
    for (int a = 0; a < mesh->dim; ++a)
        if (mesh->n[a] < 2 || mesh->n[a] > (1 << 20))
            return fail(DGMG_EINVAL, "every mesh->n[a] must be in 2..2^20");
    dgmg_opts o;
    dgmg_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.omega_dg > 0 && o.omega_dg < 2) || !(o.omega_cg > 0 && o.omega_cg < 2))
        return fail(DGMG_EINVAL, "omega_dg and omega_cg must be in (0, 2)");
    if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre > 64 || o.nu_post > 64)
        return fail(DGMG_EINVAL, "nu_pre, nu_post must be in 0..64");
    if (o.precision != DGMG_FP64 && o.precision != DGMG_MIXED_FP32) return fail(DGMG_EINVAL, "unknown precision");
    if (o.block_inverse != DGMG_BLOCK_EXACT && o.block_inverse != DGMG_BLOCK_INTERIOR_ONLY)
        return fail(DGMG_EINVAL, "unknown block_inverse");
    if (o.coarsening != 2 && o.coarsening != 3) return fail(DGMG_EINVAL, "coarsening must be 2 or 3");
    if (!(o.rtol > 0 && o.rtol < 1)) return fail(DGMG_EINVAL, "rtol must be in (0, 1)");
    if (o.maxit < 1) return fail(DGMG_EINVAL, "maxit must be >= 1");
    if (o.outer < DGMG_OUTER_AUTO || o.outer > DGMG_OUTER_MGMULT_PREC)
        return fail(DGMG_EINVAL, "unknown outer iteration");
    if ((o.outer == DGMG_OUTER_MGMULT || o.outer == DGMG_OUTER_MGMULT_PREC) && o.precision != DGMG_FP64)
        return fail(DGMG_EINVAL, "DGMG_OUTER_MGMULT runs in DGMG_FP64");
    if (o.outer == DGMG_OUTER_RELIABLE && o.precision != DGMG_MIXED_FP32)
        return fail(DGMG_EINVAL, "DGMG_OUTER_RELIABLE needs DGMG_MIXED_FP32");
    if (!(o.delta > 0 && o.delta < 1)) return fail(DGMG_EINVAL, "delta must be in (0, 1)");
    if (o.p_coarsening != 0 && o.p_coarsening != 1) return fail(DGMG_EINVAL, "p_coarsening must be 0 or 1");
    if (o.basis != DGMG_BASIS_GLL && o.basis != DGMG_BASIS_GL)
        return fail(DGMG_EINVAL, "basis must be DGMG_BASIS_GLL or DGMG_BASIS_GL");
    if (o.recompute_block != 0 && o.recompute_block != 1) return fail(DGMG_EINVAL, "recompute_block must be 0 or 1");
    if (o.outer == DGMG_OUTER_AUTO) o.outer = o.precision == DGMG_MIXED_FP32 ? DGMG_OUTER_RELIABLE : DGMG_OUTER_PCG;

    keep_pool_memory();
    std::unique_ptr<dgmg_ctx> C(new dgmg_ctx());
    {
        cudaError_t e = cudaStreamCreateWithFlags(&C->setup_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        e = cudaStreamCreateWithFlags(&C->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    }
    C->dim = mesh->dim;
    C->p = p;
    C->q = p + 1;
    for (int a = 0; a < 3; ++a) C->n[a] = a < mesh->dim ? mesh->n[a] : 1;
    C->ncell = (int64_t)C->n[0] * C->n[1] * C->n[2];
    C->nloc = C->dim == 3 ? (int64_t)C->q * C->q * C->q : (int64_t)C->q * C->q;
    C->ndof = C->ncell * C->nloc;
    C->opts = o;
    const int nf = (int)(C->nloc / C->q);
    C->cpb = std::max(1, 256 / nf);   // per-pencil tile: as many cells as fit 256 threads
    for (int k = 0; k < 2; ++k)
        for (int st = 0; st < 3; ++st) C->tile[k][st] = C->cpb;
    C->tile[0][TILE_SMOOTH] = 0;   // the one-thread-per-cell smoother and residual where they apply
    C->tile[1][TILE_SMOOTH] = 0;
    C->tile[0][TILE_RESIDUAL] = 0;
    C->tile[1][TILE_RESIDUAL] = 0;

    std::vector<double> kap(C->ncell, 1.0);
    if (kappa) {
        for (int64_t i = 0; i < C->ncell; ++i) {
            if (!(kappa[i] > 0.0) || !std::isfinite(kappa[i]))
                return fail(DGMG_EINVAL, "kappa must be positive and finite (cell " + std::to_string(i) + ")");
            kap[i] = kappa[i];
        }
    }
    SetupTrace trace;
    C->re = make_refelem(p, o.basis);
    trace.mark("refelem");

    // Q1 hierarchy
    build_q1_levels(C->dim, C->n, o.coarsening, kap, C->lv);
    trace.mark("q1 levels");
    {
        std::vector<double> inv;
        RC(coarse_inverse(*C, inv));
        RC(C->upload(&C->coarse_inv, inv));
    }
    trace.mark("coarse inverse");

    const DGSpace S0 = finest_space(*C);
    RC(setup_dg<double>(*C, S0, C->d64, kap, !(flags & CREATE_NO_FP64_SMOOTHER)));
    trace.mark("dg fp64 (factors on the device)");
    if (!(flags & CREATE_NO_SOLVER)) {   // a batch member runs its Q1 levels in the batch's kernels
        C->q1_blocks = q1_blocks_for(C->dim, o.precision == DGMG_MIXED_FP32);
        C->q1_wide = !(flags & CREATE_SHARED_GPU);
        C->q1_blocks_t[0] = q1_cycle_max_blocks<double>(C->dim, false);
        C->q1_blocks_t[1] = o.precision == DGMG_MIXED_FP32 ? q1_cycle_max_blocks<float>(C->dim, C->q1_wide) : 0;
        // beside other solves (server): no more blocks than the FP64 kernel's one per
        // SM, so that the cooperative launch finds room among concurrent kernels
        if (!C->q1_wide && C->q1_blocks_t[1] > C->q1_blocks_t[0] && C->q1_blocks_t[0] > 0)
            C->q1_blocks_t[1] = C->q1_blocks_t[0];
    }
    if (!(flags & CREATE_NO_FP64_Q1)) {
        RC(setup_cg<double>(*C, C->cg64));
        RC(setup_q1_plan<double>(*C));
    }
    trace.mark("cg upload");
    if (o.precision == DGMG_MIXED_FP32) {
        RC(setup_dg<float>(*C, S0, C->d32, kap, true, nullptr, C->d64.fd));
        RC(setup_cg<float>(*C, C->cg32));
        RC(setup_q1_plan<float>(*C));
        RC(C->alloc(&C->r32, C->ndof));
        RC(C->alloc(&C->z32, C->ndof));
        if (o.outer == DGMG_OUTER_RELIABLE) {
            RC(C->alloc(&C->p32, C->ndof));
            RC(C->alloc(&C->q32, C->ndof));
            RC(C->alloc(&C->xs32, C->ndof));
            RC(C->alloc(&C->rold32, C->ndof));
        }
    }
    RC(setup_dg_levels(*C, kap));
    trace.mark("dg levels");
    if (flags & CREATE_NO_SOLVER) {   // a member of a batch: the batch owns the solver's vectors
        trace.mark("rest");
        DG_CUDA(cudaStreamSynchronize(C->setup_stream));
        *out = C.release();
        return DGMG_OK;
    }
    RC(C->alloc(&C->w_r, C->ndof));
    RC(C->alloc(&C->w_z, C->ndof));
    RC(C->alloc(&C->w_p, C->ndof));
    RC(C->alloc(&C->w_q, C->ndof));
    RC(C->alloc(&C->w_rold, C->ndof));
    RC(C->alloc(&C->scal, S_NSCAL));
    RC(C->alloc(&C->partials, 2 * DOT_BLOCKS));
    {
        cudaError_t e = cudaMallocHost((void **)&C->host_scal, sizeof(double) * S_HOST);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
        e = wait_timeouts_addr_fp32(&C->tmo_dev[0]);
        if (e == cudaSuccess) e = wait_timeouts_addr_fp64(&C->tmo_dev[1]);
        if (e == cudaSuccess) e = q1_barrier_timeouts_addr(&C->tmo_dev[2]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        e = cudaEventCreateWithFlags(&C->ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
    // quadrature tables for the load vector: (p+2) Gauss points per axis
    {
        const int mq = p + 2;
        std::vector<double> xg, wg;
        gauss_legendre(mq, xg, wg);
        std::vector<double> V((size_t)C->q * mq), W((size_t)3 * mq);
        std::vector<double> val(C->q);
        for (int g = 0; g < mq; ++g) {
            lagrange_at(C->re.nodes, xg[g], val.data(), nullptr);
            for (int i = 0; i < C->q; ++i) V[(size_t)i * mq + g] = val[i];
        }
        for (int a = 0; a < 3; ++a)
            for (int g = 0; g < mq; ++g) W[(size_t)a * mq + g] = wg[g] * 0.5 / C->n[a];
        RC(C->upload(&C->quad_x1, xg));
        RC(C->upload(&C->quad_V, V));
        RC(C->upload(&C->quad_w, W));
    }
    trace.mark("rest");
    DG_CUDA(cudaStreamSynchronize(C->setup_stream));   // uploads done before any use
    trace.mark("sync");
    if (o.autotune) {
        RC(autotune_tiles(*C));
        trace.mark("autotune");
    }
    *out = C.release();
    return DGMG_OK;
}

}  // namespace dgmg

extern "C" {

int dgmg_destroy(dgmg_ctx *ctx) {
    if (!ctx) return DGMG_OK;
    cudaDeviceSynchronize();
    delete ctx;
    return DGMG_OK;
}

int dgmg_info(const dgmg_ctx *C, dgmg_info_t *info) {
    RC(check_ctx(C));
    if (!info) return fail(DGMG_EINVAL, "info is NULL");
    std::memset(info, 0, sizeof(*info));
    info->dim = C->dim;
    info->p = C->p;
    info->q = C->q;
    for (int a = 0; a < 3; ++a) info->n[a] = C->n[a];
    info->ncell = C->ncell;
    info->ndof = C->ndof;
    info->nlevels_cg = (int)C->lv.size();
    info->nvert0 = C->lv[0].nv;
    info->ncoarse = C->ncoarse;
    info->omega_dg = C->opts.omega_dg;
    info->omega_cg = C->opts.omega_cg;
    info->nu_pre = C->opts.nu_pre;
    info->nu_post = C->opts.nu_post;
    info->precision = C->opts.precision;
    info->block_inverse = C->opts.block_inverse;
    info->coarsening = C->opts.coarsening;
    info->device_bytes = C->bytes;
    info->outer = C->opts.outer;
    info->dg_levels = (int)C->dgs.size();
    const bool mixed = C->opts.precision == DGMG_MIXED_FP32;
    for (int k = 0; k < 6; ++k) info->tiles[k] = (k < 3 || mixed) ? C->tile[k / 3][k % 3] : 0;
    return DGMG_OK;
}

int dgmg_update_kappa(dgmg_ctx *C, const double *kappa) {
    using namespace dgmg;
    RC(check_ctx(C));
    if (!kappa) return fail(DGMG_EINVAL, "kappa is NULL");
    std::vector<double> kap(kappa, kappa + C->ncell);
    for (int64_t i = 0; i < C->ncell; ++i)
        if (!(kap[i] > 0.0) || !std::isfinite(kap[i]))
            return fail(DGMG_EINVAL, "kappa must be positive and finite (cell " + std::to_string(i) + ")");
    // host: the Q1 operators of the new kappa (same shapes) and the coarsest inverse
    std::vector<CGLevelHost> lv;
    build_q1_levels(C->dim, C->n, C->opts.coarsening, kap, lv);
    if (lv.size() != C->lv.size()) return fail(DGMG_EINVAL, "Q1 hierarchy changed shape");
    C->lv = std::move(lv);
    std::vector<double> inv;
    RC(coarse_inverse(*C, inv));
    cudaStream_t s = C->setup_stream;
    // everything in flight on the context's own stream must see the old data
    DG_CUDA(cudaStreamSynchronize(s));
    const bool mixed = C->opts.precision == DGMG_MIXED_FP32;
    const std::vector<float> kap32 = convert<float>(kap);
    DG_CUDA(cudaMemcpyAsync(C->d64.kappa, kap.data(), sizeof(double) * C->ncell, cudaMemcpyHostToDevice, s));
    if (mixed)
        DG_CUDA(cudaMemcpyAsync(C->d32.kappa, kap32.data(), sizeof(float) * C->ncell, cudaMemcpyHostToDevice, s));
    DG_CUDA(cudaMemcpyAsync(C->coarse_inv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice, s));
    // facet coefficients (the lower DG levels share the finest level's)
    LC(launch_facet_coefficients<double>(C->dim, C->n, C->ncell, C->d64.kappa, C->d64.kfac, s));
    if (mixed) LC(launch_facet_coefficients<float>(C->dim, C->n, C->ncell, C->d64.kappa, C->d32.kfac, s));
    std::vector<std::vector<float>> st32(C->lv.size());
    for (size_t l = 0; l < C->lv.size(); ++l) {
        const std::vector<double> &st = C->lv[l].st;
        if (l < C->cg64.size())
            DG_CUDA(cudaMemcpyAsync(C->cg64[l].st, st.data(), sizeof(double) * st.size(), cudaMemcpyHostToDevice, s));
        if (mixed) {
            st32[l] = convert<float>(st);
            DG_CUDA(cudaMemcpyAsync(C->cg32[l].st, st32[l].data(), sizeof(float) * st.size(),
                                    cudaMemcpyHostToDevice, s));
        }
    }
    // device: the per-cell factors of every DG level that has them
    for (size_t l = 0; l < C->dgs.size(); ++l) {
        DGDev<double> &D64 = l == 0 ? C->d64 : C->lvl64[l].D;
        if (D64.fd) RC(compute_factors<double>(*C, C->dgs[l], D64));
        if (mixed) {
            DGDev<float> &D32 = l == 0 ? C->d32 : C->lvl32[l].D;
            if (D32.fd) RC(compute_factors<float>(*C, C->dgs[l], D32, D64.fd));
        }
    }
    DG_CUDA(cudaStreamSynchronize(s));
    return DGMG_OK;
}

int dgmg_gll_nodes(const dgmg_ctx *C, double *nodes) {
    RC(check_ctx(C));
    if (!nodes) return fail(DGMG_EINVAL, "nodes is NULL");
    for (int i = 0; i < C->q; ++i) nodes[i] = C->re.nodes[i];
    return DGMG_OK;
}

int64_t dgmg_cg_size(const dgmg_ctx *C, int level) {
    if (!C || level < 0 || level >= (int)C->lv.size()) return -1;
    return C->lv[level].nv;
}

#define NEED(ptr) \
    if (!(ptr)) return fail(DGMG_EINVAL, #ptr " is NULL")

int dgmg_apply(dgmg_ctx *C, const double *u, double *y, void *stream) {
    RC(check_ctx(C));
    NEED(u);
    NEED(y);
    if (u == y) return fail(DGMG_EINVAL, "u and y must not overlap");
    return apply64(*C, u, nullptr, y, (cudaStream_t)stream);
}

int dgmg_residual(dgmg_ctx *C, const double *u, const double *b, double *r, void *stream) {
    RC(check_ctx(C));
    NEED(u);
    NEED(b);
    NEED(r);
    if (u == r) return fail(DGMG_EINVAL, "u and r must not overlap");
    return apply64(*C, u, b, r, (cudaStream_t)stream);
}

int dgmg_smooth(dgmg_ctx *C, double *u, const double *b, int nsteps, void *stream) {
    RC(check_ctx(C));
    NEED(u);
    NEED(b);
    if (nsteps < 0) return fail(DGMG_EINVAL, "nsteps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    DGDev<double> &D = C->d64;
    C->prof.begin(ST_PROJECT, s);
    LC(launch_project<double>(C->dim, C->q, D.c, C->tile[0][TILE_PROJECT], u, nullptr, D.tr[0], s));
    C->prof.end(s);
    int cur = 0;
    for (int k = 0; k < nsteps; ++k) {
        C->prof.begin(ST_SMOOTH, s);
        if (C->opts.recompute_block) RC(recompute_factors<double>(*C, C->dgs[0], D, s));
        LC(launch_smooth<double>(C->dim, C->q, D.c, C->tile[0][TILE_SMOOTH], exact_block(*C), u, b, D.kappa, D.fd, D.linv,
                                 D.tr[cur], D.tr[cur ^ 1], s));
        C->prof.end(s);
        cur ^= 1;
    }
    return DGMG_OK;
}

int dgmg_vcycle(dgmg_ctx *C, const double *r, double *e, void *stream) {
    RC(check_ctx(C));
    NEED(r);
    NEED(e);
    if (r == e) return fail(DGMG_EINVAL, "r and e must not overlap");
    return vcycle64(*C, r, e, (cudaStream_t)stream);
}

int dgmg_project(dgmg_ctx *C, double *u, const double *e, double *traces, void *stream) {
    RC(check_ctx(C));
    NEED(u);
    NEED(traces);
    LC(launch_project<double>(C->dim, C->q, C->d64.c, C->tile[0][TILE_PROJECT], u, e, traces, (cudaStream_t)stream));
    return DGMG_OK;
}

int dgmg_residual_restrict(dgmg_ctx *C, const double *u, const double *b, const double *traces, double *r,
                           double *rc, void *stream) {
    RC(check_ctx(C));
    NEED(u);
    NEED(b);
    NEED(traces);
    cudaStream_t s = (cudaStream_t)stream;
    int mode = RES_HAS_B;
    if (r) mode |= RES_WRITE_R;
    if (rc) mode |= RES_CORNERS;
    LC(launch_residual<double>(C->dim, C->q, C->d64.c, C->tile[0][TILE_RESIDUAL], mode, u, b, C->d64.kappa, traces, r,
                               C->d64.corners, exact_fd(*C, C->d64), s));
    if (rc) LC(launch_corner_gather<double>(C->dim, C->n, C->d64.corners, rc, s));
    return DGMG_OK;
}

static int check_level(dgmg_ctx *C, int level, bool need_next) {
    RC(check_ctx(C));
    if (level < 0 || level >= (int)C->lv.size() - (need_next ? 1 : 0))
        return fail(DGMG_EINVAL, "level out of range");
    if (C->cg64.size() != C->lv.size()) return fail(DGMG_EINVAL, "ctx holds no FP64 Q1 levels");
    return DGMG_OK;
}

int dgmg_cg_smooth(dgmg_ctx *C, int level, double *u, const double *b, int nsteps, void *stream) {
    RC(check_level(C, level, false));
    NEED(u);
    NEED(b);
    cudaStream_t s = (cudaStream_t)stream;
    CGDev<double> &L = C->cg64[level];
    for (int k = 0; k < nsteps; ++k) {
        LC(launch_cg_jacobi<double>(C->dim, L.L, u, b, L.u[0], C->opts.omega_cg, false, s));
        LC(cudaMemcpyAsync(u, L.u[0], sizeof(double) * L.L.nv, cudaMemcpyDeviceToDevice, s));
    }
    return DGMG_OK;
}

int dgmg_cg_residual(dgmg_ctx *C, int level, const double *u, const double *b, double *r, void *stream) {
    RC(check_level(C, level, false));
    NEED(u);
    NEED(b);
    NEED(r);
    LC(launch_cg_residual<double>(C->dim, C->cg64[level].L, u, b, r, (cudaStream_t)stream));
    return DGMG_OK;
}

int dgmg_h_restrict(dgmg_ctx *C, int level, const double *rf, double *rc, void *stream) {
    RC(check_level(C, level, true));
    NEED(rf);
    NEED(rc);
    LC(launch_h_restrict<double>(C->dim, C->cg64[level].L, rf, rc, (cudaStream_t)stream));
    return DGMG_OK;
}

int dgmg_h_prolong(dgmg_ctx *C, int level, const double *ec, double *uf, void *stream) {
    RC(check_level(C, level, true));
    NEED(ec);
    NEED(uf);
    LC(launch_h_prolong<double>(C->dim, C->cg64[level].L, ec, uf, (cudaStream_t)stream));
    return DGMG_OK;
}

int dgmg_coarse_solve(dgmg_ctx *C, const double *r, double *e, void *stream) {
    RC(check_ctx(C));
    NEED(r);
    NEED(e);
    LC(launch_coarse_solve<double>(C->ncoarse, C->coarse_inv, r, e, (cudaStream_t)stream));
    return DGMG_OK;
}

int dgmg_quad_points(dgmg_ctx *C, double *xq, void *stream) {
    RC(check_ctx(C));
    NEED(xq);
    LC(launch_quad_points(C->dim, C->q, C->n, C->p + 2, C->quad_x1, xq, C->ncell, (cudaStream_t)stream));
    return DGMG_OK;
}

int dgmg_load_vector(dgmg_ctx *C, const double *fq, double *b, void *stream) {
    RC(check_ctx(C));
    NEED(fq);
    NEED(b);
    LC(launch_load_vector(C->dim, C->q, C->p + 2, C->ncell, C->quad_V, C->quad_w, fq, b, (cudaStream_t)stream));
    return DGMG_OK;
}

int dgmg_estimate_bytes(const dgmg_mesh *mesh, int p, const dgmg_opts *opts, size_t *bytes) {
    if (!mesh || !bytes) return fail(DGMG_EINVAL, "mesh and bytes must not be NULL");
    if (mesh->dim != 2 && mesh->dim != 3) return fail(DGMG_EINVAL, "mesh->dim must be 2 or 3");
    if (p < 1 || p > PMAX) return fail(DGMG_EINVAL, "p must be in 1..6");
    for (int a = 0; a < mesh->dim; ++a)
        if (mesh->n[a] < 2 || mesh->n[a] > (1 << 20)) return fail(DGMG_EINVAL, "every mesh->n[a] must be in 2..2^20");
    dgmg_opts o;
    dgmg_default_opts(&o);
    if (opts) o = *opts;
    if (o.coarsening != 2 && o.coarsening != 3) return fail(DGMG_EINVAL, "coarsening must be 2 or 3");
    const int dim = mesh->dim, q = p + 1, f = o.coarsening;
    const bool mixed = o.precision == DGMG_MIXED_FP32;
    const bool reliable = mixed && o.outer != DGMG_OUTER_PCG;
    int n[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) n[a] = mesh->n[a];
    const int64_t ncell = (int64_t)n[0] * n[1] * n[2];
    const int64_t nloc = dim == 3 ? (int64_t)q * q * q : (int64_t)q * q, ndof = ncell * nloc;
    const int64_t nf = nloc / q, ns = dim == 3 ? 27 : 9;
    const int64_t tr = ncell * 2 * dim * trace_face_stride<double>((int)nf);
    const int64_t tr32 = ncell * 2 * dim * trace_face_stride<float>((int)nf);
    auto sz = [](int64_t count, size_t elem) { return (size_t)std::max<int64_t>(count, 1) * elem; };
    size_t dg64 = sz(ncell, 8) + 2 * sz(ncell * dim * (q * q + q), 8) + sz(ndof, 8) + 2 * sz(tr, 8) +
                  sz(ncell << dim, 8) + sz(ncell * 2 * dim, 8);   // kappa, factors and residual factors,
                                                                  // table, traces, corners, facet coefficients
    size_t dg32 = sz(ncell, 4) + 2 * sz(ncell * dim * (q * q + q), 4) + 2 * sz(tr32, 4) + sz(ncell << dim, 4) +
                  sz(ncell * 2 * dim, 4);
    size_t cg64 = 0, cg32 = 0;
    int cur[3] = {n[0], n[1], n[2]};
    int64_t nv = 1;
    for (;;) {
        nv = (int64_t)(cur[0] - 1) * (dim >= 2 ? cur[1] - 1 : 1) * (dim == 3 ? cur[2] - 1 : 1);
        cg64 += sz(ns * nv, 8) + 4 * sz(nv, 8);
        cg32 += sz(ns * nv, 4) + 4 * sz(nv, 4);
        bool any = false;
        for (int a = 0; a < dim; ++a) any = any || can_coarsen(cur[a], f);
        if (!any) break;
        int64_t ints = 0, dbl = 0;
        int nxt[3] = {cur[0], cur[1], cur[2]};
        for (int a = 0; a < dim; ++a) {
            const int mf = cur[a] - 1;
            const int nc = can_coarsen(cur[a], f) ? (int)coarse_positions(cur[a], f).size() - 1 : cur[a];
            ints += 2 * mf + 2 * (nc - 1);
            dbl += 2 * mf + 5 * (nc - 1);
            nxt[a] = nc;
        }
        cg64 += sz(ints, 4) + sz(dbl, 8);
        cg32 += sz(ints, 4) + sz(dbl, 4);
        for (int a = 0; a < 3; ++a) cur[a] = nxt[a];
    }
    size_t total = sz(nv * nv, 8) + dg64 + cg64 + 5 * sz(ndof, 8) + sz(S_NSCAL, 8) + sz(2 * DOT_BLOCKS, 8) +
                   sz(p + 2, 8) + sz((int64_t)q * (p + 2), 8) + sz(3 * (p + 2), 8);
    if (mixed) total += dg32 + cg32 + 2 * sz(ndof, 4) + (reliable ? 4 * sz(ndof, 4) : 0);
    if (q1_blocks_for(dim, mixed) > 0)   // the plans of the cooperative Q1 cycle and their counters
        total += sizeof(Q1Plan<double>) + (mixed ? sizeof(Q1Plan<float>) : 0) + 2 * sizeof(unsigned long long);
    if (o.p_coarsening == 1 && p >= 2) {
        // lower DG levels p-1 .. 1 (kappa shared with the finest level): factors,
        // traces, corners, iterate, right-hand side and residual; FP64 also the
        // table of inverse eigenvalue sums; the finest residual scratch
        for (int pc = p - 1; pc >= 1; --pc) {
            const int ql = pc + 1;
            const int64_t nl = dim == 3 ? (int64_t)ql * ql * ql : (int64_t)ql * ql, nd = ncell * nl;
            const int64_t trl = ncell * 2 * dim * trace_face_stride<double>((int)(nl / ql));
            const int64_t trl32 = ncell * 2 * dim * trace_face_stride<float>((int)(nl / ql));
            const int64_t fdl = ncell * dim * (ql * ql + ql);
            total += 2 * sz(fdl, 8) + sz(nd, 8) + 2 * sz(trl, 8) + sz(ncell << dim, 8) + 3 * sz(nd, 8);
            if (mixed) total += 2 * sz(fdl, 4) + 2 * sz(trl32, 4) + sz(ncell << dim, 4) + 3 * sz(nd, 4);
        }
        total += sz(ndof, 8) + (mixed ? sz(ndof, 4) : 0);
    }
    *bytes = total;
    return DGMG_OK;
}


int dgmg_profile(dgmg_ctx *C, int enable) {
    RC(check_ctx(C));
    C->prof.reset();
    C->prof.on = enable != 0;
    return DGMG_OK;
}

int dgmg_profile_read(dgmg_ctx *C, double *ms, long long *launches, int nstage) {
    RC(check_ctx(C));
    if (nstage < 0 || (nstage > 0 && (!ms || !launches))) return fail(DGMG_EINVAL, "bad output arrays");
    C->prof.collect();
    for (int i = 0; i < nstage && i < ST_N; ++i) {
        ms[i] = C->prof.ms[i];
        launches[i] = C->prof.cnt[i];
    }
    for (int i = 0; i < ST_N; ++i) {
        C->prof.ms[i] = 0;
        C->prof.cnt[i] = 0;
    }
    return DGMG_OK;
}

long long dgmg_kernel_launches(void) { return g_kernel_launches.load(); }

int dgmg_wait_timeouts(unsigned long long *count) {
    if (!count) return fail(DGMG_EINVAL, "dgmg_wait_timeouts: count is NULL");
    unsigned long long a = 0, b = 0, c = 0, v = 0;
    cudaError_t e = wait_timeouts_fp32(&a);
    if (e == cudaSuccess) e = wait_timeouts_fp64(&b);
    if (e == cudaSuccess) e = q1_barrier_timeouts(&c);
    if (e == cudaSuccess) e = wait_timeouts_volume(&v);
    if (e != cudaSuccess) return cuda_fail(e, "dgmg_wait_timeouts");
    *count = a + b + c + v;
    return DGMG_OK;
}

}  // extern "C"


// ------------------------------------------------ scratch-parameterised stage
namespace dgmg {

// Per-cell corner partial sums needed by the residual + p-restriction of ctx.
int64_t corner_scratch_count(const dgmg_ctx *C) { return C->ncell * (int64_t)(1 << C->dim); }

// dgmg_residual_restrict with the corner partial sums written to `corner_scratch`
// (corner_scratch_count(C) doubles) instead of the ctx's own buffer.
int residual_restrict_with_scratch(dgmg_ctx *C, const double *u, const double *b, const double *traces,
                                   double *r, double *rc, double *corner_scratch, cudaStream_t s) {
    int mode = RES_HAS_B;
    if (r) mode |= RES_WRITE_R;
    if (rc) mode |= RES_CORNERS;
    LC(launch_residual<double>(C->dim, C->q, C->d64.c, C->tile[0][TILE_RESIDUAL], mode, u, b, C->d64.kappa, traces, r,
                               corner_scratch, exact_fd(*C, C->d64), s));
    if (rc) LC(launch_corner_gather<double>(C->dim, C->n, corner_scratch, rc, s));
    return DGMG_OK;
}

}  // namespace dgmg
