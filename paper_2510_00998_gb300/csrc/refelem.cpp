// Host-side 1D reference element and small dense linear algebra for the
// set-up of libdgmg (double precision).
//
// GLL nodes: the end points and the roots of P_p' (Sec. 2.2 basis), found by
// Newton's method from the Chebyshev-Gauss-Lobatto points. Gauss-Legendre
// rules: Newton's method on P_m from the usual cosine initial guesses, weights
// 2 / ((1 - x^2) P_m'(x)^2); the q GL points are also the nodes of the GL
// basis (Sec. 6.4). Legendre values through the three-term recurrence.
// Exact 1D mass and stiffness matrices use q-point Gauss-Legendre quadrature
// (degree 2p integrands), matching the paper's remark that the GLL mass matrix
// is not diagonal (exact integration, Sec. 4.1).
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace dgmg {

// P_m(x) and P_m'(x) by the three-term recurrence.
static void legendre(int m, double x, double &P, double &dP) {
    double p0 = 1.0, p1 = x;
    if (m == 0) {
        P = 1.0;
        dP = 0.0;
        return;
    }
    for (int k = 2; k <= m; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    P = p1;
    // derivative from (1-x^2) P_m' = m (P_{m-1} - x P_m), valid for |x| < 1
    dP = m * (p0 - x * p1) / (1.0 - x * x);
}

void gauss_legendre(int m, std::vector<double> &x, std::vector<double> &w) {
    x.assign(m, 0.0);
    w.assign(m, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < m; ++i) {
        double z = std::cos(pi * (i + 0.75) / (m + 0.5));
        double P, dP;
        for (int it = 0; it < 100; ++it) {
            legendre(m, z, P, dP);
            const double dz = P / dP;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        legendre(m, z, P, dP);
        x[m - 1 - i] = z;                       // ascending order
        w[m - 1 - i] = 2.0 / ((1.0 - z * z) * dP * dP);
    }
}

static std::vector<double> gll_points(int p) {
    std::vector<double> x(p + 1);
    x[0] = -1.0;
    x[p] = 1.0;
    const double pi = 3.14159265358979323846;
    for (int j = 1; j < p; ++j) {
        // root of P_p' near the Chebyshev-Gauss-Lobatto point -cos(pi j / p)
        double z = -std::cos(pi * j / p);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(p, z, P, dP);
            // P_p'' from the Legendre ODE: (1-z^2) P'' = 2 z P' - p(p+1) P
            const double d2P = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
            const double dz = dP / d2P;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[j] = z;
    }
    return x;
}

void lagrange_at(const std::vector<double> &nodes, double x, double *val, double *der) {
    const int n = (int)nodes.size();
    for (int i = 0; i < n; ++i) {
        double v = 1.0;
        for (int m = 0; m < n; ++m)
            if (m != i) v *= (x - nodes[m]) / (nodes[i] - nodes[m]);
        double d = 0.0;
        for (int k = 0; k < n; ++k) {
            if (k == i) continue;
            double term = 1.0 / (nodes[i] - nodes[k]);
            for (int m = 0; m < n; ++m)
                if (m != i && m != k) term *= (x - nodes[m]) / (nodes[i] - nodes[m]);
            d += term;
        }
        if (val) val[i] = v;
        if (der) der[i] = d;
    }
}

RefElem1D make_refelem(int p, int basis) {
    RefElem1D r;
    r.p = p;
    r.q = p + 1;
    r.basis = basis;
    const int q = r.q;
    std::vector<double> xg, wg;
    gauss_legendre(q, xg, wg);
    r.nodes = basis == DGMG_BASIS_GL ? xg : gll_points(p);
    r.M.assign(q * q, 0.0);
    r.K.assign(q * q, 0.0);
    std::vector<double> v(q), d(q);
    for (int g = 0; g < q; ++g) {
        lagrange_at(r.nodes, xg[g], v.data(), d.data());
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                r.M[i * q + j] += wg[g] * v[i] * v[j];
                r.K[i * q + j] += wg[g] * d[i] * d[j];
            }
    }
    r.e0.assign(q, 0.0);
    r.ep.assign(q, 0.0);
    r.d0.assign(q, 0.0);
    r.dp.assign(q, 0.0);
    // with GLL nodes the end values are exactly the unit vectors (the factor
    // (x - x_end) of every other basis function vanishes in floating point)
    lagrange_at(r.nodes, -1.0, r.e0.data(), r.d0.data());
    lagrange_at(r.nodes, 1.0, r.ep.data(), r.dp.data());
    return r;
}

bool cholesky_inverse_lower(int q, const double *M, double *Linv) {
    std::vector<double> L(q * q, 0.0);
    for (int j = 0; j < q; ++j) {
        double s = M[j * q + j];
        for (int k = 0; k < j; ++k) s -= L[j * q + k] * L[j * q + k];
        if (!(s > 0.0)) return false;
        L[j * q + j] = std::sqrt(s);
        for (int i = j + 1; i < q; ++i) {
            double t = M[i * q + j];
            for (int k = 0; k < j; ++k) t -= L[i * q + k] * L[j * q + k];
            L[i * q + j] = t / L[j * q + j];
        }
    }
    // invert the lower triangular factor column by column
    std::memset(Linv, 0, sizeof(double) * q * q);
    for (int c = 0; c < q; ++c) {
        for (int i = c; i < q; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s -= L[i * q + k] * Linv[k * q + c];
            Linv[i * q + c] = s / L[i * q + i];
        }
    }
    return true;
}

}  // namespace dgmg
