// Test helper: prints the library's host reference element (the code the
// set-up runs, compiled on its own) for degrees 1..6 in both bases, one
// labelled line of %.17g numbers per array, for comparison with the oracle.
#include <cstdio>
#include <vector>

#include "internal.h"

static void row(const char *name, int p, int basis, const std::vector<double> &v) {
    std::printf("%s %d %d", name, p, basis);
    for (double x : v) std::printf(" %.17g", x);
    std::printf("\n");
}

int main() {
    for (int basis = DGMG_BASIS_GLL; basis <= DGMG_BASIS_GL; ++basis)
        for (int p = 1; p <= dgmg::PMAX; ++p) {
            const dgmg::RefElem1D r = dgmg::make_refelem(p, basis);
            row("nodes", p, basis, r.nodes);
            row("M", p, basis, r.M);
            row("K", p, basis, r.K);
            row("e0", p, basis, r.e0);
            row("ep", p, basis, r.ep);
            row("d0", p, basis, r.d0);
            row("dp", p, basis, r.dp);
            std::vector<double> Linv(r.q * r.q);
            if (!dgmg::cholesky_inverse_lower(r.q, r.M.data(), Linv.data())) return 1;
            row("Linv", p, basis, Linv);
        }
    std::vector<double> x, w;
    for (int m = 1; m <= 9; ++m) {
        dgmg::gauss_legendre(m, x, w);
        row("glx", m, 0, x);
        row("glw", m, 0, w);
    }
    return 0;
}
