// Test shim: plain-C entry points over the library's host set-up routines (spectrum,
// quadrature nodes, preconditioner fit, 1D stiffness eigen-decomposition, factor
// compression), so that the CPU tests can check them against closed forms and LAPACK without
// a GPU.  Compiled by the tests together with csrc/setup_host.cpp; not part of libfc.
#include "setup_host.h"

#include <algorithm>

namespace {
fc::SymbolSpec spec_of(double a, double sn, double b, double sp, double c) {
    fc::SymbolSpec g;
    g.a = a; g.sn = sn; g.b = b; g.sp = sp; g.c = c;
    return g;
}
// Copies the node list out; returns the number of terms, or -1 if it does not fit `cap`.
int copy_nodes(const fc::SymbolNodes& s, int cap, double* tau, double* w, int* mode, int* counts,
               double* err) {
    const int r = (int)s.tau.size();
    if (r > cap) return -1;
    std::copy(s.tau.begin(), s.tau.end(), tau);
    std::copy(s.w.begin(), s.w.end(), w);
    std::copy(s.mode.begin(), s.mode.end(), mode);
    if (counts) { counts[0] = s.r_minus; counts[1] = s.r_plus; }
    if (err) *err = s.err;
    return r;
}
}  // namespace

extern "C" {

void shim_spectrum(int n, double* out) {
    const std::vector<double> lam = fc::spectrum(n);
    std::copy(lam.begin(), lam.end(), out);
}

int shim_symbol_nodes(double rmin, double rmax, int d, double a, double sn, double b, double sp,
                      double c, double delta, int cap, double* tau, double* w, int* mode,
                      int* counts, double* err) {
    fc::SymbolNodes s;
    if (!fc::build_symbol_nodes(rmin, rmax, d, spec_of(a, sn, b, sp, c), delta, s)) return -2;
    return copy_nodes(s, cap, tau, w, mode, counts, err);
}

int shim_precond_nodes(double rmin, double rmax, double a, double sn, double b, double sp,
                       double c, int rank, int cap, double* tau, double* w, int* mode) {
    fc::SymbolNodes s;
    if (!fc::build_precond_nodes(rmin, rmax, spec_of(a, sn, b, sp, c), rank, s)) return -2;
    return copy_nodes(s, cap, tau, w, mode, nullptr, nullptr);
}

int shim_inverse_power_nodes(double rmin, double rmax, int d, double s_, double delta, int cap,
                             double* tau, double* w, int* mode) {
    fc::SymbolNodes s;
    if (!fc::build_inverse_power_nodes(rmin, rmax, d, s_, delta, s)) return -2;
    return copy_nodes(s, cap, tau, w, mode, nullptr, nullptr);
}

void shim_stiffness_1d(int n, const double* a_half, double* diag, double* off) {
    std::vector<double> dg, of;
    fc::stiffness_1d(n, a_half, dg, of);
    std::copy(dg.begin(), dg.end(), diag);
    std::copy(of.begin(), of.end(), off);
}

int shim_tridiag_eig(int n, const double* d, const double* e, double* lam, double* V) {
    std::vector<double> dv(d, d + n), ev(e, e + (n > 1 ? n - 1 : 0)), l, v;
    if (!fc::tridiag_eig(n, dv, ev, l, v)) return -1;
    std::copy(l.begin(), l.end(), lam);
    std::copy(v.begin(), v.end(), V);
    return 0;
}

// Returns the compressed rank r (Et: n x r, Mt: r x R, column-major), or -1.
int shim_compress(const double* E, int n, int R, const double* xa, double tol, double* Et,
                  double* Mt) {
    fc::Compressed c;
    if (!fc::compress_factor(E, n, R, xa, tol, c)) return -1;
    std::copy(c.Et.begin(), c.Et.end(), Et);
    std::copy(c.Mt.begin(), c.Mt.end(), Mt);
    return c.r;
}

}  // extern "C"
