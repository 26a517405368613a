/*
 * eigerr.c -- oracle (test infrastructure only): error of a CP-format solution against the
 * exact full-format solution of g(A) u = b, evaluated over the whole n^d grid without
 * forming either n^d array.
 *
 * The exact solution is u* = (F x .. x F) diag(1/g(rho)) (F x .. x F) b (paper Section 3.2,
 * eqn:DiagFLaplace3D / eqn:DiagFLaplace2D), F the orthonormal DST-I, rho_i = sum_l
 * lambda_{i_l}.  F x .. x F is orthogonal, so with uh = (F x .. x F) u and bh = (F x .. x F) b
 * (CP tensors whose factor columns are the DSTs of the original columns, computed by the
 * caller)
 *
 *     ||u - u*||^2 = sum_i (uh_i - bh_i / g(rho_i))^2 ,   ||u*||^2 = sum_i (bh_i / g(rho_i))^2 .
 *
 * Both sums are taken point by point over every multi-index i (no cancellation between the
 * two CP tensors is left to a difference of large sums).  g(rho) = a rho^-sn + b rho^sp + c.
 *
 * Factor matrices are row-major n x R per mode (element (i, r) at i*R + r).  d in {2, 3}.
 * The sums run over the box i_l < m[l] (m[l] <= n; m[l] = n is the whole grid): the caller
 * accounts for the part outside the box (eigerr.py).  lam holds d blocks of n eigenvalues.
 * Threads: OpenMP over the outermost index.
 */
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double symbol(double rho, double a, double sn, double b, double sp, double c) {
    if (sn == sp) {                       /* a rho^-s + b rho^s + c with one exponential */
        double x = exp(sp * log(rho));
        return a / x + b * x + c;
    }
    double v = c;
    if (a != 0.0) v += a * exp(-sn * log(rho));
    if (b != 0.0) v += b * exp(sp * log(rho));
    return v;
}

int eig_error(int d, int n, const int* m, const double* lam, double a, double sn, double b,
              double sp, double c, int Ru, const double* xu, const double* const* Uu, int Rb,
              const double* xb, const double* const* Ub, int threads, double* out) {
    if (!(d == 2 || d == 3) || n < 1 || Ru < 0 || Rb < 0 || !out || !m) return -1;
    for (int l = 0; l < d; ++l)
        if (m[l] < 0 || m[l] > n) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    const int outer = (d == 3) ? m[2] : 1;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma omp parallel reduction(+ : s0, s1, s2)
    {
        double* cu = (double*)malloc(sizeof(double) * (Ru > 0 ? Ru : 1));
        double* cb = (double*)malloc(sizeof(double) * (Rb > 0 ? Rb : 1));
#pragma omp for schedule(dynamic, 1)
        for (int i3 = 0; i3 < outer; ++i3) {
            const double l3 = (d == 3) ? lam[2 * n + i3] : 0.0;
            for (int i2 = 0; i2 < m[1]; ++i2) {
                const double l23 = lam[n + i2] + l3;
                for (int r = 0; r < Ru; ++r) {
                    double v = xu[r] * Uu[1][(size_t)i2 * Ru + r];
                    if (d == 3) v *= Uu[2][(size_t)i3 * Ru + r];
                    cu[r] = v;
                }
                for (int r = 0; r < Rb; ++r) {
                    double v = xb[r] * Ub[1][(size_t)i2 * Rb + r];
                    if (d == 3) v *= Ub[2][(size_t)i3 * Rb + r];
                    cb[r] = v;
                }
                double e0 = 0.0, e1 = 0.0, e2 = 0.0;
                for (int i1 = 0; i1 < m[0]; ++i1) {
                    const double* ur = Uu[0] + (size_t)i1 * Ru;
                    const double* br = Ub[0] + (size_t)i1 * Rb;
                    double u = 0.0, bv = 0.0;
                    for (int r = 0; r < Ru; ++r) u += cu[r] * ur[r];
                    for (int r = 0; r < Rb; ++r) bv += cb[r] * br[r];
                    const double w = bv / symbol(lam[i1] + l23, a, sn, b, sp, c);
                    const double e = u - w;
                    e0 += e * e;
                    e1 += w * w;
                    e2 += u * u;
                }
                s0 += e0;
                s1 += e1;
                s2 += e2;
            }
        }
        free(cu);
        free(cb);
    }
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
    return 0;
}
