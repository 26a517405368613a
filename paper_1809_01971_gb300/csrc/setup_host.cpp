// Host-side setup of libfc (cold path, FP64): the 1D spectrum, the exponential-sum
// quadratures of rho^-s and the least-squares preconditioner fit.  The factor matrices
// themselves are built on the device from the node lists produced here.
//
// Paper: Section 3.2 (eqn:eig_lap), Section 4.2 (eqn:Sinc_quadr_trunc, eqn:Func_of_rho,
// eqn:Laplace_transf_rhom1), Lemma 4.1 (positive powers), Section 3.3 (preconditioner).
#include "setup_host.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace fc {

std::vector<double> spectrum(int n) {
    // lambda_k = (4/h^2) sin^2(pi k / (2(n+1))), h = 1/(n+1), k = 1..n  (eqn:eig_lap)
    const double N = n + 1.0;
    std::vector<double> lam(n);
    for (int k = 1; k <= n; ++k) {
        double s = std::sin(M_PI * k / (2.0 * N));
        lam[k - 1] = 4.0 * N * N * s * s;
    }
    return lam;
}

// 1D stiffness matrix of -(a u')' (Remark on variable coefficients, A_l = -grad^T a_l grad):
// with a_half[i] = a((i + 1/2) h), i = 0..n, row i of the symmetric tridiagonal matrix has
// diagonal (a_half[i] + a_half[i+1]) / h^2 and off-diagonal -a_half[i+1] / h^2 (Dirichlet).
void stiffness_1d(int n, const double* a_half, std::vector<double>& diag, std::vector<double>& off) {
    const double N2 = (n + 1.0) * (n + 1.0);
    diag.assign(n, 0.0);
    off.assign(n > 0 ? n - 1 : 0, 0.0);
    for (int i = 0; i < n; ++i) diag[i] = (a_half[i] + a_half[i + 1]) * N2;
    for (int i = 0; i + 1 < n; ++i) off[i] = -a_half[i + 1] * N2;
}

// Symmetric tridiagonal eigen-decomposition T = V diag(lam) V^T by implicit QR steps with the
// Wilkinson shift (the shift is the eigenvalue of the trailing 2 x 2 block closer to its last
// diagonal entry).  A step chases the bulge of one Givens rotation down the unreduced block;
// each rotation acts on the 4 x 4 window around it, held densely, and on two columns of V.
// Off-diagonals below 4e-16 (|d_i| + |d_i+1|) are set to zero (deflation).  Eigenvalues
// ascending, eigenvectors orthonormal columns of V (n x n, column-major).  O(n^3) with the
// vectors: meant for the 1D problems, n up to a few thousand.
bool tridiag_eig(int n, std::vector<double> d, std::vector<double> e, std::vector<double>& lam,
                 std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i + (size_t)i * n] = 1.0;
    lam = d;
    if (n <= 1) return n == 1;
    e.resize(n - 1);
    int guard = 0;
    for (int q = n - 1; q > 0;) {
        // deflate from the bottom
        while (q > 0 && std::fabs(e[q - 1]) <= 4e-16 * (std::fabs(d[q - 1]) + std::fabs(d[q]))) {
            e[q - 1] = 0.0;
            --q;
        }
        if (q == 0) break;
        int p = q - 1;
        while (p > 0 && std::fabs(e[p - 1]) > 4e-16 * (std::fabs(d[p - 1]) + std::fabs(d[p]))) --p;
        if (++guard > 60 * n) return false;
        // Wilkinson shift from the trailing 2 x 2 block of the unreduced block [p, q]
        const double t = 0.5 * (d[q - 1] - d[q]);
        const double b2 = e[q - 1] * e[q - 1];
        const double den = t + (t >= 0.0 ? 1.0 : -1.0) * std::sqrt(t * t + b2);
        const double mu = d[q] - (den != 0.0 ? b2 / den : 0.0);
        double x = d[p] - mu, z = e[p];
        double bulge = 0.0;                      // T[k+1][k-1] entry created by the previous rotation
        for (int k = p; k < q; ++k) {
            // rotation G in the plane (k, k+1) with G^T [x; z] = [r; 0]
            const double r = std::hypot(x, z);
            const double c = (r > 0.0) ? x / r : 1.0, s = (r > 0.0) ? z / r : 0.0;
            // window rows/cols k-1 .. k+2 (local 0..3), entries of the symmetric matrix
            double W[4][4] = {{0}};
            const int base = k - 1;
            for (int a = 0; a < 4; ++a) {
                const int ia = base + a;
                if (ia < p || ia > q) continue;
                W[a][a] = d[ia];
                if (a + 1 < 4 && ia + 1 <= q) W[a][a + 1] = W[a + 1][a] = e[ia];
            }
            if (k > p) W[0][2] = W[2][0] = bulge;   // T[k+1][k-1]
            // W <- G^T W G on local indices 1, 2
            for (int a = 0; a < 4; ++a) {            // rows
                const double u = W[1][a], v = W[2][a];
                W[1][a] = c * u + s * v;
                W[2][a] = -s * u + c * v;
            }
            for (int a = 0; a < 4; ++a) {            // columns
                const double u = W[a][1], v = W[a][2];
                W[a][1] = c * u + s * v;
                W[a][2] = -s * u + c * v;
            }
            // write back the tridiagonal part and the new bulge T[k+2][k]
            for (int a = 0; a < 4; ++a) {
                const int ia = base + a;
                if (ia < p || ia > q) continue;
                d[ia] = W[a][a];
                if (a + 1 < 4 && ia + 1 <= q) e[ia] = W[a][a + 1];
            }
            if (k > p) e[k - 1] = W[0][1];           // T[k][k-1] (the old bulge is annihilated)
            bulge = (k + 2 <= q) ? W[1][3] : 0.0;    // T[k+2][k] = W[3][1]
            // V <- V G
            double* vk = &V[(size_t)k * n];
            double* vk1 = &V[(size_t)(k + 1) * n];
            for (int i = 0; i < n; ++i) {
                const double u = vk[i], v = vk1[i];
                vk[i] = c * u + s * v;
                vk1[i] = -s * u + c * v;
            }
            if (k + 1 < q) { x = e[k]; z = bulge; }
        }
    }
    // ascending order
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] < d[b]; });
    std::vector<double> Vs((size_t)n * n);
    lam.resize(n);
    for (int j = 0; j < n; ++j) {
        lam[j] = d[idx[j]];
        std::copy(&V[(size_t)idx[j] * n], &V[(size_t)idx[j] * n] + n, &Vs[(size_t)j * n]);
    }
    V.swap(Vs);
    return true;
}

// Symmetric eigenvalues/vectors of a small dense matrix by cyclic Jacobi (row-major a, m x m).
static void small_sym_eig(std::vector<double>& a, int m, std::vector<double>& w,
                          std::vector<double>& v) {
    v.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) v[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) off += a[(size_t)p * m + q] * a[(size_t)p * m + q];
        if (off < 1e-300) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                double apq = a[(size_t)p * m + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = a[(size_t)p * m + p], aqq = a[(size_t)q * m + q];
                double th = (aqq - app) / (2.0 * apq);
                double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {  // columns p, q
                    double akp = a[(size_t)k * m + p], akq = a[(size_t)k * m + q];
                    a[(size_t)k * m + p] = c * akp - s * akq;
                    a[(size_t)k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {  // rows p, q
                    double apk = a[(size_t)p * m + k], aqk = a[(size_t)q * m + k];
                    a[(size_t)p * m + k] = c * apk - s * aqk;
                    a[(size_t)q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    double vkp = v[(size_t)k * m + p], vkq = v[(size_t)k * m + q];
                    v[(size_t)k * m + p] = c * vkp - s * vkq;
                    v[(size_t)k * m + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(m);
    for (int i = 0; i < m; ++i) w[i] = a[(size_t)i * m + i];
}

// m-point Gauss rule of the positive discrete measure sum_k c_k delta(t - t_k):
// Stieltjes three-term recurrence on the support points, then the eigen-decomposition of
// the Jacobi matrix (Golub-Welsch).
static void gauss_rule(const std::vector<double>& t, const std::vector<double>& c, int m,
                       std::vector<double>& nodes, std::vector<double>& weights) {
    const size_t K = t.size();
    double scale = 0.0, mu0 = 0.0;
    for (size_t k = 0; k < K; ++k) { scale = std::max(scale, t[k]); mu0 += c[k]; }
    std::vector<double> x(K), p(K, 1.0), pprev(K, 0.0), pnext(K);
    for (size_t k = 0; k < K; ++k) x[k] = t[k] / scale;
    std::vector<double> al(m, 0.0), be(m, 0.0);
    double normPrev = 1.0;
    for (int j = 0; j < m; ++j) {
        double nrm = 0.0, xn = 0.0;
        for (size_t k = 0; k < K; ++k) { nrm += c[k] * p[k] * p[k]; xn += c[k] * x[k] * p[k] * p[k]; }
        al[j] = xn / nrm;
        if (j > 0) be[j] = nrm / normPrev;
        for (size_t k = 0; k < K; ++k)
            pnext[k] = (x[k] - al[j]) * p[k] - (j > 0 ? be[j] * pprev[k] : 0.0);
        pprev.swap(p);
        p.swap(pnext);
        normPrev = nrm;
    }
    std::vector<double> J((size_t)m * m, 0.0), w, v;
    for (int i = 0; i < m; ++i) {
        J[(size_t)i * m + i] = al[i];
        if (i + 1 < m) {
            double e = std::sqrt(be[i + 1]);
            J[(size_t)i * m + i + 1] = e;
            J[(size_t)(i + 1) * m + i] = e;
        }
    }
    small_sym_eig(J, m, w, v);
    nodes.resize(m);
    weights.resize(m);
    for (int i = 0; i < m; ++i) {
        nodes[i] = w[i] * scale;
        weights[i] = mu0 * v[i] * v[i];   // first component of eigenvector i (row 0)
    }
}

ExpSum exp_sum(double s, double B, double delta, double s0) {
    // rho^-s = Gamma(s)^-1 int_R exp(s u - rho e^u) du  (Laplace transform with t = e^u),
    // trapezoid rule with step h (eqn:Sinc_quadr_trunc); see the readings in the header.
    ExpSum out;
    if (!(s > 0.0) || !(B >= 1.0) || !(delta > 0.0)) return out;
    const double h = M_PI * M_PI / (std::log(1.0 / delta) + 3.0);
    int m = 1;
    {
        // smallest m with s0^(2m)/(2m)! <= delta/100
        auto term = [&](int mm) { return std::exp(2 * mm * std::log(s0) - std::lgamma(2.0 * mm + 1.0)); };
        while (term(m) > delta / 100.0 && m < 40) ++m;
    }
    const double gs = std::tgamma(s);
    const long k0 = (long)std::floor(std::log(s0 / B) / h);
    const long L = (long)std::ceil(46.0 / (s * h));
    std::vector<double> tt, ct;
    for (long k = k0 - L; k < k0; ++k) {
        double u = k * h;
        tt.push_back(std::exp(u));
        ct.push_back(h * std::exp(s * u) / gs);
    }
    std::vector<double> tg, cg;
    gauss_rule(tt, ct, m, tg, cg);
    out.t = tg;
    out.c = cg;
    for (long k = k0;; ++k) {
        double u = k * h;
        double t = std::exp(u);
        double c = h * std::exp(s * u) / gs;
        double r = std::min(std::max(1.0, s / t), B);
        double contrib = c * std::exp(-t * r) * std::pow(r, s);
        if (u > 0.0 && contrib < delta / 20.0) break;
        out.t.push_back(t);
        out.c.push_back(c);
        if (out.t.size() > 4000) break;
    }
    return out;
}

double SymbolSpec::eval(double rho) const {
    double g = c;
    if (a != 0.0) g += a * std::pow(rho, -sn);
    if (b != 0.0) g += b * std::pow(rho, sp);
    return g;
}

bool build_symbol_nodes(double rmin, double rmax, int d, const SymbolSpec& g, double delta,
                        SymbolNodes& out) {
    const double B = rmax / rmin;
    out = SymbolNodes();
    out.rho_min = rmin;
    out.rho_max = rmax;
    ExpSum em, ep;
    if (g.a != 0.0) {
        em = exp_sum(g.sn, B, delta, 0.5);
        if (em.t.empty()) return false;
        for (size_t k = 0; k < em.t.size(); ++k) {
            out.tau.push_back(em.t[k] / rmin);
            out.w.push_back(g.a * em.c[k] * std::pow(rmin, -g.sn));
            out.mode.push_back(-1);
        }
    }
    out.r_minus = (int)out.tau.size();
    if (g.b != 0.0) {
        if (g.sp < 1.0) {
            // b rho^sp = b rho * rho^(sp-1) (Lemma 4.1): d terms per node of the rho^(sp-1) sum
            ep = exp_sum(1.0 - g.sp, B, delta, 0.5);
            if (ep.t.empty()) return false;
            for (size_t k = 0; k < ep.t.size(); ++k)
                for (int m = 0; m < d; ++m) {
                    out.tau.push_back(ep.t[k] / rmin);
                    out.w.push_back(g.b * ep.c[k] * std::pow(rmin, g.sp - 1.0));
                    out.mode.push_back(m);
                }
            out.r_plus = (int)ep.t.size();
        } else {
            for (int m = 0; m < d; ++m) {            // b rho = b sum_m lambda_m (rank d)
                out.tau.push_back(0.0);
                out.w.push_back(g.b);
                out.mode.push_back(m);
            }
        }
    }
    if (g.c != 0.0) {                                // constant: exp(0 lambda) in every mode
        out.tau.push_back(0.0);
        out.w.push_back(g.c);
        out.mode.push_back(-1);
    }
    if (out.tau.empty()) return false;
    // accuracy on a geometric rho grid: separable sums evaluated at rho = sum of lambdas
    double err = 0.0;
    const int G = 2000;
    for (int i = 0; i < G; ++i) {
        const double rho = rmin * std::pow(B, i / (G - 1.0));
        double v = g.c;
        if (g.a != 0.0) {
            double sm = 0.0;
            for (size_t k = 0; k < em.t.size(); ++k) sm += em.c[k] * std::exp(-em.t[k] * rho / rmin);
            v += g.a * std::pow(rmin, -g.sn) * sm;
        }
        if (g.b != 0.0) {
            if (g.sp < 1.0) {
                double sp = 0.0;
                for (size_t k = 0; k < ep.t.size(); ++k) sp += ep.c[k] * std::exp(-ep.t[k] * rho / rmin);
                v += g.b * rho * std::pow(rmin, g.sp - 1.0) * sp;
            } else {
                v += g.b * rho;
            }
        }
        err = std::max(err, std::fabs(v / g.eval(rho) - 1.0));
    }
    out.err = err;
    return true;
}

bool build_inverse_power_nodes(double rmin, double rmax, int d, double s, double delta,
                               SymbolNodes& out) {
    SymbolSpec g;
    g.a = 1.0;
    g.sn = s;
    return build_symbol_nodes(rmin, rmax, d, g, delta, out);
}

// Least squares min ||A x - b|| (A is m x k column-major, m >= k) by Householder QR.
static bool lstsq(std::vector<double> A, int m, int k, std::vector<double> b, std::vector<double>& x) {
    std::vector<double> tau(k);
    for (int j = 0; j < k; ++j) {
        double nrm = 0.0;
        for (int i = j; i < m; ++i) nrm += A[i + (size_t)j * m] * A[i + (size_t)j * m];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) return false;
        double a0 = A[j + (size_t)j * m];
        double beta = (a0 >= 0) ? -nrm : nrm;
        double v0 = a0 - beta;
        for (int i = j + 1; i < m; ++i) A[i + (size_t)j * m] /= v0;
        tau[j] = (beta - a0) / beta;
        A[j + (size_t)j * m] = beta;
        // apply H = I - tau v v^T (v0 = 1) to the remaining columns and to b
        for (int c = j + 1; c <= k; ++c) {
            double* col = (c < k) ? &A[(size_t)c * m] : b.data();
            double s = col[j];
            for (int i = j + 1; i < m; ++i) s += A[i + (size_t)j * m] * col[i];
            s *= tau[j];
            col[j] -= s;
            for (int i = j + 1; i < m; ++i) col[i] -= s * A[i + (size_t)j * m];
        }
    }
    x.assign(k, 0.0);
    for (int j = k - 1; j >= 0; --j) {
        double s = b[j];
        for (int c = j + 1; c < k; ++c) s -= A[j + (size_t)c * m] * x[c];
        x[j] = s / A[j + (size_t)j * m];
    }
    return true;
}

bool build_precond_nodes(double rmin, double rmax, const SymbolSpec& gs, int rank,
                         SymbolNodes& out) {
    // Fit p(rho) = sum_k w_k exp(-tau_k rho) to 1/g(rho) by least squares of p*g - 1 on a
    // geometric grid of [rho_min, rho_max], nodes tau_k geometric in
    // [0.2/rho_max, 20/rho_min]; columns scaled to unit norm before the solve.
    out = SymbolNodes();
    out.rho_min = rmin;
    out.rho_max = rmax;
    if (rank < 1) return false;
    if (!(rmax > rmin * (1.0 + 1e-9))) {
        // a single eigenvalue (n = 1): the exact inverse symbol is the constant 1/g(rho_min)
        out.tau.push_back(0.0);
        out.w.push_back(1.0 / gs.eval(rmin));
        out.mode.push_back(-1);
        out.r_minus = 1;
        out.err = 0.0;
        return true;
    }
    const int G = 3000;
    std::vector<double> tau(rank), rho(G), g(G);
    const double lt0 = std::log(0.2 / rmax), lt1 = std::log(20.0 / rmin);
    for (int k = 0; k < rank; ++k) tau[k] = std::exp(rank == 1 ? lt0 : lt0 + (lt1 - lt0) * k / (rank - 1.0));
    const double lr0 = std::log(rmin), lr1 = std::log(rmax);
    for (int i = 0; i < G; ++i) {
        rho[i] = std::exp(lr0 + (lr1 - lr0) * i / (G - 1.0));
        g[i] = gs.eval(rho[i]);
    }
    std::vector<double> A((size_t)G * rank), cn(rank), b(G, 1.0), w;
    for (int k = 0; k < rank; ++k) {
        double s = 0.0;
        for (int i = 0; i < G; ++i) {
            double v = g[i] * std::exp(-rho[i] * tau[k]);
            A[i + (size_t)k * G] = v;
            s += v * v;
        }
        cn[k] = std::sqrt(s);
        for (int i = 0; i < G; ++i) A[i + (size_t)k * G] /= cn[k];
    }
    if (!lstsq(A, G, rank, b, w)) return false;
    double err = 0.0;
    for (int k = 0; k < rank; ++k) w[k] /= cn[k];
    for (int i = 0; i < G; ++i) {
        double p = 0.0;
        for (int k = 0; k < rank; ++k) p += w[k] * std::exp(-rho[i] * tau[k]);
        if (!(p > 0.0)) return false;
        err = std::max(err, std::fabs(p * g[i] - 1.0));
    }
    for (int k = 0; k < rank; ++k) {
        out.tau.push_back(tau[k]);
        out.w.push_back(w[k]);
        out.mode.push_back(-1);
    }
    out.r_minus = rank;
    out.err = err;
    return true;
}

// Householder QR of the column-major m x c matrix A (m >= c), in place: returns the upper
// triangle R (c x c, column-major) of A = Q R.
static std::vector<double> householder_r(std::vector<double> A, int m, int c) {
    for (int j = 0; j < c; ++j) {
        double nrm = 0.0;
        for (int i = j; i < m; ++i) nrm += A[i + (size_t)j * m] * A[i + (size_t)j * m];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) continue;
        const double a0 = A[j + (size_t)j * m];
        const double beta = (a0 >= 0) ? -nrm : nrm;
        const double v0 = a0 - beta;
        const double tau = (beta - a0) / beta;
        for (int i = j + 1; i < m; ++i) A[i + (size_t)j * m] /= v0;
        A[j + (size_t)j * m] = beta;
        for (int q = j + 1; q < c; ++q) {
            double* col = &A[(size_t)q * m];
            double s = col[j];
            for (int i = j + 1; i < m; ++i) s += A[i + (size_t)j * m] * col[i];
            s *= tau;
            col[j] -= s;
            for (int i = j + 1; i < m; ++i) col[i] -= s * A[i + (size_t)j * m];
        }
    }
    std::vector<double> R((size_t)c * c, 0.0);
    for (int q = 0; q < c; ++q)
        for (int i = 0; i <= q; ++i) R[i + (size_t)q * c] = A[i + (size_t)q * m];
    return R;
}

bool compress_factor(const double* E, int n, int R, const double* xa, double tol, Compressed& out) {
    out = Compressed();
    if (n <= 0 || R <= 0) return false;
    std::vector<double> X0((size_t)n * R);
    for (int k = 0; k < R; ++k) {
        const double s = std::fabs(xa[k]);
        for (int i = 0; i < n; ++i) X0[i + (size_t)k * n] = E[i + (size_t)k * n] * s;
    }
    // The right singular vectors come from the row-normalised D^-1 X (D = diag of the row
    // norms): truncating its SVD relative to its largest singular value keeps every row of X
    // (every eigenvalue index of the symbol) accurate relative to that row's own size, not to
    // the largest row; the symbol's rows span many orders of magnitude at large n (the
    // Lemma 4.1 terms carry lambda up to 4 (n+1)^2).  The one-sided Jacobi runs on the
    // R x R triangle of a QR factorisation for tall X (same right singular vectors).
    std::vector<double> Xs(X0);
    for (int i = 0; i < n; ++i) {
        double s2 = 0.0;
        for (int k = 0; k < R; ++k) s2 += X0[i + (size_t)k * n] * X0[i + (size_t)k * n];
        const double inv = (s2 > 0.0) ? 1.0 / std::sqrt(s2) : 1.0;
        for (int k = 0; k < R; ++k) Xs[i + (size_t)k * n] *= inv;
    }
    const bool tall = n > R;
    const int m = tall ? R : n;
    std::vector<double> X = tall ? householder_r(Xs, n, R) : Xs;
    std::vector<double> V((size_t)R * R, 0.0), nrm(R);
    for (int k = 0; k < R; ++k) V[k + (size_t)k * R] = 1.0;
    const int n_full = n;
    n = m;
    auto dot = [&](int p, int q) {
        double s = 0.0;
        const double* a = &X[(size_t)p * n];
        const double* b = &X[(size_t)q * n];
        for (int i = 0; i < n; ++i) s += a[i] * b[i];
        return s;
    };
    for (int k = 0; k < R; ++k) nrm[k] = dot(k, k);
    for (int sweep = 0; sweep < 60; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < R; ++p)
            for (int q = p + 1; q < R; ++q) {
                const double a = nrm[p], b = nrm[q];
                if (a == 0.0 || b == 0.0) continue;
                const double g = dot(p, q);
                if (std::fabs(g) <= 1e-15 * std::sqrt(a * b)) continue;
                rotated = true;
                const double zeta = (b - a) / (2.0 * g);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                double* xp = &X[(size_t)p * n];
                double* xq = &X[(size_t)q * n];
                for (int i = 0; i < n; ++i) {
                    const double u = xp[i], w = xq[i];
                    xp[i] = c * u - s * w;
                    xq[i] = s * u + c * w;
                }
                double* vp = &V[(size_t)p * R];
                double* vq = &V[(size_t)q * R];
                for (int i = 0; i < R; ++i) {
                    const double u = vp[i], w = vq[i];
                    vp[i] = c * u - s * w;
                    vq[i] = s * u + c * w;
                }
                nrm[p] = dot(p, p);
                nrm[q] = dot(q, q);
            }
        if (!rotated) break;
    }
    std::vector<int> idx(R);
    for (int k = 0; k < R; ++k) idx[k] = k;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return nrm[a] > nrm[b]; });
    const double smax = std::sqrt(nrm[idx[0]]);
    if (!(smax > 0.0)) return false;
    int r = 0;
    while (r < R && std::sqrt(nrm[idx[r]]) > tol * smax) ++r;
    out.r = r;
    out.Et.assign((size_t)n_full * r, 0.0);
    out.Mt.assign((size_t)r * R, 0.0);
    for (int a = 0; a < r; ++a) {
        const int k = idx[a];
        // Et[:, a] = X0 V[:, k] (= U S column; computed from the full matrix)
        for (int i = 0; i < n_full; ++i) {
            double s = 0.0;
            for (int j = 0; j < R; ++j) s += X0[i + (size_t)j * n_full] * V[j + (size_t)k * R];
            out.Et[i + (size_t)a * n_full] = s;
        }
        for (int j = 0; j < R; ++j)
            out.Mt[a + (size_t)j * r] = (xa[j] != 0.0) ? V[j + (size_t)k * R] / std::fabs(xa[j]) : 0.0;
    }
    return true;
}

}  // namespace fc
