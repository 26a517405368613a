// Host setup of libfc: spectrum, exponential-sum quadrature nodes, preconditioner fit.
//
// Readings of the paper used here (Section 4.2 leaves the quadrature parameters open):
//  * substitution t = e^u in the Laplace transform (eqn:Laplace_transf) so the right tail
//    decays double-exponentially; rho is scaled to [1, B] by rho_min (eqn:Laplace_transf_rhom1);
//  * trapezoid step h = pi^2 / (ln(1/delta) + 3); the sum is cut on the right at the first
//    node whose largest relative contribution on [1, B] is below delta/20;
//  * nodes with t_k B < s0 = 1/2 (exponentials nearly linear on [1, B]) form a positive
//    discrete measure that is replaced by its m-point Gauss rule, m the smallest with
//    s0^(2m)/(2m)! <= delta/100;
//  * gamma rho^alpha = gamma rho * rho^(alpha-1) (Lemma 4.1): each node of the rho^(alpha-1)
//    sum gives d rank-one terms whose mode-m factor carries lambda; at alpha = 1 the term is
//    gamma * sum_m lambda (rank d);
//  * the preconditioner is the least-squares exponential sum of 1/g on fixed geometric nodes.
#pragma once
#include <vector>

namespace fc {

struct ExpSum { std::vector<double> t, c; };

// Separable symbol as node list: term k has factor f(lambda) = exp(-tau_k lambda) in every
// mode, times lambda in mode `mode[k]` (mode[k] = -1: no lambda factor), and weight w[k].
struct SymbolNodes {
    std::vector<double> tau, w;
    std::vector<int> mode;
    int r_minus = 0, r_plus = 0;
    double rho_min = 0, rho_max = 0, err = 0;
};

std::vector<double> spectrum(int n);
ExpSum exp_sum(double s, double B, double delta, double s0);
double g_exact(double rho, double alpha, double beta, double gamma);
// The 1D spectrum lam (ascending) is passed in: lambda_k of the Laplacian, or lambda_k^alpha
// for the directionally fractional operator (which then uses exponent 1).
bool build_control_nodes(const std::vector<double>& lam, int d, double alpha, double beta,
                         double gamma, double delta, SymbolNodes& out);
bool build_precond_nodes(const std::vector<double>& lam, int d, double alpha, double beta,
                         double gamma, int rank, SymbolNodes& out);

// Compressed mode factor of a CP symbol: with X = E diag|xa| (n x R, E column-major with unit
// columns) and its thin SVD X = U S V^T truncated to the r singular values above tol * S_max,
//   Et = U S = X V_r  (n x r),   Mt = V_r^T diag(1/|xa|)  (r x R),
// so that E ~ Et Mt (weighted error sqrt(sum_{i>r} s_i^2)) and Mt diag(xa^2) Mt^T = I.
// The SVD is a one-sided (Hestenes) Jacobi on the columns of X, in FP64.
struct Compressed {
    int r = 0;
    std::vector<double> Et;   // n x r
    std::vector<double> Mt;   // r x R
};
bool compress_factor(const double* E, int n, int R, const double* xa, double tol, Compressed& out);

}  // namespace fc
