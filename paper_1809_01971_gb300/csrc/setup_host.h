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

// Operator symbol g(rho) = a rho^-sn + b rho^sp + c with 0 < sn <= 1, 0 < sp <= 1:
//   control operator beta^2 A^-alpha + gamma A^alpha: a = beta^2, sn = sp = alpha, b = gamma;
//   the test operators of Section 6 (Tables 6.1-6.4): A^alpha (a = 0, b = 1, sp = alpha) and
//   I + A^(2 alpha) (a = 0, b = 1, sp = 2 alpha <= 1, c = 1); A^alpha + A^-alpha is the control
//   operator at beta = gamma = 1.
struct SymbolSpec {
    double a = 0, sn = 1, b = 0, sp = 1, c = 0;
    double eval(double rho) const;
};

std::vector<double> spectrum(int n);
ExpSum exp_sum(double s, double B, double delta, double s0);
// The 1D spectrum lam (ascending) is passed in: lambda_k of the Laplacian, or lambda_k^alpha
// for the directionally fractional operator (which then uses exponent 1).  Terms in the
// order: the rho^-sn sum (r_minus terms), the Lemma 4.1 terms of rho^sp, the constant c.
// [rmin, rmax] is the range of rho = sum_l lambda_{i_l, l} (sums of the per-mode extremes).
bool build_symbol_nodes(double rmin, double rmax, int d, const SymbolSpec& g, double delta,
                        SymbolNodes& out);
// Preconditioner: least-squares exponential sum of 1/g (rank terms) ...
bool build_precond_nodes(double rmin, double rmax, const SymbolSpec& g, int rank,
                         SymbolNodes& out);
// ... or the sinc-quadrature exponential sum of rho^-s itself (the symbol g_1 = rho^-alpha of
// Section 6, the exact inverse of A^alpha).
bool build_inverse_power_nodes(double rmin, double rmax, int d, double s, double delta,
                               SymbolNodes& out);
// Variable coefficients (Remark on generalised directionally fractional operators): the 1D
// stiffness matrix of -(a u')' from a((i+1/2) h), i = 0..n, and its eigen-decomposition.
void stiffness_1d(int n, const double* a_half, std::vector<double>& diag, std::vector<double>& off);
bool tridiag_eig(int n, std::vector<double> d, std::vector<double> e, std::vector<double>& lam,
                 std::vector<double>& V);

// Compressed mode factor of a CP symbol: with X = E diag|xa| (n x R, E column-major with unit
// columns), D the diagonal of its row norms and the thin SVD D^-1 X = U S V^T truncated to the
// r singular values above tol * S_max,
//   Et = X V_r  (n x r),   Mt = V_r^T diag(1/|xa|)  (r x R),
// so that E ~ Et Mt with every row of X kept to ~tol relative to its own norm, and
// Mt diag(xa^2) Mt^T = I.  The SVD is a one-sided (Hestenes) Jacobi, in FP64.
struct Compressed {
    int r = 0;
    std::vector<double> Et;   // n x r
    std::vector<double> Mt;   // r x R
};
bool compress_factor(const double* E, int n, int R, const double* xa, double tol, Compressed& out);

}  // namespace fc
