// Launch wrappers of libfc's kernels (host-callable, stream-ordered, no synchronisation).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace fc {

// ---- k_linalg.cu ---------------------------------------------------------------------
size_t pchol_smem();
// ---- k_symeig.cu ------------------------------------------------------------------------
// Batched symmetric eigen-decomposition: item b is the symmetric c x c matrix at A + b*bsA with
// c = dims ? min(dims[b*dstride], cmax) : cmax; eigenvalues descending into ev + b*bsE,
// orthonormal eigenvectors as columns of V + b*bsV (cmax x cmax, zero-padded).
void launch_symeig(cudaStream_t st, int batch, const double* A, int lda, long long bsA,
                   const int* dims, int dstride, int cmax, double* ev, long long bsE,
                   double* V, int ldv, long long bsV);
size_t symeig_smem();
// Graded variant (FP32 Jacobi + FP64 orthonormalisation), same contract; eigenvalues are FP64
// Rayleigh quotients if rq, else the FP32 Jacobi values.  floorRel: off-diagonal entries below
// floorRel * max diagonal are treated as zero (the rounding level of the Gram's formation);
// with floorAbs (device pointer) also those below floorFrac * (*floorAbs) in absolute terms.
void launch_gjacobi(cudaStream_t st, int batch, const double* A, int lda, long long bsA,
                    const int* dims, int dstride, int cmax, double* ev, long long bsE,
                    double* V, int ldv, long long bsV, bool rq, float floorRel = 1e-20f,
                    const double* floorAbs = nullptr, double floorFrac = 0.0);
size_t gjacobi_smem();
cudaError_t set_symeig_attributes();
// Opt the large-shared-memory kernels in to their dynamic shared memory (per device).
cudaError_t set_linalg_attributes();
void launch_pchol(cudaStream_t st, int batch, const double* M, int ldm, long long bsM,
                  const int* dims, int dstride, int cmax, double relTol, double* T, int ldt,
                  long long bsT, int* rank, int rstride);
// Tucker rank per mode: smallest r with sum_{i >= r} rho[i] + missed <= epsfac2 * wn2
// (rho: energies along the ordered basis directions, live entries dims live[l]).
void launch_select_tucker(cudaStream_t st, int d, const double* rho, int ldrho,
                          const double* missed, const double* wn2, double epsfac2, int cap,
                          int* r_out, double* tail2_out, const int* live);
void launch_select_terms(cudaStream_t st, const double* mu, int ldmu, const int* nslice,
                         const int* nper, int smax, int pmax, const double* core_e, double frac2,
                         int maxq, int* q_out, double* sigma, int* tslice, int* tidx,
                         double* dropped);

// ---- k_fft.cu ------------------------------------------------------------------------
// One pass of the full-format solve over an n^d column-major array (N = n + 1 a power of two,
// N <= 4096): the orthonormal DST-I of every line of `axis` (in may equal out); with scale,
// the line is transformed, divided by g(rho) = ga rho^-sn + gb rho^sp + gc and transformed
// back (axis = d - 1).  tw[k] = e^{-i pi k / N}, k < N.
void launch_dst_pass(cudaStream_t st, const double* in, double* out, int d, int axis, int n,
                     const double2* tw, bool scale, const double* lam, int lstride, double ga,
                     double sn, double gb, double sp, double gc);
cudaError_t set_fft_attributes(int N);
size_t fft_smem_bytes(int N, bool scale);

// ---- k_tensor.cu ---------------------------------------------------------------------
struct Piece { const double* xi; const double* U[3]; int ld; int K; double scale; };

void launch_build_symbol(cudaStream_t st, int n, int d, const double* lam, int lstride,
                         const double* tau, const double* w, const int* mode, int R, double* E,
                         int lde, long long bsE, double* xi);
// out columns = normalised columns of the pieces (in order); weights scale*xi*prod norms.
void launch_concat_normalize(cudaStream_t st, int d, int n, Piece p0, Piece p1, double* U,
                             int ldo, long long bsU, double* w);
// Y[:, t] = |w_t| U[:, t] for t < K (batch over modes)
// p[i + k*ld] *= w[k], i < rows, k < K (in place)
void launch_scale_cols(cudaStream_t st, int rows, int K, double* p, int ld, const double* w);
void launch_scale_cols_abs(cudaStream_t st, int d, int n, int K, const double* U, int ldu,
                           long long bsU, const double* w, double* Y, int ldy, long long bsY);
// Y[:, (k,j)] = |xa_k xb_j| E[:,k] . Yh[:,j]  (explicit Khatri-Rao columns, K = Ra*S)
void launch_kr_cols(cudaStream_t st, int d, int n, int Ra, int S, const double* E, int lde,
                    long long bsE, const double* xa, const double* Yh, int ldy, long long bsY,
                    const double* xb, int absw, double* Y, int ldo, long long bsO);
// Y = (U diag|w|) Omega, Omega[k,t] ~ N(0,1) from a counter-based hash (seed, mode, k, t)
void launch_sketch_dense(cudaStream_t st, int prec, int d, int n, int K, int c, const double* U,
                         int ldu, long long bsU, const double* w, unsigned long long seed,
                         double* Y, int ldy, long long bsY);
// Y = (E diag|xa| Oa) . (Yh diag|xb| Ob) with Gaussian Oa (Ra x c), Ob (S x c); both sketch
// launches take the contraction form (GemmPrec) of their GEMMs
void launch_sketch_kr(cudaStream_t st, int prec, int d, int n, int Ra, int S, int c,
                      const double* E, int lde, long long bsE, const double* xa, const double* Yh,
                      int ldy, long long bsY, const double* xb, unsigned long long seed,
                      double* Y, int ldo, long long bsO, double* tmp);
// Yr = Y - Q P (deflation), then columns of Yr scaled to unit norm (zero if tiny)
void launch_deflate_normalize(cudaStream_t st, int d, int n, int c, double* Yr, int ld,
                              long long bs, const double* Yorig, double relTiny);
// Q[:, off + j] = Qr[:, j] for j < min(cr, c - off), off = c1 (device counts per mode)
void launch_combine_cols(cudaStream_t st, int d, int n, int c, double* Q, int ld, long long bs,
                         const double* Qr, const int* c1, const int* cr, int* ctot);
// out[0..nout) = sum_k w_k^2
void launch_sumsq(cudaStream_t st, int K, const double* w, double* out, int nout);
// out[l] = scale * sum_{e < count} p[l*stride + e]^2
void launch_block_energy(cudaStream_t st, int d, long long count, const double* p,
                         long long stride, double scale, double* out);
// rho[l*ldrho + i] = sum_{k < K} w[l*bsw + k]^2 B[l*bs + i + k*ld]^2, i < rows
void launch_row_energy(cudaStream_t st, int d, int rows, int K, const double* B, int ld,
                       long long bs, const double* w, double* rho, int ldrho, long long bsw = 0);
// w[l*bsw + k*S + j] = |xa_k xb_j| prod_{m != l} sqrt(Nu[m*bsnu + k + j*ldnu]) (the column-
// normalised weights of a Khatri-Rao tensor seen from mode l)
void launch_kr_norm_weights(cudaStream_t st, int d, int Ra, int S, const double* xa,
                            const double* xb, const double* Nu, int ldnu, long long bsnu,
                            double* w, long long bsw);
// mus[s*ldmu + i] = ||S_s y_{s,i}||^2 for slices s < dims[D_R3], i < dims[D_R+1]
void launch_slice_energy(cudaStream_t st, int smax, int rmax, const int* dims, const double* S,
                         long long ldS, const double* V, int ldv, long long bsV, double* mus,
                         int ldmu);
// stage-2 gather of the canonical terms into X_l (rmax x q, ld rmax) of each mode
void launch_gather_terms(cudaStream_t st, int d, int rmax, const int* dims_r, const int* q,
                         int qmax, const double* sigma, const int* tslice, const int* tidx,
                         const double* core, int ldcore, const double* W3, int ldw3,
                         const double* Vs, int ldvs, long long bsVs, double* X, int ldx,
                         long long bsX);
// out[0] = sum_{k<Rx, j<Ry} xi_k eta_j prod_l M_l[k,j]  (square: (xi_k eta_j)^2 in place of
// xi_k eta_j)
void launch_inner_reduce(cudaStream_t st, int d, int Rx, int Ry, const double* xi,
                         const double* eta, const double* M, int ldm, long long bsM, double* out,
                         bool square = false);
void launch_to_full(cudaStream_t st, int d, int n, int R, const double* xi, const double* U0,
                    const double* U1, const double* U2, int ld, double* dense);
// u_hat[i] /= g(rho_i), g = ga rho^-sn + gb rho^sp + gc, rho_i = sum_l lam[l*lstride + i_l]
// (full-format eigenbasis solve)
void launch_full_scale(cudaStream_t st, int d, int n, const double* lam, int lstride, double ga,
                       double sn, double gb, double sp, double gc, double* x);
void launch_copy_weights(cudaStream_t st, int K, const double* src, double scale, double* dst);
// w[(k,j)] = xa[k] * xb[j]
void launch_outer_weights(cudaStream_t st, int Ra, const double* xa, int S, const double* xb,
                          double* w);
// sum of squares of a device vector: out = sum x^2 ; and out = ||core||^2 over live sizes
void launch_core_energy(cudaStream_t st, int d, const double* core, int ldcore, const int* dims,
                        double* out);
// dims bookkeeping for stage 2: dims[3] = min(r1, r2) etc.  (see api.cu for layout)
void launch_stage2_dims(cudaStream_t st, int d, int* dims);

}  // namespace fc

namespace fc {
// Held-out sketch columns that estimate the energy outside the sketched basis.
constexpr int kHold = 8;
// Layout of the per-truncation device dims array (ints).
enum {
    D_R = 0,        // [0..2] Tucker ranks r_l after stage 1
    D_R12 = 3,      // r_0 * r_1 (rows of the core unfolding)
    D_R3 = 4,       // r_2 (d = 3) or 1 (d = 2)
    D_NPER = 5,     // r_1: candidate canonical terms per slice
    D_Q = 6,        // selected canonical rank
    D_C1 = 8,       // [8..10]  sketch rank after pass 1 (per mode)
    D_CR = 11,      // [11..13] rank of the deflated remainder
    D_CT = 14,      // [14..16] combined basis size
    D_C3 = 17,      // [17..19] rank after the final orthonormalisation
    D_FLAG = 23,    // tensor-core error flag of the handle (bounded wait expired); cleared at
                    // the entry of each API call, not by the per-truncation reset of [0, D_FLAG)
    D_SIZE = 24
};
}  // namespace fc
