// Tensor-format kernels of libfc (FP64): symbol factors, Khatri-Rao columns and sketches,
// column normalisation / concatenation (the CP linear combinations of Algorithm 1), traces,
// canonical-term gather, CP inner products, full expansion and the full-format scaling.
#include "fc_common.cuh"
#include "fc_kernels.h"
#include <math.h>

namespace fc {

__global__ void gemm_prescale_kernel(int M, int N, const int* dM, const int* dN, double beta,
                                     double* C, int ldc, long long bsC)
{
    if (dM) M = min(M, *dM);
    if (dN) N = min(N, *dN);
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= M || j >= N) return;
    double* c = C + blockIdx.z * bsC + i + (long long)j * ldc;
    *c = (beta == 0.0) ? 0.0 : beta * (*c);
}

// ---------------------------------------------------------------------------------------
// Symbol factors (eqn:Func_of_rho, Lemma 4.1): term k, mode l:
//   E_l[i, k] = exp(-tau_k lambda_i) * (l == mode_k ? lambda_i : 1),
// normalised to unit columns; xi_k = w_k * prod_l ||E_l[:, k]||.  One CTA per term.
// ---------------------------------------------------------------------------------------
__global__ void build_symbol_kernel(int n, int d, const double* lam, int lstride,
                                    const double* tau, const double* w, const int* mode, double* E,
                                    int lde, long long bsE, double* xi)
{
    __shared__ double red[32];
    const int k = blockIdx.x;
    const double t = tau[k];
    const int mk = mode[k];
    double prod = 1.0;
    for (int l = 0; l < d; ++l) {
        double* col = E + l * bsE + (long long)k * lde;
        double s = 0.0;
        const double* lm = lam + (long long)l * lstride;     // spectrum of mode l
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double v = exp(-t * lm[i]);
            if (l == mk) v *= lm[i];
            col[i] = v;
            s += v * v;
        }
        double nrm = sqrt(block_sum(s, red));
        double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] *= inv;
        prod *= nrm;
        __syncthreads();
    }
    if (threadIdx.x == 0) xi[k] = w[k] * prod;
}

void launch_build_symbol(cudaStream_t st, int n, int d, const double* lam, int lstride,
                         const double* tau, const double* w, const int* mode, int R, double* E,
                         int lde, long long bsE, double* xi)
{
    if (R <= 0) return;
    note_launch(); build_symbol_kernel<<<R, 256, 0, st>>>(n, d, lam, lstride, tau, w, mode, E, lde, bsE, xi);
}

// ---------------------------------------------------------------------------------------
// CP linear combination with normalisation (Algorithm 1: X + a P, R - a S, Z + b P):
// the output lists the columns of piece 0 then piece 1, each mode's column scaled to unit
// norm; weight = scale * xi * prod_l norm.  One CTA per output column.
// ---------------------------------------------------------------------------------------
__global__ void concat_normalize_kernel(int d, int n, Piece p0, Piece p1, double* U, int ldo,
                                        long long bsU, double* w)
{
    __shared__ double red[32];
    const int col = blockIdx.x;
    const Piece& P = (col < p0.K) ? p0 : p1;
    const int k = (col < p0.K) ? col : col - p0.K;
    double prod = 1.0;
    for (int l = 0; l < d; ++l) {
        const double* src = P.U[l] + (long long)k * P.ld;
        double s = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) { double v = src[i]; s += v * v; }
        double nrm = sqrt(block_sum(s, red));
        double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        double* dst = U + l * bsU + (long long)col * ldo;
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i] * inv;
        prod *= nrm;
    }
    if (threadIdx.x == 0) w[col] = P.scale * P.xi[k] * prod;
}

void launch_concat_normalize(cudaStream_t st, int d, int n, Piece p0, Piece p1, double* U,
                             int ldo, long long bsU, double* w)
{
    int K = p0.K + p1.K;
    if (K <= 0) return;
    note_launch(); concat_normalize_kernel<<<K, 128, 0, st>>>(d, n, p0, p1, U, ldo, bsU, w);
}

__global__ void scale_cols_abs_kernel(int n, int K, const double* U, int ldu, long long bsU,
                                      const double* w, double* Y, int ldy, long long bsY)
{
    const int l = blockIdx.y;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % n), k = (int)(e / n);
        Y[l * bsY + i + (long long)k * ldy] = fabs(w[k]) * U[l * bsU + i + (long long)k * ldu];
    }
}

void launch_scale_cols_abs(cudaStream_t st, int d, int n, int K, const double* U, int ldu,
                           long long bsU, const double* w, double* Y, int ldy, long long bsY)
{
    long long tot = (long long)n * K;
    if (tot <= 0) return;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    note_launch(); scale_cols_abs_kernel<<<dim3(blocks, d), 256, 0, st>>>(n, K, U, ldu, bsU, w, Y, ldy, bsY);
}

// p[i + k*ld] *= w[k] for i < rows, k < K (in place)
__global__ void scale_cols_kernel(int rows, int K, double* p, int ld, const double* w)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)rows * K;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), k = (int)(e / rows);
        p[i + (long long)k * ld] *= w[k];
    }
}

void launch_scale_cols(cudaStream_t st, int rows, int K, double* p, int ld, const double* w)
{
    long long tot = (long long)rows * K;
    if (tot <= 0) return;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 4 * 152) blocks = 4 * 152;
    note_launch(); scale_cols_kernel<<<blocks, 256, 0, st>>>(rows, K, p, ld, w);
}

__global__ void kr_cols_kernel(int n, int Ra, int S, const double* E, int lde, long long bsE,
                               const double* xa, const double* Yh, int ldy, long long bsY,
                               const double* xb, int absw, double* Y, int ldo, long long bsO)
{
    const int l = blockIdx.y;
    const long long tot = (long long)n * Ra * S;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % n);
        int kj = (int)(e / n);
        int k = kj / S, j = kj - k * S;
        double s = 1.0;
        if (xa) s = absw ? fabs(xa[k] * xb[j]) : xa[k] * xb[j];
        else if (xb) s = absw ? fabs(xb[j]) : xb[j];
        Y[l * bsO + i + (long long)kj * ldo] =
            s * E[l * bsE + i + (long long)k * lde] * Yh[l * bsY + i + (long long)j * ldy];
    }
}

void launch_kr_cols(cudaStream_t st, int d, int n, int Ra, int S, const double* E, int lde,
                    long long bsE, const double* xa, const double* Yh, int ldy, long long bsY,
                    const double* xb, int absw, double* Y, int ldo, long long bsO)
{
    long long tot = (long long)n * Ra * S;
    if (tot <= 0) return;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    note_launch(); kr_cols_kernel<<<dim3(blocks, d), 256, 0, st>>>(n, Ra, S, E, lde, bsE, xa, Yh, ldy, bsY, xb,
                                                    absw, Y, ldo, bsO);
}

// ---------------------------------------------------------------------------------------
// Counter-based Gaussian numbers for the sketches (splitmix64 + Box-Muller).  The transform
// runs in FP32: a sketch needs Gaussian samples, not FP64-exact ones, and the FP64 log, square
// root and cosine were a third of the sketch contraction's time (the generator runs in the
// operand loader, once per tile that reads the element).  24-bit uniforms, |g| <= 5.8.
// ---------------------------------------------------------------------------------------
FC_DEV unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
FC_DEV double gauss_at(unsigned long long seed, int a, int b) {
    unsigned long long h = mix64(seed ^ mix64(((unsigned long long)(unsigned)a << 32) | (unsigned)b));
    unsigned long long h2 = mix64(h);
    const float u1 = (float)((h >> 40) + 1) * (1.0f / 16777216.0f);   // (0, 1]
    const float u2 = (float)(h2 >> 40) * (1.0f / 16777216.0f);         // [0, 1)
    return (double)(sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2));
}

// B operand: Omega[k, t] * |w_k| with Omega Gaussian; batch item (mode) folds into the seed
struct LdGauss {
    unsigned long long seed; const double* w;
    FC_DEV double operator()(int k, int t, int b) const {
        double s = w ? fabs(w[k]) : 1.0;
        return s * gauss_at(seed + 7919ull * (unsigned long long)b, k, t);
    }
};

void launch_sketch_dense(cudaStream_t st, int prec, int d, int n, int K, int c, const double* U,
                         int ldu, long long bsU, const double* w, unsigned long long seed,
                         double* Y, int ldy, long long bsY)
{
    LdN A{U, ldu, bsU};
    LdGauss B{seed, w};
    gemm_p(prec, st, n, c, K, A, B, 1.0, 0.0, Y, ldy, bsY, d);
}

__global__ void hadamard_kernel(long long count, int n, int c, double* Y, int ldy, long long bsY,
                                const double* T, int ldt, long long bsT)
{
    const int l = blockIdx.y;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % n), t = (int)(e / n);
        Y[l * bsY + i + (long long)t * ldy] *= T[l * bsT + i + (long long)t * ldt];
    }
}

void launch_sketch_kr(cudaStream_t st, int prec, int d, int n, int Ra, int S, int c,
                      const double* E, int lde, long long bsE, const double* xa, const double* Yh,
                      int ldy, long long bsY, const double* xb, unsigned long long seed,
                      double* Y, int ldo, long long bsO, double* tmp)
{
    // Y = E diag|xa| Oa ; tmp = Yh diag|xb| Ob ; Y .= tmp   (Khatri-Rao structured sketch)
    gemm_p(prec, st, n, c, Ra, LdN{E, lde, bsE}, LdGauss{seed, xa}, 1.0, 0.0, Y, ldo, bsO, d);
    gemm_p(prec, st, n, c, S, LdN{Yh, ldy, bsY}, LdGauss{seed ^ 0x5bd1e995ull, xb}, 1.0, 0.0,
           tmp, ldo, bsO, d);
    long long cnt = (long long)n * c;
    int blocks = (int)((cnt + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    note_launch(); hadamard_kernel<<<dim3(blocks, d), 256, 0, st>>>(cnt, n, c, Y, ldo, bsO, tmp, ldo, bsO);
}

// Yr (already Y - Q1 P) columns normalised to unit length, relative to the original column
// norms: a column whose remainder is below relTiny * ||Y[:, t]|| is zeroed.
__global__ void deflate_normalize_kernel(int n, double* Yr, int ld, long long bs,
                                         const double* Yorig, double relTiny)
{
    __shared__ double red[32];
    const int l = blockIdx.y, t = blockIdx.x;
    double* y = Yr + l * bs + (long long)t * ld;
    const double* yo = Yorig + l * bs + (long long)t * ld;
    double s = 0.0, so = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) { s += y[i] * y[i]; so += yo[i] * yo[i]; }
    s = block_sum(s, red);
    so = block_sum(so, red);
    double nrm = sqrt(s);
    double inv = (nrm > relTiny * sqrt(so) && nrm > 0.0) ? 1.0 / nrm : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] *= inv;
}

void launch_deflate_normalize(cudaStream_t st, int d, int n, int c, double* Yr, int ld,
                              long long bs, const double* Yorig, double relTiny)
{
    note_launch(); deflate_normalize_kernel<<<dim3(c, d), 128, 0, st>>>(n, Yr, ld, bs, Yorig, relTiny);
}

__global__ void combine_cols_kernel(int n, int c, double* Q, int ld, long long bs,
                                    const double* Qr, const int* c1, const int* cr, int* ctot)
{
    const int l = blockIdx.y;
    const int off = c1[l];
    const int take = min(cr[l], c - off);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctot[l] = off + max(take, 0);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * c;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        if (j < off) continue;
        double v = 0.0;
        if (j - off < take) v = Qr[l * bs + i + (long long)(j - off) * ld];
        Q[l * bs + i + (long long)j * ld] = v;
    }
}

void launch_combine_cols(cudaStream_t st, int d, int n, int c, double* Q, int ld, long long bs,
                         const double* Qr, const int* c1, const int* cr, int* ctot)
{
    long long cnt = (long long)n * c;
    int blocks = (int)((cnt + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    note_launch(); combine_cols_kernel<<<dim3(blocks, d), 256, 0, st>>>(n, c, Q, ld, bs, Qr, c1, cr, ctot);
}

__global__ void sumsq_kernel(int K, const double* w, double* out, int nout)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) s += w[k] * w[k];
    s = block_sum(s, red);
    if (threadIdx.x < nout) out[threadIdx.x] = s;
}

void launch_sumsq(cudaStream_t st, int K, const double* w, double* out, int nout)
{
    note_launch(); sumsq_kernel<<<1, 256, 0, st>>>(K, w, out, nout);
}

__global__ void block_energy_kernel(long long count, const double* p, long long stride,
                                    double scale, double* out)
{
    __shared__ double red[32];
    const int l = blockIdx.x;
    double s = 0.0;
    for (long long e = threadIdx.x; e < count; e += blockDim.x) {
        double v = p[l * stride + e];
        s += v * v;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[l] = scale * s;
}

void launch_block_energy(cudaStream_t st, int d, long long count, const double* p,
                         long long stride, double scale, double* out)
{
    note_launch(); block_energy_kernel<<<d, 512, 0, st>>>(count, p, stride, scale, out);
}

// one CTA per (row i, mode l): sum over the K columns of a row of a column-major matrix
__global__ void row_energy_kernel(int K, const double* B, int ld, long long bs, const double* w,
                                  long long bsw, double* rho, int ldrho)
{
    __shared__ double red[32];
    const int i = blockIdx.x, l = blockIdx.y;
    const double* row = B + l * bs + i;
    const double* wl = w + l * bsw;
    double s = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double v = wl[k] * row[(long long)k * ld];
        s += v * v;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) rho[(long long)l * ldrho + i] = s;
}

void launch_row_energy(cudaStream_t st, int d, int rows, int K, const double* B, int ld,
                       long long bs, const double* w, double* rho, int ldrho, long long bsw)
{
    if (rows <= 0) return;
    note_launch();
    row_energy_kernel<<<dim3(rows, d), 256, 0, st>>>(K, B, ld, bs, w, bsw, rho, ldrho);
}

// Column-normalised weights of a Khatri-Rao tensor, seen from mode l: the term (k, j) with
// factors e_mk . y_mj has the normalised weight |xa_k xb_j| prod_m nu_m(k, j); its unit mode-l
// column is (e_lk . y_lj) / nu_l, so in mode l's side matrix the column e_lk . y_lj carries
// w_l[k S + j] = |xa_k xb_j| prod_{m != l} nu_m(k, j),  nu_m^2 = Nu[m bsnu + k + j ldnu].
__global__ void kr_norm_weights_kernel(int d, int Ra, int S, const double* xa, const double* xb,
                                       const double* Nu, int ldnu, long long bsnu, double* w,
                                       long long bsw)
{
    const int l = blockIdx.y;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ra * S; e += gridDim.x * blockDim.x) {
        const int k = e / S, j = e - k * S;
        double v = fabs(xa[k] * xb[j]);
        for (int m = 0; m < d; ++m)
            if (m != l) v *= sqrt(fmax(Nu[m * bsnu + k + (long long)j * ldnu], 0.0));
        w[l * bsw + e] = v;
    }
}

void launch_kr_norm_weights(cudaStream_t st, int d, int Ra, int S, const double* xa,
                            const double* xb, const double* Nu, int ldnu, long long bsnu,
                            double* w, long long bsw)
{
    const int tot = Ra * S;
    if (tot <= 0) return;
    note_launch();
    kr_norm_weights_kernel<<<dim3(std::min((tot + 255) / 256, 1024), d), 256, 0, st>>>(
        d, Ra, S, xa, xb, Nu, ldnu, bsnu, w, bsw);
}

// mus[s*ldmu + i] = ||S_s y_i||^2, S_s compact r0 x r1 at S + s*ldS (element (a,b) at a + r0 b),
// y_i = column i of V + s*bsV (ld ldv).  One CTA per slice, one warp per candidate i.
__global__ void slice_energy_kernel(int rmax, const int* dims, const double* S, long long ldS,
                                    const double* V, int ldv, long long bsV, double* mus, int ldmu)
{
    const int s = blockIdx.x;
    if (s >= dims[D_R3]) return;
    const int r0 = dims[D_R + 0], r1 = dims[D_R + 1];
    const double* Ss = S + s * ldS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < r1; i += nw) {
        const double* y = V + s * bsV + (long long)i * ldv;
        double e = 0.0;
        for (int a = lane; a < r0; a += 32) {
            double v = 0.0;
            for (int b = 0; b < r1; ++b) v += Ss[a + r0 * b] * y[b];
            e += v * v;
        }
        e = warp_sum(e);
        if (lane == 0) mus[(long long)s * ldmu + i] = e;
    }
    (void)rmax;
}

void launch_slice_energy(cudaStream_t st, int smax, int rmax, const int* dims, const double* S,
                         long long ldS, const double* V, int ldv, long long bsV, double* mus,
                         int ldmu)
{
    if (smax <= 0) return;
    note_launch(); slice_energy_kernel<<<smax, 256, 0, st>>>(rmax, dims, S, ldS, V, ldv, bsV, mus, ldmu);
}

// ---------------------------------------------------------------------------------------
// Stage-2 gather (eqn:two_level): kept term t = (slice s, index i), sigma_t:
//   X_0[:, t] = S_s y_{s,i} / sigma_t   (S_s = slice s of the rotated core, r0 x r1 compact)
//   X_1[:, t] = y_{s,i}                 (eigenvector i of S_s^T S_s)
//   X_2[:, t] = W3[:, s]                (d = 3: mode-3 singular vector of the core)
// Rows beyond the live Tucker ranks are zero.  One CTA per term.
// ---------------------------------------------------------------------------------------
__global__ void gather_terms_kernel(int d, int rmax, const int* dims, const double* sigma,
                                    const int* tslice, const int* tidx, const double* core,
                                    int ldcore, const double* W3, int ldw3, const double* Vs,
                                    int ldvs, long long bsVs, double* X, int ldx, long long bsX)
{
    const int t = blockIdx.x;
    if (t >= dims[D_Q]) return;
    const int r0 = dims[D_R + 0], r1 = dims[D_R + 1];
    const int s = tslice[t], i = tidx[t];
    const double sg = sigma[t];
    const double* y = Vs + s * bsVs + (long long)i * ldvs;
    const double* Ss = core + (long long)s * ldcore;
    for (int a = threadIdx.x; a < rmax; a += blockDim.x) {
        double v = 0.0;
        if (a < r0) {
            for (int b = 0; b < r1; ++b) v += Ss[a + r0 * b] * y[b];
            v = sg > 0.0 ? v / sg : 0.0;
        }
        X[0 * bsX + a + (long long)t * ldx] = v;
        X[1 * bsX + a + (long long)t * ldx] = (a < r1) ? y[a] : 0.0;
        if (d == 3) X[2 * bsX + a + (long long)t * ldx] = (a < dims[D_R + 2]) ? W3[a + (long long)s * ldw3] : 0.0;
    }
}

void launch_gather_terms(cudaStream_t st, int d, int rmax, const int* dims_r, const int* q,
                         int qmax, const double* sigma, const int* tslice, const int* tidx,
                         const double* core, int ldcore, const double* W3, int ldw3,
                         const double* Vs, int ldvs, long long bsVs, double* X, int ldx,
                         long long bsX)
{
    (void)q;
    if (qmax <= 0) return;
    note_launch(); gather_terms_kernel<<<qmax, 64, 0, st>>>(d, rmax, dims_r, sigma, tslice, tidx, core, ldcore,
                                             W3, ldw3, Vs, ldvs, bsVs, X, ldx, bsX);
}

// <X, Y> = sum_{k,j} xi_k eta_j prod_l M_l[k, j]  (M_l = U_l^T V_l)
__global__ void inner_reduce_kernel(int d, int Rx, int Ry, const double* xi, const double* eta,
                                    const double* M, int ldm, long long bsM, double* out,
                                    int square)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int e = threadIdx.x; e < Rx * Ry; e += blockDim.x) {
        int k = e % Rx, j = e / Rx;
        double p = xi[k] * eta[j];
        if (square) p *= p;
        for (int l = 0; l < d; ++l) p *= M[l * bsM + k + (long long)j * ldm];
        s += p;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[0] = s;
}

void launch_inner_reduce(cudaStream_t st, int d, int Rx, int Ry, const double* xi,
                         const double* eta, const double* M, int ldm, long long bsM, double* out,
                         bool square)
{
    note_launch();
    inner_reduce_kernel<<<1, 1024, 0, st>>>(d, Rx, Ry, xi, eta, M, ldm, bsM, out, square ? 1 : 0);
}

// full expansion, column-major with i_1 fastest
__global__ void to_full_kernel(int d, int n, int R, const double* xi, const double* U0,
                               const double* U1, const double* U2, int ld, double* dense)
{
    const long long tot = (d == 3) ? (long long)n * n * n : (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int i0 = (int)(e % n);
        long long rest = e / n;
        int i1 = (int)(rest % n);
        int i2 = (int)(rest / n);
        double s = 0.0;
        for (int r = 0; r < R; ++r) {
            double v = xi[r] * U0[i0 + (long long)r * ld] * U1[i1 + (long long)r * ld];
            if (d == 3) v *= U2[i2 + (long long)r * ld];
            s += v;
        }
        dense[e] = s;
    }
}

void launch_to_full(cudaStream_t st, int d, int n, int R, const double* xi, const double* U0,
                    const double* U1, const double* U2, int ld, double* dense)
{
    long long tot = (d == 3) ? (long long)n * n * n : (long long)n * n;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    note_launch(); to_full_kernel<<<blocks, 256, 0, st>>>(d, n, R, xi, U0, U1, U2, ld, dense);
}

__global__ void full_scale_kernel(int d, int n, const double* lam, int lstride, double ga,
                                  double sn, double gb, double sp, double gc, double* x)
{
    const long long tot = (d == 3) ? (long long)n * n * n : (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int i0 = (int)(e % n);
        long long rest = e / n;
        int i1 = (int)(rest % n);
        int i2 = (int)(rest / n);
        double rho = lam[i0] + lam[lstride + i1] + (d == 3 ? lam[2 * lstride + i2] : 0.0);
        double g = gc;
        if (ga != 0.0) g += ga * pow(rho, -sn);
        if (gb != 0.0) g += gb * pow(rho, sp);
        x[e] /= g;
    }
}

void launch_full_scale(cudaStream_t st, int d, int n, const double* lam, int lstride, double ga,
                       double sn, double gb, double sp, double gc, double* x)
{
    long long tot = (d == 3) ? (long long)n * n * n : (long long)n * n;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    note_launch(); full_scale_kernel<<<blocks, 256, 0, st>>>(d, n, lam, lstride, ga, sn, gb, sp, gc, x);
}

__global__ void copy_weights_kernel(int K, const double* src, double scale, double* dst)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
        dst[k] = scale * src[k];
}

void launch_copy_weights(cudaStream_t st, int K, const double* src, double scale, double* dst)
{
    if (K <= 0) return;
    note_launch(); copy_weights_kernel<<<(K + 255) / 256, 256, 0, st>>>(K, src, scale, dst);
}

__global__ void outer_weights_kernel(int Ra, const double* xa, int S, const double* xb, double* w)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ra * S; e += gridDim.x * blockDim.x) {
        int k = e / S, j = e - k * S;
        w[e] = xa[k] * xb[j];
    }
}

void launch_outer_weights(cudaStream_t st, int Ra, const double* xa, int S, const double* xb,
                          double* w)
{
    int tot = Ra * S;
    if (tot <= 0) return;
    note_launch(); outer_weights_kernel<<<(tot + 255) / 256, 256, 0, st>>>(Ra, xa, S, xb, w);
}

// ||core||_F^2 over the live part: core is (r0 r1) x r3 compact rows, column stride ldcore
__global__ void core_energy_kernel(const double* core, int ldcore, const int* dims, double* out)
{
    __shared__ double red[32];
    const int r12 = dims[D_R12], r3 = dims[D_R3];
    double s = 0.0;
    for (long long e = threadIdx.x; e < (long long)r12 * r3; e += blockDim.x) {
        int a = (int)(e % r12), c = (int)(e / r12);
        double v = core[a + (long long)c * ldcore];
        s += v * v;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[0] = s;
}

void launch_core_energy(cudaStream_t st, int d, const double* core, int ldcore, const int* dims,
                        double* out)
{
    (void)d;
    note_launch(); core_energy_kernel<<<1, 1024, 0, st>>>(core, ldcore, dims, out);
}

__global__ void stage2_dims_kernel(int d, int* dims)
{
    if (threadIdx.x != 0) return;
    int r0 = dims[D_R + 0], r1 = dims[D_R + 1];
    dims[D_R12] = r0 * r1;
    dims[D_R3] = (d == 3) ? dims[D_R + 2] : 1;
    dims[D_NPER] = r1;
}

void launch_stage2_dims(cudaStream_t st, int d, int* dims)
{
    note_launch(); stage2_dims_kernel<<<1, 32, 0, st>>>(d, dims);
}

}  // namespace fc
