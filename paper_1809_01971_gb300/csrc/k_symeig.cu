// Symmetric eigen-decomposition of small FP64 matrices (m <= kMaxC = 64), one CTA per matrix.
// It orders the bases of the RHOSVD truncation (Section 5): the Rayleigh-Ritz matrix of the
// sketched side matrices, the mode-3 Gram of the Tucker core and the core slices' Grams.
//
// Steps (textbook dense symmetric eigen-solver, Golub & Van Loan Ch. 8):
//   1. Householder tridiagonalisation A = Q T Q^T; the reflectors stay in A's lower triangle.
//   2. Eigenvalues of T by bisection on Sturm-sequence counts, one thread per eigenvalue; the
//      brackets come from counts on a geometric grid of 256 points (one per thread).
//   3. Eigenvectors of T by inverse iteration (tridiagonal LU with partial pivoting), one
//      thread per eigenvector, then Gram-Schmidt (two passes) in order of decreasing
//      eigenvalue, so that vectors of close eigenvalues come out orthonormal.
//   4. Back-transformation V = Q Z.
// The matrix is scaled to unit Frobenius norm first, which keeps the Sturm recurrence in
// range and makes all tolerances absolute.  Flops ~ (4/3 + 2 + 2) m^3 against ~100 m^3 for a
// cyclic Jacobi solve; on GB300 (2 FP64 FMA per clock per SM) that is what decides the time.
// Eigenvalues are accurate to ~u ||A|| in absolute terms (as for any backward-stable method);
// the eigenvectors are orthonormal to ~u.
#include "fc_common.cuh"
#include "fc_kernels.h"

namespace fc {

// Algorithmic work of the instrumented eigen-solves (fc_prof_*): a symmetric eigen-
// decomposition with eigenvectors counts 9 m^3 flops (the textbook dense figure).
__device__ unsigned long long g_prof_work = 0;

unsigned long long* prof_work_counter()
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_prof_work) != cudaSuccess) return nullptr;
    return static_cast<unsigned long long*>(p);
}

namespace {

constexpr int kEigThreads = 256;
constexpr int kGrid = 256;            // bracket grid: one Sturm count per thread
constexpr double kTolAbs = 4e-16;     // bisection stops at this width (matrix scaled to norm 1)

FC_DEV bool neg(double x) { return __double_as_longlong(x) < 0; }

// Number of eigenvalues of the symmetric tridiagonal (d, e) below sigma: sign changes of the
// Sturm sequence p_0 = 1, p_1 = d_0 - sigma, p_k = (d_{k-1} - sigma) p_{k-1} - e_{k-2}^2 p_{k-2}
// (a zero term takes the sign opposite to its predecessor).  With ||T|| <= 1 a term grows by at
// most 3x per step, so only underflow needs guarding: every 8 steps the pair is rescaled.
FC_DEV int sturm_below(const double* d, const double* e2, int m, double sigma) {
    double pm2 = 1.0, pm1 = d[0] - sigma;
    if (pm1 == 0.0) pm1 = -1e-300;
    int cnt = neg(pm1);
    for (int k = 1; k < m; ++k) {
        double p = fma(d[k] - sigma, pm1, -e2[k - 1] * pm2);
        if ((__double_as_longlong(p) << 1) == 0) p = neg(pm1) ? 1e-300 : -1e-300;
        cnt += (neg(p) != neg(pm1));
        if ((k & 7) == 0) {
            int ex = (int)((__double_as_longlong(p) >> 52) & 0x7ff);
            if (ex < 1023 - 300) { p *= 0x1p+600; pm1 *= 0x1p+600; }
        }
        pm2 = pm1;
        pm1 = p;
    }
    return cnt;
}

// x <- (T - lam I)^-1 x for the tridiagonal (d, e) (x in shared memory, stride xs), by an LU
// factorisation with partial pivoting computed once per call; pivots below tol are replaced
// by +-tol.  u0/u1/u2: the three diagonals of U (u0 stored inverted), l: multipliers,
// sw: row swap at step k.
struct TriLU {
    double u0[kMaxC], u1[kMaxC], u2[kMaxC], l[kMaxC];
    unsigned char sw[kMaxC];
};

FC_DEV void tri_factor(const double* d, const double* e, int m, double lam, double tol, TriLU& f) {
    double a = d[0] - lam, c = (m > 1) ? e[0] : 0.0, g = 0.0;
    for (int k = 0; k + 1 < m; ++k) {
        const double b = e[k], a1 = d[k + 1] - lam, c1 = (k + 2 < m) ? e[k + 1] : 0.0;
        if (fabs(a) >= fabs(b)) {
            if (fabs(a) < tol) a = neg(a) ? -tol : tol;
            const double mult = b / a;
            f.u0[k] = 1.0 / a; f.u1[k] = c; f.u2[k] = g; f.l[k] = mult; f.sw[k] = 0;
            a = a1 - mult * c;
            c = c1 - mult * g;
            g = 0.0;
        } else {
            const double mult = a / b;
            f.u0[k] = 1.0 / b; f.u1[k] = a1; f.u2[k] = c1; f.l[k] = mult; f.sw[k] = 1;
            const double na = c - mult * a1, nc = g - mult * c1;
            a = na;
            c = nc;
            g = 0.0;
        }
    }
    if (fabs(a) < tol) a = neg(a) ? -tol : tol;
    f.u0[m - 1] = 1.0 / a;
}

FC_DEV void tri_solve(const TriLU& f, int m, double* x, int xs) {
    for (int k = 0; k + 1 < m; ++k) {
        if (f.sw[k]) { double t = x[k * xs]; x[k * xs] = x[(k + 1) * xs]; x[(k + 1) * xs] = t; }
        x[(k + 1) * xs] -= f.l[k] * x[k * xs];
    }
    x[(m - 1) * xs] *= f.u0[m - 1];
    if (m >= 2) x[(m - 2) * xs] = (x[(m - 2) * xs] - f.u1[m - 2] * x[(m - 1) * xs]) * f.u0[m - 2];
    for (int k = m - 3; k >= 0; --k)
        x[k * xs] = (x[k * xs] - f.u1[k] * x[(k + 1) * xs] - f.u2[k] * x[(k + 2) * xs]) * f.u0[k];
}

}  // namespace

__global__ void __launch_bounds__(kEigThreads)
symeig_kernel(const double* __restrict__ A, int lda, long long bsA, const int* __restrict__ dims,
              int dstride, int cmax, double* __restrict__ ev, long long bsE,
              double* __restrict__ V, int ldv, long long bsV, int prof)
{
    extern __shared__ double sm[];
    const int b = blockIdx.x, tid = threadIdx.x;
    int m = cmax;
    if (dims) m = min(dims[b * dstride], cmax);
    if (m < 0) m = 0;
    if (prof && tid == 0) atomicAdd(&g_prof_work, 9ull * (unsigned long long)m * m * m);
    const int S = kMaxC + 1;
    double* a = sm;                      // m x S, row-major: a[i*S + j]
    double* z = a + kMaxC * S;           // eigenvectors of T, column c = eigenvalue rank c
    double* d = z + kMaxC * S;
    double* e = d + kMaxC;
    double* e2 = e + kMaxC;
    double* tau = e2 + kMaxC;
    double* lam = tau + kMaxC;           // ascending
    double* wv = lam + kMaxC;            // work vector (p / w of the reflector update)
    double* coef = wv + kMaxC;           // Gram-Schmidt coefficients
    double* gpt = coef + kMaxC;          // grid points (kGrid)
    int* gcnt = (int*)(gpt + kGrid);     // counts at the grid points
    __shared__ double red[32];
    __shared__ double sh_scal[4];

    const double* Ab = A + b * bsA;
    double* evb = ev + b * bsE;
    double* Vb = V + b * bsV;
    for (int e_ = tid; e_ < cmax * cmax; e_ += blockDim.x) Vb[(e_ % cmax) + (long long)(e_ / cmax) * ldv] = 0.0;
    for (int i = tid; i < cmax; i += blockDim.x) evb[i] = 0.0;
    if (m == 0) return;

    // ---- load (symmetrised) and scale to unit Frobenius norm -----------------------------
    double fro = 0.0;
    for (int e_ = tid; e_ < m * m; e_ += blockDim.x) {
        int i = e_ % m, j = e_ / m;
        double x = 0.5 * (Ab[i + (long long)j * lda] + Ab[j + (long long)i * lda]);
        a[i * S + j] = x;
        fro += x * x;
    }
    fro = sqrt(block_sum(fro, red));
    if (!(fro > 0.0) || !isfinite(fro)) {
        // zero (or non-finite) matrix: eigenvalues 0, V = I
        __syncthreads();
        for (int i = tid; i < m; i += blockDim.x) Vb[i + (long long)i * ldv] = 1.0;
        return;
    }
    const double inv = 1.0 / fro;
    for (int e_ = tid; e_ < m * m; e_ += blockDim.x) a[(e_ / m) * S + (e_ % m)] *= inv;
    __syncthreads();

    // ---- 1. Householder tridiagonalisation ------------------------------------------------
    for (int k = 0; k + 2 < m; ++k) {
        const int L = m - k - 1;                        // rows k+1 .. m-1
        double s = 0.0;
        for (int i = 1 + tid; i < L; i += blockDim.x) { double x = a[(k + 1 + i) * S + k]; s += x * x; }
        const double sigma = block_sum(s, red);
        const double alpha = a[(k + 1) * S + k];
        if (tid == 0) {
            d[k] = a[k * S + k];
            if (sigma == 0.0) {
                tau[k] = 0.0;
                e[k] = alpha;
                sh_scal[0] = 0.0;
            } else {
                const double mu = sqrt(alpha * alpha + sigma);
                const double beta = (alpha <= 0.0) ? mu : -mu;
                tau[k] = (beta - alpha) / beta;
                e[k] = beta;
                sh_scal[0] = 1.0 / (alpha - beta);
            }
        }
        __syncthreads();
        const double t = tau[k];
        if (t == 0.0) continue;
        const double sc = sh_scal[0];
        for (int i = 1 + tid; i < L; i += blockDim.x) a[(k + 1 + i) * S + k] *= sc;
        if (tid == 0) a[(k + 1) * S + k] = 1.0;
        __syncthreads();
        // p = t A22 v ; K = t/2 v^T p ; w = p - K v ; A22 -= v w^T + w v^T
        double kk = 0.0;
        for (int r = tid; r < L; r += blockDim.x) {
            double acc = 0.0;
            const double* row = a + (k + 1 + r) * S + (k + 1);
            for (int c = 0; c < L; ++c) acc = fma(row[c], a[(k + 1 + c) * S + k], acc);
            acc *= t;
            wv[r] = acc;
            kk += acc * a[(k + 1 + r) * S + k];
        }
        const double K = 0.5 * t * block_sum(kk, red);
        for (int r = tid; r < L; r += blockDim.x) wv[r] -= K * a[(k + 1 + r) * S + k];
        __syncthreads();
        for (int e_ = tid; e_ < L * L; e_ += blockDim.x) {
            const int r = e_ / L, c = e_ - r * L;
            const double vr = a[(k + 1 + r) * S + k], vc = a[(k + 1 + c) * S + k];
            a[(k + 1 + r) * S + (k + 1 + c)] -= vr * wv[c] + wv[r] * vc;
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (m >= 2) {
            d[m - 2] = a[(m - 2) * S + (m - 2)];
            e[m - 2] = a[(m - 1) * S + (m - 2)];
            tau[m - 2] = 0.0;
        }
        d[m - 1] = a[(m - 1) * S + (m - 1)];
        e[m - 1] = 0.0;
        tau[m - 1] = 0.0;
    }
    __syncthreads();
    for (int i = tid; i < m; i += blockDim.x) e2[i] = e[i] * e[i];
    __syncthreads();

    // ---- 2. eigenvalues: grid of counts, then bisection per eigenvalue ---------------------
    // grid: +-10^(-g/8), g = 0..127 (covers the scaled spectrum [-1, 1] down to 1e-16)
    {
        const int g = tid;
        double x = exp10(-(double)(g & 127) / 8.0);
        if (g >= 128) x = -x;
        gpt[g] = x;
        gcnt[g] = sturm_below(d, e2, m, x);
    }
    __syncthreads();
    const int c0 = sturm_below(d, e2, m, 0.0);    // eigenvalues below 0 (computed redundantly)
    if (tid < m) {
        const int j = tid;                          // j-th smallest eigenvalue
        double lo = -1.0000001, hi = 1.0000001;     // |lambda| <= ||T||_F = 1
        if (j < c0) hi = 0.0; else lo = 0.0;
        for (int g = 0; g < kGrid; ++g) {
            const double x = gpt[g];
            const int cnt = gcnt[g];
            if (cnt <= j && x > lo) lo = x;         // at most j eigenvalues below x
            if (cnt > j && x < hi) hi = x;
        }
        for (int it = 0; it < 80 && hi - lo > kTolAbs; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (sturm_below(d, e2, m, mid) > j) hi = mid; else lo = mid;
        }
        lam[j] = 0.5 * (lo + hi);
    }
    __syncthreads();

    // ---- 3. eigenvectors of T: inverse iteration, then Gram-Schmidt ----------------------
    // column c of z holds the eigenvector of the c-th largest eigenvalue
    if (tid < m) {
        const int j = tid, c = m - 1 - j;
        TriLU f;
        tri_factor(d, e, m, lam[j], 4e-16, f);
        double* x = z + c;
        unsigned int h = 0x9E3779B9u * (unsigned)(j + 1);
        for (int i = 0; i < m; ++i) {
            h ^= h << 13; h ^= h >> 17; h ^= h << 5;
            x[i * S] = 1.0 + 0.25 * ((double)(h & 0xffff) / 65536.0 - 0.5);
        }
        for (int it = 0; it < 3; ++it) {
            tri_solve(f, m, x, S);
            double mx = 0.0;
            for (int i = 0; i < m; ++i) mx = fmax(mx, fabs(x[i * S]));
            const double s_ = (mx > 0.0 && isfinite(mx)) ? 1.0 / mx : 0.0;
            for (int i = 0; i < m; ++i) x[i * S] *= s_;
        }
    }
    __syncthreads();
    for (int c = 0; c < m; ++c) {
        // two classical Gram-Schmidt passes against columns 0..c-1, then normalise; a column
        // that vanishes (repeated eigenvalue) is replaced by unit vectors until one survives
        for (int attempt = 0; attempt <= m; ++attempt) {
            double n0 = 0.0;
            for (int i = tid; i < m; i += blockDim.x) n0 += z[i * S + c] * z[i * S + c];
            n0 = block_sum(n0, red);
            for (int pass = 0; pass < 2; ++pass) {
                for (int q = tid; q < c; q += blockDim.x) {
                    double s_ = 0.0;
                    for (int i = 0; i < m; ++i) s_ = fma(z[i * S + q], z[i * S + c], s_);
                    coef[q] = s_;
                }
                __syncthreads();
                for (int i = tid; i < m; i += blockDim.x) {
                    double s_ = z[i * S + c];
                    for (int q = 0; q < c; ++q) s_ = fma(-coef[q], z[i * S + q], s_);
                    z[i * S + c] = s_;
                }
                __syncthreads();
            }
            double n1 = 0.0;
            for (int i = tid; i < m; i += blockDim.x) n1 += z[i * S + c] * z[i * S + c];
            n1 = block_sum(n1, red);
            if (n1 > 1e-6 * n0 && n1 > 0.0 && isfinite(n1)) {
                const double s_ = 1.0 / sqrt(n1);
                for (int i = tid; i < m; i += blockDim.x) z[i * S + c] *= s_;
                __syncthreads();
                break;
            }
            // replace by the unit vector e_((c + attempt) mod m) and orthogonalise again
            for (int i = tid; i < m; i += blockDim.x) z[i * S + c] = (i == (c + attempt) % m) ? 1.0 : 0.0;
            __syncthreads();
        }
    }

    // ---- 4. back-transformation V = H_0 H_1 ... H_{m-3} Z --------------------------------
    for (int k = m - 3; k >= 0; --k) {
        const double t = tau[k];
        if (t == 0.0) continue;                      // uniform across the block
        const int L = m - k - 1;
        for (int c = tid; c < m; c += blockDim.x) {
            double s_ = 0.0;
            for (int i = 0; i < L; ++i) s_ = fma(a[(k + 1 + i) * S + k], z[(k + 1 + i) * S + c], s_);
            coef[c] = t * s_;
        }
        __syncthreads();
        for (int e_ = tid; e_ < L * m; e_ += blockDim.x) {
            const int i = e_ / m, c = e_ - i * m;
            z[(k + 1 + i) * S + c] -= a[(k + 1 + i) * S + k] * coef[c];
        }
        __syncthreads();
    }

    // ---- outputs: eigenvalues descending (unscaled), eigenvectors as columns -------------
    for (int c = tid; c < m; c += blockDim.x) evb[c] = fro * lam[m - 1 - c];
    for (int e_ = tid; e_ < m * m; e_ += blockDim.x) {
        const int i = e_ % m, c = e_ / m;
        Vb[i + (long long)c * ldv] = z[i * S + c];
    }
}

// ---------------------------------------------------------------------------------------
// Graded eigen-solver for the truncation: cyclic Jacobi sweeps in FP32 on the matrix scaled
// by its largest diagonal entry, then FP64 orthonormalisation of the eigenvectors.
//
// The RHOSVD's Gram matrices are graded (their basis comes from a pivoted Cholesky-QR, so the
// diagonal falls from ~1 to ~1e-18); two-sided Jacobi determines the eigen-directions of a
// graded positive definite matrix to high *relative* accuracy, entry by entry (Demmel and
// Veselic, 1992), which Householder reduction does not: with Householder the small
// directions mix and the truncation keeps up to all sketch columns, with Jacobi it reaches
// the optimal rank.  FP32 keeps that grading (it stores each entry with 1e-7 relative
// precision) at 64x GB300's FP64 rate; the eigenvectors are then made orthonormal to FP64
// precision by Cholesky-QR taken in order of *increasing* eigenvalue, so a direction only
// ever absorbs components of smaller ones (never a large one leaking into a small one).
// Eigenvalues: FP64 Rayleigh quotients of the final vectors if `rq`, else the FP32 values.
// ---------------------------------------------------------------------------------------
constexpr int kGjThreads = 1024;

__global__ void __launch_bounds__(kGjThreads, 1)
gjacobi_kernel(const double* __restrict__ A, int lda, long long bsA, const int* __restrict__ dims,
               int dstride, int cmax, double* __restrict__ ev, long long bsE,
               double* __restrict__ V, int ldv, long long bsV, int rq, float floorRel, int prof,
               const double* __restrict__ floorAbs, double floorFrac)
{
    extern __shared__ double sm[];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
    int c = cmax;
    if (dims) c = min(dims[b * dstride], cmax);
    if (c < 0) c = 0;
    if (prof && tid == 0) atomicAdd(&g_prof_work, 9ull * (unsigned long long)c * c * c);
    const int S = kMaxC + 1;
    double* A64 = sm;                      // c x S  input (FP64), for the Rayleigh quotients
    double* G = A64 + kMaxC * S;           // c x S  Gram -> Cholesky factor L -> output vectors
    double* Li = G + kMaxC * S;            // c x S  L^-1 (lower triangle)
    float2* Lf = (float2*)(Li + kMaxC * S);   // c x S  L^-1 as double-float pairs
    float* a = (float*)(Lf + kMaxC * S);   // m x S (FP32 working matrix)
    float* v = a + kMaxC * S;              // m x S (FP32 eigenvectors, row-major v[r*S+col])
    float2* cso = (float2*)(v + kMaxC * S);  // (cos, sin) of each pair's rotation; sin = 0: none
    int* order = (int*)(cso + kMaxC);      // ascending eigenvalue order
    int* pairs = order + kMaxC;            // (m-1) x m/2 round-robin pairs, p | q << 8
    __shared__ double red[32];
    __shared__ double dinv[kMaxC];         // 1 / L_kk of the Cholesky-QR
    __shared__ int anyRot;
    __shared__ int roundRot[kMaxC];        // per round of a sweep: some pair rotates

    const double* Ab = A + b * bsA;
    double* evb = ev + b * bsE;
    double* Vb = V + b * bsV;
    for (int e_ = tid; e_ < cmax * cmax; e_ += blockDim.x) Vb[(e_ % cmax) + (long long)(e_ / cmax) * ldv] = 0.0;
    for (int i = tid; i < cmax; i += blockDim.x) evb[i] = 0.0;
    if (c == 0) return;
    const int m = (c + 1) & ~1;           // even number of players (padded with a zero row)

    double dmax = 0.0;
    for (int e_ = tid; e_ < c * c; e_ += blockDim.x) {
        const int i = e_ % c, j = e_ / c;
        const double x = 0.5 * (Ab[i + (long long)j * lda] + Ab[j + (long long)i * lda]);
        A64[i * S + j] = x;
        if (i == j) dmax = fmax(dmax, fabs(x));
    }
    dmax = warp_max(dmax);
    if (lane == 0) red[wid] = dmax;
    __syncthreads();
    if (tid < 32) {
        double t = (tid < nwarp) ? red[tid] : 0.0;
        t = warp_max(t);
        if (tid == 0) red[0] = t;
    }
    __syncthreads();
    dmax = red[0];
    __syncthreads();
    if (!(dmax > 0.0) || !isfinite(dmax)) {
        for (int i = tid; i < c; i += blockDim.x) Vb[i + (long long)i * ldv] = 1.0;
        return;
    }
    const double sc = 1.0 / dmax;
    // absolute floor (energy units): off-diagonal entries below floorFrac * (*floorAbs) cannot
    // change a rank decision taken from projected energies; relative to the scaled matrix
    if (floorAbs) {
        const double fa = floorFrac * (*floorAbs) * sc;
        if (fa > (double)floorRel) floorRel = (float)fmin(fa, 1.0);
    }
    for (int e_ = tid; e_ < m * m; e_ += blockDim.x) {
        const int i = e_ % m, j = e_ / m;
        a[i * S + j] = (i < c && j < c) ? (float)(A64[i * S + j] * sc) : 0.0f;
        v[i * S + j] = (i == j) ? 1.0f : 0.0f;
    }

    // ---- FP32 cyclic Jacobi, round-robin pairing (m/2 disjoint rotations per round) -------
    // pair i of round rnd: (rnd, m-1) for i = 0, else ((rnd+i) mod (m-1), (rnd-i) mod (m-1));
    // the table is built once; each pair's rotation J = [[c, s], [-s, c]] acts on (p < q).
    // One round: the m/2 rotation parameters (one warp), then every 2x2 block of A (J^T A J)
    // and every row pair of V (V J) in one pass over the block's threads.
    const int half = m / 2;
    for (int e_ = tid; e_ < (m - 1) * half; e_ += blockDim.x) {
        const int rnd = e_ / half, i = e_ - rnd * half;
        int p, q;
        if (i == 0) { p = rnd; q = m - 1; }
        else { p = (rnd + i) % (m - 1); q = (rnd - i + (m - 1)) % (m - 1); }
        if (p > q) { int t = p; p = q; q = t; }
        pairs[e_] = p | (q << 8);
    }
    __syncthreads();
    // this thread's work items of a round, the same in every round (no index division in the
    // sweeps): kind 0 = 2x2 block (pair pi rows, pair pj columns) of A, kind 1 = row r of V
    // on pair pi; at most 3 items per thread (m <= 64: 32^2 + 64 * 32 <= 3 * 1024)
    const int nblk = half * half, nwork = nblk + m * half;
    int itA[3], itB[3], nit = 0;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int e_ = tid + t * kGjThreads;
        itA[t] = 0; itB[t] = 0;
        if (e_ < nblk) { itA[t] = e_ % half; itB[t] = e_ / half; nit = t + 1; }
        else if (e_ < nwork) { const int e2 = e_ - nblk; itA[t] = -1 - e2 % m; itB[t] = e2 / m; nit = t + 1; }
    }
    for (int sweep = 0; sweep < 15; ++sweep) {
        // A sweep rotates some pair only if some off-diagonal entry passes the rotation test
        // now (a round without rotations leaves the matrix as it is), so one pass over all
        // entries with the same test ends the iteration without a sweep of empty rounds.
        int hot = 0;
        for (int e_ = tid; e_ < m * m; e_ += blockDim.x) {
            const int p = e_ % m, q = e_ / m;
            if (p < q) {
                const float app = a[p * S + p], aqq = a[q * S + q], apq = a[p * S + q];
                if (fabsf(apq) > fmaxf(1e-6f * sqrtf(fabsf(app * aqq)), floorRel)) hot = 1;
            }
        }
        if (!__syncthreads_or(hot)) break;
        if (tid == 0) anyRot = 0;
        __syncthreads();
        for (int rnd = 0; rnd < m - 1; ++rnd) {
            const int* pr = pairs + rnd * half;
            if (tid < 32) {
              bool rot_ = false;
              if (tid < half) {
                const int pq = pr[tid];
                const int p = pq & 255, q = pq >> 8;
                const float app = a[p * S + p], aqq = a[q * S + q], apq = a[p * S + q];
                float cs = 1.0f, sn = 0.0f;
                // relative threshold a few FP32 ulps above rounding noise, with a floor at
                // floorRel of the largest diagonal entry: the rounding level of the FP64 Gram
                // (1e-15 for a Gram formed normwise, ~1e-20 for a row-graded one), below which
                // entries carry no information; at most 15 sweeps
                if (fabsf(apq) > fmaxf(1e-6f * sqrtf(fabsf(app * aqq)), floorRel)) {
                    const float th = __fdividef(aqq - app, 2.0f * apq);
                    float t;
                    if (fabsf(th) > 1e18f) t = __fdividef(0.5f, th);
                    else t = copysignf(1.0f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
                    cs = rsqrtf(fmaf(t, t, 1.0f));
                    sn = t * cs;
                    if (sn != 0.0f) anyRot = 1;
                }
                cso[tid] = make_float2(cs, sn);
                rot_ = (sn != 0.0f);
              }
              const unsigned any_ = __ballot_sync(0xffffffffu, rot_);
              if (tid == 0) roundRot[rnd] = (any_ != 0u);
            }
            __syncthreads();
            // a round without rotations writes nothing: no apply pass, no second barrier
            // (the next round's rotation pass only reads what this round left unchanged)
            if (!roundRot[rnd]) continue;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (t >= nit) break;
                if (itA[t] >= 0) {
                    // A <- J^T A J on the 2x2 block (pair pi rows, pair pj columns)
                    const int pi = itA[t], pj = itB[t];
                    const float2 ki = cso[pi], kj = cso[pj];
                    if (ki.y == 0.0f && kj.y == 0.0f) continue;
                    const int pqi = pr[pi], pqj = pr[pj];
                    const int p1 = pqi & 255, q1 = pqi >> 8, p2 = pqj & 255, q2 = pqj >> 8;
                    const float ci = ki.x, si = ki.y, cj = kj.x, sj = kj.y;
                    const float b00 = a[p1 * S + p2], b01 = a[p1 * S + q2];
                    const float b10 = a[q1 * S + p2], b11 = a[q1 * S + q2];
                    const float r00 = ci * b00 - si * b10, r01 = ci * b01 - si * b11;   // J_i^T B
                    const float r10 = si * b00 + ci * b10, r11 = si * b01 + ci * b11;
                    float o00 = cj * r00 - sj * r01, o01 = sj * r00 + cj * r01;        // (.) J_j
                    float o10 = cj * r10 - sj * r11, o11 = sj * r10 + cj * r11;
                    if (pi == pj) { o01 = 0.0f; o10 = 0.0f; }                     // annihilated
                    a[p1 * S + p2] = o00; a[p1 * S + q2] = o01;
                    a[q1 * S + p2] = o10; a[q1 * S + q2] = o11;
                } else {
                    // V <- V J on row r, pair pi
                    const int r = -1 - itA[t], pi = itB[t];
                    const float2 k_ = cso[pi];
                    if (k_.y == 0.0f) continue;
                    const int pq = pr[pi], p = pq & 255, q = pq >> 8;
                    const float vp = v[r * S + p], vq = v[r * S + q];
                    v[r * S + p] = k_.x * vp - k_.y * vq;
                    v[r * S + q] = k_.y * vp + k_.x * vq;
                }
            }
            __syncthreads();
        }
        if (!anyRot) break;
        __syncthreads();
    }

    // ---- ascending order of the FP32 eigenvalues (ties by index) -------------------------
    for (int i = tid; i < c; i += blockDim.x) {
        const float di = a[i * S + i];
        int rk = 0;
        for (int j = 0; j < c; ++j) {
            const float dj = a[j * S + j];
            rk += (dj < di) || (dj == di && j < i);
        }
        order[rk] = i;
    }
    __syncthreads();
    // ---- orthonormalisation of W = v[:, order] (columns in ascending order) -------------
    // Cholesky-QR W <- W L^-T with W^T W = L L^T.  W's entries are FP32 numbers, so the Gram
    // is formed from exact products in double-float arithmetic (FP32 pipe) and rounded to
    // FP64; Cholesky and L^-1 run in FP64; the product W L^-T again in double-float with
    // L^-1 split into FP32 pairs.  Orthonormal to ~1e-14 (double-float rounding).
    for (int e_ = tid; e_ < c * c; e_ += blockDim.x) {
        const int i = e_ % c, j = e_ / c;
        if (i < j) continue;
        const int oi = order[i], oj = order[j];
        float2 acc = make_float2(0.0f, 0.0f);
        for (int r = 0; r < c; ++r)
            df_fma(acc, make_float2(v[r * S + oi], 0.0f), make_float2(v[r * S + oj], 0.0f));
        G[i * S + j] = (double)acc.x + (double)acc.y;    // lower triangle of W^T W
    }
    __syncthreads();
    for (int k = 0; k < c; ++k) {
        if (tid == 0) {
            const double g = fmax(G[k * S + k], 1e-300), y = fc_rsqrt(g);
            G[k * S + k] = g * y;
            dinv[k] = y;
        }
        __syncthreads();
        const double ik = dinv[k];
        for (int i = k + 1 + tid; i < c; i += blockDim.x) G[i * S + k] *= ik;
        __syncthreads();
        for (int e_ = tid; e_ < (c - k - 1) * (c - k - 1); e_ += blockDim.x) {
            const int i = k + 1 + e_ % (c - k - 1), j = k + 1 + e_ / (c - k - 1);
            if (j <= i) G[i * S + j] -= G[i * S + k] * G[j * S + k];
        }
        __syncthreads();
    }
    // L^-1 column by column, one warp per column j: x_j = 1 / L_jj,
    // x_i = -(sum_{j <= k < i} L_ik x_k) / L_ii (lane-parallel dot products)
    for (int j = wid; j < c; j += nwarp) {
        if (lane == 0) Li[j * S + j] = dinv[j];
        __syncwarp();
        for (int i = j + 1; i < c; ++i) {
            double s_ = 0.0;
            for (int k = j + lane; k < i; k += 32) s_ = fma(G[i * S + k], Li[k * S + j], s_);
            s_ = warp_sum(s_);
            if (lane == 0) Li[i * S + j] = -s_ * dinv[i];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int e_ = tid; e_ < c * c; e_ += blockDim.x) {
        const int i = e_ % c, j = e_ / c;
        if (j <= i) Lf[i * S + j] = df_split(Li[i * S + j]);
    }
    __syncthreads();
    // G[r][j] = (W L^-T)[r, j] = sum_{k <= j} W[r, k] (L^-1)[j, k]
    for (int e_ = tid; e_ < c * c; e_ += blockDim.x) {
        const int r = e_ % c, j = e_ / c;
        float2 acc = make_float2(0.0f, 0.0f);
        for (int k = 0; k <= j; ++k)
            df_fma(acc, make_float2(v[r * S + order[k]], 0.0f), Lf[j * S + k]);
        G[r * S + j] = (double)acc.x + (double)acc.y;
    }
    __syncthreads();

    // ---- eigenvalues and outputs (descending) --------------------------------------------
    for (int j = tid; j < c; j += blockDim.x) {
        double lam;
        if (rq) {
            lam = 0.0;
            for (int i = 0; i < c; ++i) {
                double t = 0.0;
                for (int k2 = 0; k2 < c; ++k2) t = fma(A64[i * S + k2], G[k2 * S + j], t);
                lam = fma(G[i * S + j], t, lam);
            }
        } else {
            lam = dmax * (double)a[order[j] * S + order[j]];
        }
        evb[c - 1 - j] = lam;
    }
    for (int e_ = tid; e_ < c * c; e_ += blockDim.x) {
        const int r = e_ % c, j = e_ / c;
        Vb[r + (long long)(c - 1 - j) * ldv] = G[r * S + j];
    }
}

size_t gjacobi_smem() {
    const int S = kMaxC + 1;
    return sizeof(double) * 4 * (size_t)kMaxC * S + sizeof(float) * 2 * (size_t)kMaxC * S +
           sizeof(float2) * kMaxC + sizeof(int) * (kMaxC + (size_t)kMaxC * kMaxC / 2);
}

void launch_gjacobi(cudaStream_t st, int batch, const double* A, int lda, long long bsA,
                    const int* dims, int dstride, int cmax, double* ev, long long bsE,
                    double* V, int ldv, long long bsV, bool rq, float floorRel,
                    const double* floorAbs, double floorFrac)
{
    if (batch <= 0) return;
    const bool prof = prof_active(KC_JACOBI);
    ProfMark mark;
    if (prof) prof_begin(st, mark);
    note_launch(); gjacobi_kernel<<<batch, kGjThreads, gjacobi_smem(), st>>>(A, lda, bsA, dims, dstride, cmax, ev, bsE, V, ldv, bsV, rq ? 1 : 0, floorRel, prof ? 1 : 0, floorAbs, floorFrac);
    if (prof) prof_end(st, mark);
}

size_t symeig_smem() {
    const int S = kMaxC + 1;
    return sizeof(double) * (2 * (size_t)kMaxC * S + 7 * kMaxC + kGrid) + sizeof(int) * kGrid;
}

void launch_symeig(cudaStream_t st, int batch, const double* A, int lda, long long bsA,
                   const int* dims, int dstride, int cmax, double* ev, long long bsE,
                   double* V, int ldv, long long bsV)
{
    if (batch <= 0) return;
    const bool prof = prof_active(KC_JACOBI);
    ProfMark mark;
    if (prof) prof_begin(st, mark);
    note_launch(); symeig_kernel<<<batch, kEigThreads, symeig_smem(), st>>>(A, lda, bsA, dims, dstride, cmax, ev, bsE, V, ldv, bsV, prof ? 1 : 0);
    if (prof) prof_end(st, mark);
}

cudaError_t set_symeig_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(symeig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)symeig_smem());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(gjacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gjacobi_smem());
}

}  // namespace fc
