// Shared device helpers of libfc: the FP64 tiled GEMM with operand loaders, reductions,
// and launch-wrapper declarations.  All matrices are column-major.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <algorithm>
#include <atomic>

#define FC_DEV __device__ __forceinline__

namespace fc {

// Count of kernels launched by this library in this process (fc_launch_count).
void note_launch();
// Record a CUDA error's text for fc_last_cuda_error (calling thread) and return FC_ECUDA.
int record_cuda_error(cudaError_t e);

// Kernel-class timing for instrumentation (fc_prof_*): while a class is enabled, each of
// its launches is bracketed by a pair of CUDA events recorded on the launching stream.
enum KernelClass { KC_NONE = 0, KC_JACOBI = 1, KC_TC = 2, KC_F64 = 3 };
struct ProfMark { int slot = -1; };
bool prof_active(int kclass);
void prof_begin(cudaStream_t st, ProfMark& m);
void prof_end(cudaStream_t st, const ProfMark& m);
unsigned long long* prof_work_counter();   // device counter of the class's algorithmic flops

// Launch schedule (fc_schedule in fc.h): the tile and split rules of the contraction launches
// and the policy of fc_solve_batched, set by fc_set_schedule or chosen by fc_autotune.  Each
// field is read on its own at every launch (relaxed loads; fc_set_schedule is not called
// while solves run).
struct SchedState {
    std::atomic<int> gemm_cover{8};     // FP64 GEMM tiles: cover gemm_cover / 8 of the SMs
    std::atomic<int> gemm_split{4};     // split-K until about gemm_split CTAs per SM (0: never)
    std::atomic<int> tc_split{1};       // tensor-core K ranges: 1 fill the waves, 0 fewest
    std::atomic<int> tc_min_log2{22};   // form 3: tensor cores from 2^tc_min_log2 multiply-adds
    std::atomic<int> workers{16};       // fc_solve_batched host threads / worker streams
    std::atomic<int> order{0};          // fc_solve_batched: 0 given order, 1 largest first
};
extern SchedState g_sched;
inline int sched(const std::atomic<int>& f) { return f.load(std::memory_order_relaxed); }

constexpr int kMaxC = 64;       // largest dense eigen / Cholesky problem handled by one CTA
constexpr int kThreads = 256;

// ---------------------------------------------------------------------------------------
// Operand loaders.  op(A) is M x K, op(B) is K x N; a loader returns element (i, k) of the
// operand for batch item b.  Plain matrices are column-major with leading dimension ld and
// batch stride bs (elements).
// ---------------------------------------------------------------------------------------
struct LdN {  // op(X) = X
    const double* p; int ld; long long bs;
    FC_DEV double operator()(int i, int k, int b) const { return p[b * bs + i + (long long)k * ld]; }
};
struct LdT {  // op(X) = X^T
    const double* p; int ld; long long bs;
    FC_DEV double operator()(int i, int k, int b) const { return p[b * bs + k + (long long)i * ld]; }
};
// Orthonormal DST-I matrix F[i,k] = sqrt(2/N) sin(pi (i+1)(k+1)/N) from a table
// tab[m] = sqrt(2/N) sin(pi m / N), m = 0..2N-1 (Section 3.2).
struct LdSine {
    const double* tab; int N2;
    FC_DEV double operator()(int i, int k, int) const {
        // (i+1)(k+1) <= (n+1)^2 <= 2^26 for n <= 8191: 32-bit arithmetic
        const unsigned m = (unsigned)(i + 1) * (unsigned)(k + 1);
        return tab[m % (unsigned)N2];
    }
};
// Khatri-Rao column (k,j) -> e_k . y_j, column index kj = k*S + j, row i (Section 3.2,
// the mode factors of eqn:Lap3DtimesX in the eigenbasis).  Batch b selects the mode.
struct LdKR {
    const double* E; int lde; long long bsE;
    const double* Y; int ldy; long long bsY;
    int S;
    FC_DEV double operator()(int i, int kj, int b) const {
        int k = kj / S, j = kj - k * S;
        return E[b * bsE + i + (long long)k * lde] * Y[b * bsY + i + (long long)j * ldy];
    }
};
// Rows (a,b) of the mode-(1,2) unfolding of a CP tensor's projected factors:
// A[(a + r1*b), K] = w_K C1[a,K] C2[b,K]  (core assembly, eqn:coret with a CP input).
struct LdCore12 {
    const double* C1; const double* C2; const double* w; int ldc; int r1;
    FC_DEV double operator()(int ab, int K, int) const {
        int b = ab / r1, a = ab - b * r1;
        return w[K] * C1[a + (long long)K * ldc] * C2[b + (long long)K * ldc];
    }
};
// A[a, K] = w_K C1[a, K]  (2D core: (C1 diag(w)) C2^T)
struct LdScaledN {
    const double* p; int ld; const double* w;
    FC_DEV double operator()(int i, int k, int) const { return w[k] * p[i + (long long)k * ld]; }
};


// ---- further operand loaders used by the truncation --------------------------------------
struct LdSq {     // w_k^2 * X[i, k]  (w of batch item b at w + b * bsw)
    const double* p; int ld; long long bs; const double* w; long long bsw = 0;
    FC_DEV double operator()(int i, int k, int b) const {
        const double wk = w[b * bsw + k];
        return wk * wk * p[b * bs + i + (long long)k * ld];
    }
};
struct LdSqN {    // X[i, k]^2
    const double* p; int ld; long long bs;
    FC_DEV double operator()(int i, int k, int b) const {
        const double v = p[b * bs + i + (long long)k * ld];
        return v * v;
    }
};
struct LdSqT {    // X[k, i]^2  (op = transpose)
    const double* p; int ld; long long bs;
    FC_DEV double operator()(int i, int k, int b) const {
        const double v = p[b * bs + k + (long long)i * ld];
        return v * v;
    }
};
struct LdAbsN {   // |w_k| * X[i, k]
    const double* p; int ld; long long bs; const double* w;
    FC_DEV double operator()(int i, int k, int b) const { return fabs(w[k]) * p[b * bs + i + (long long)k * ld]; }
};
// A[(a + r0 b), k] = w_k C0[a, k] C1[b, k], r0 read from device memory
struct LdCore {
    const double* C0; const double* C1; const double* w; int ldc; const int* r0p;
    FC_DEV double operator()(int ab, int k, int) const {
        int r0 = *r0p; int b = ab / r0, a = ab - b * r0;
        return w[k] * C0[a + (long long)k * ldc] * C1[b + (long long)k * ldc];
    }
};
// A[(a + r0 b), k] = C0[a, k] C1w[b, k] with C1w = C1 diag(w) formed beforehand
struct LdCoreW {
    const double* C0; const double* C1w; int ldc; const int* r0p;
    FC_DEV double operator()(int ab, int k, int) const {
        int r0 = *r0p; int b = ab / r0, a = ab - b * r0;
        return C0[a + (long long)k * ldc] * C1w[b + (long long)k * ldc];
    }
};
// columns (k*S + b) of a column-major matrix, batch item b (the input column j of a
// Khatri-Rao product): element (i, k) of batch b = p[i + (k*S + b)*ld]
struct LdColsJ {
    const double* p; int ld; int S;
    FC_DEV double operator()(int i, int k, int b) const { return p[i + ((long long)k * S + b) * ld]; }
};
struct LdOnes { FC_DEV double operator()(int, int, int) const { return 1.0; } };
struct LdPart {   // sum of S partial results (split-K reduction), element i
    const double* p; int S; long long stride;
    FC_DEV double operator()(int i, int, int) const {
        double s = 0; for (int t = 0; t < S; ++t) s += p[t * stride + i]; return s;
    }
};
// slice s of a compact (r0 x r1) column: element (a, b) = S[s*ld + a + r0*b]
struct LdSlT {    // op = slice^T : (b, a)
    const double* S; long long ld; const int* r0p;
    FC_DEV double operator()(int b, int a, int s) const { return S[s * ld + a + (long long)(*r0p) * b]; }
};
struct LdSl {     // op = slice : (a, b)
    const double* S; long long ld; const int* r0p;
    FC_DEV double operator()(int a, int b, int s) const { return S[s * ld + a + (long long)(*r0p) * b]; }
};

// ---------------------------------------------------------------------------------------
// C[b] = alpha * op(A)[b] * op(B)[b] + beta * C[b]   (M x N, inner K), FP64.
// Sizes can come from device memory (dM/dN/dK non-null) so that one launch covers the
// largest case and blocks outside the live size return.  Split-K: gridDim.z = batch*splits;
// split s handles the K range [s*kchunk, (s+1)*kchunk) and adds alpha * its partial product
// to C with FP64 atomics (C pre-scaled by beta in a separate launch).  GB300 issues few
// FP64 FMAs per SM per clock, so a GEMM whose output tiles cannot fill the 152 SMs is
// split along K until they do.  Register tile 4x4 per thread, 64x64 block tile, BK = 16.
// ---------------------------------------------------------------------------------------
constexpr int GBK = 16;
constexpr int kNumSMs = 152;

// Tile T x T (T = 64, 32 or 16) with 256 threads, each owning a (T/16) x (T/16) register block.
template <int T, class LA, class LB>
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int K, const int* dM, const int* dN, const int* dK,
            LA A, LB B, double alpha, double beta, double* C, int ldc, long long bsC,
            int batch, int splits, int kchunk, unsigned long long* work)
{
    constexpr int R = T / 16;                  // register block per thread
    constexpr int LOADS = T * GBK / 256;       // tile elements loaded per thread
    __shared__ double As[GBK][T + 1];
    __shared__ double Bs[GBK][T + 1];
    if (dM) M = min(M, *dM);
    if (dN) N = min(N, *dN);
    if (dK) K = min(K, *dK);
    const int zb = blockIdx.z / splits, zs = blockIdx.z - zb * splits;
    const int m0 = blockIdx.x * T, n0 = blockIdx.y * T;
    if (m0 >= M || n0 >= N || zb >= batch) return;
    int kbeg = zs * kchunk, kend = min(K, kbeg + kchunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
        for (int t = 0; t < LOADS; ++t) {          // T x 16 tile of op(A)
            int e = threadIdx.x + t * 256;
            int ii = e % T, kk = e / T;
            int gi = m0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < M && gk < kend) ? A(gi, gk, zb) : 0.0;
        }
#pragma unroll
        for (int t = 0; t < LOADS; ++t) {          // 16 x T tile of op(B)
            int e = threadIdx.x + t * 256;
            int kk = e & 15, jj = e >> 4;
            int gj = n0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gj < N && gk < kend) ? B(gk, gj, zb) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            double a[R], b[R];
#pragma unroll
            for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < R; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double* Cb = C + zb * bsC;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int gi = m0 + ty + 16 * i;
        if (gi >= M) continue;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            int gj = n0 + tx + 16 * j;
            if (gj >= N) continue;
            double* c = Cb + gi + (long long)gj * ldc;
            if (splits > 1) atomicAdd(c, alpha * acc[i][j]);
            else *c = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*c);
        }
    }
    // instrumentation: 2 flop per multiply-add of the live tile and K range
    if (work && threadIdx.x == 0 && kend > kbeg)
        atomicAdd(work, 2ull * (unsigned long long)min(T, M - m0) * (unsigned long long)min(T, N - n0) *
                            (unsigned long long)(kend - kbeg));
}

// ---------------------------------------------------------------------------------------
// Double-float variant of gemm_kernel: operands are split on load into FP32 pairs
// (hi = fl32(v), lo = fl32(v - hi)) and every multiply-add runs on the FP32 pipe as an exact
// product (fmaf error term) plus cross terms and a two-sum accumulation, ~48 mantissa bits
// (relative error ~1e-14).  GB300 issues 64x more FP32 than FP64 FMAs per clock, so this
// runs ~4x faster than the FP64 kernel on contraction-bound GEMMs.  Values must stay within
// the FP32 exponent range (|v| < 2^126; parts below 2^-126 flush to zero, relative to the
// operands' scale that is far below the FP64 rounding of the result).
// ---------------------------------------------------------------------------------------
FC_DEV void df_fma(float2& acc, float2 a, float2 b) {
    const float p = a.x * b.x;
    float pe = fmaf(a.x, b.x, -p);
    pe = fmaf(a.x, b.y, pe);
    pe = fmaf(a.y, b.x, pe);
    const float s = acc.x + p;
    const float bb = s - acc.x;
    const float err = (acc.x - (s - bb)) + (p - bb);
    const float lo = acc.y + pe + err;
    const float hi = s + lo;
    acc.y = lo - (hi - s);
    acc.x = hi;
}
FC_DEV float2 df_split(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

template <int T, class LA, class LB>
__global__ void __launch_bounds__(256)
gemm_df_kernel(int M, int N, int K, const int* dM, const int* dN, const int* dK,
               LA A, LB B, double alpha, double beta, double* C, int ldc, long long bsC,
               int batch, int splits, int kchunk)
{
    constexpr int R = T / 16;
    constexpr int LOADS = T * GBK / 256;
    __shared__ float2 As[GBK][T + 1];
    __shared__ float2 Bs[GBK][T + 1];
    if (dM) M = min(M, *dM);
    if (dN) N = min(N, *dN);
    if (dK) K = min(K, *dK);
    const int zb = blockIdx.z / splits, zs = blockIdx.z - zb * splits;
    const int m0 = blockIdx.x * T, n0 = blockIdx.y * T;
    if (m0 >= M || n0 >= N || zb >= batch) return;
    int kbeg = zs * kchunk, kend = min(K, kbeg + kchunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float2 acc[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = make_float2(0.0f, 0.0f);
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
        for (int t = 0; t < LOADS; ++t) {
            int e = threadIdx.x + t * 256;
            int ii = e % T, kk = e / T;
            int gi = m0 + ii, gk = k0 + kk;
            As[kk][ii] = df_split((gi < M && gk < kend) ? A(gi, gk, zb) : 0.0);
        }
#pragma unroll
        for (int t = 0; t < LOADS; ++t) {
            int e = threadIdx.x + t * 256;
            int kk = e & 15, jj = e >> 4;
            int gj = n0 + jj, gk = k0 + kk;
            Bs[kk][jj] = df_split((gj < N && gk < kend) ? B(gk, gj, zb) : 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float2 a[R], b[R];
#pragma unroll
            for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < R; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < R; ++j) df_fma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    double* Cb = C + zb * bsC;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int gi = m0 + ty + 16 * i;
        if (gi >= M) continue;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            int gj = n0 + tx + 16 * j;
            if (gj >= N) continue;
            const double v = (double)acc[i][j].x + (double)acc[i][j].y;
            double* c = Cb + gi + (long long)gj * ldc;
            if (splits > 1) atomicAdd(c, alpha * v);
            else *c = (beta == 0.0) ? alpha * v : alpha * v + beta * (*c);
        }
    }
}

// C[b][i, j] *= beta (beta == 0: set to 0) over the live M x N (split-K pre-pass).
__global__ void gemm_prescale_kernel(int M, int N, const int* dM, const int* dN, double beta,
                                     double* C, int ldc, long long bsC);

}  // namespace fc
#include "fc_tc.cuh"
namespace fc {

// Launch (rules of the schedule, defaults in brackets): the largest tile (64, 32, 16) whose
// grid still has gemm_cover / 8 [1] tiles per SM, then, for grids below two tiles per SM,
// split-K until about gemm_split [4] CTAs per SM (GB300 runs few FP64 FMAs per SM per clock,
// so for one solve alone the SM count decides the rate; with many solves in flight larger
// tiles and fewer splits waste less).
// Precision of a contraction: FP64, double-float on the FP32 pipe (gemm_df_kernel), or
// FP64-accurate digit products on the BF16 tensor cores (gemm_tc_kernel) for contractions
// of at least 2^tc_min_log2 [2^22] multiply-adds (smaller ones stay on the FP64 kernel,
// whose latency is lower).
enum GemmPrec { GP_F64 = 0, GP_DF32 = 1, GP_TC64 = 2 };

template <class LA, class LB>
inline void gemm_p(int prec, cudaStream_t st, int M, int N, int K, LA A, LB B, double alpha,
                   double beta, double* C, int ldc, long long bsC = 0, int batch = 1,
                   const int* dM = nullptr, const int* dN = nullptr, const int* dK = nullptr)
{
    if (M <= 0 || N <= 0 || batch <= 0) return;
    if (prec == GP_TC64 && (long long)M * N * K * batch >= (1ll << sched(g_sched.tc_min_log2)) &&
        gemm_tc(st, M, N, K, A, B, alpha, beta, C, ldc, bsC, batch, dM, dN, dK))
        return;
    auto tiles_of = [&](int T) {
        return (long long)((M + T - 1) / T) * ((N + T - 1) / T) * batch;
    };
    // FP64: the largest tile that still covers the SMs.  Double-float: operand splitting
    // costs FP64 work per loaded element, so keep 64-wide tiles down to a quarter of the SMs.
    int T = 64;
    const long long cover = sched(g_sched.gemm_cover);
    const long long need = std::max(1ll, kNumSMs * cover / ((prec == GP_DF32) ? 32 : 8));
    if (tiles_of(64) < need) T = (tiles_of(32) < need) ? 16 : 32;
    const long long tiles = tiles_of(T);
    int splits = 1;
    const long long spl = sched(g_sched.gemm_split);
    if (spl > 0 && tiles < 2 * kNumSMs && K >= 128) {
        long long want = (spl * kNumSMs + tiles - 1) / tiles;
        long long most = (K + 63) / 64;            // at least 64 of K per split
        splits = (int)std::min<long long>(std::min(want, most), 64);
    }
    int kchunk = K;
    if (splits > 1) {
        kchunk = (K + splits - 1) / splits;
        kchunk = (kchunk + GBK - 1) / GBK * GBK;
        splits = (K + kchunk - 1) / kchunk;
    }
    if (splits > 1 && beta != 1.0) {
        dim3 g((M + 255) / 256, N, batch);
        note_launch(); gemm_prescale_kernel<<<g, 256, 0, st>>>(M, N, dM, dN, beta, C, ldc, bsC);
    }
    dim3 grid((M + T - 1) / T, (N + T - 1) / T, batch * splits);
    note_launch();
    const bool prof = prec != GP_DF32 && prof_active(KC_F64);
    unsigned long long* work = prof ? prof_work_counter() : nullptr;
    ProfMark mark;
    if (prof) prof_begin(st, mark);
    if (prec == GP_DF32) {
        if (T == 64)
            gemm_df_kernel<64, LA, LB><<<grid, 256, 0, st>>>(M, N, K, dM, dN, dK, A, B, alpha, beta,
                                                             C, ldc, bsC, batch, splits, kchunk);
        else if (T == 32)
            gemm_df_kernel<32, LA, LB><<<grid, 256, 0, st>>>(M, N, K, dM, dN, dK, A, B, alpha, beta,
                                                             C, ldc, bsC, batch, splits, kchunk);
        else
            gemm_df_kernel<16, LA, LB><<<grid, 256, 0, st>>>(M, N, K, dM, dN, dK, A, B, alpha, beta,
                                                             C, ldc, bsC, batch, splits, kchunk);
        return;
    }
    if (T == 64)
        gemm_kernel<64, LA, LB><<<grid, 256, 0, st>>>(M, N, K, dM, dN, dK, A, B, alpha, beta, C,
                                                      ldc, bsC, batch, splits, kchunk, work);
    else if (T == 32)
        gemm_kernel<32, LA, LB><<<grid, 256, 0, st>>>(M, N, K, dM, dN, dK, A, B, alpha, beta, C,
                                                      ldc, bsC, batch, splits, kchunk, work);
    else
        gemm_kernel<16, LA, LB><<<grid, 256, 0, st>>>(M, N, K, dM, dN, dK, A, B, alpha, beta, C,
                                                      ldc, bsC, batch, splits, kchunk, work);
    if (prof) prof_end(st, mark);
}

template <class LA, class LB>
inline void gemm(cudaStream_t st, int M, int N, int K, LA A, LB B, double alpha, double beta,
                 double* C, int ldc, long long bsC = 0, int batch = 1,
                 const int* dM = nullptr, const int* dN = nullptr, const int* dK = nullptr)
{
    gemm_p(GP_F64, st, M, N, K, A, B, alpha, beta, C, ldc, bsC, batch, dM, dN, dK);
}

// ---------------------------------------------------------------------------------------
// Block reductions
// ---------------------------------------------------------------------------------------
FC_DEV double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
FC_DEV double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// 1/sqrt(x) for a positive FP64 x: the argument scaled by an even power of two into [1, 4),
// an FP32 reciprocal-square-root estimate, two Newton steps y <- y (3 - m y^2) / 2 in FP64
// (relative error at the FP64 rounding level), rescaled.  A dependent FP64 square root and
// divide take ~600 and ~360 cycles on GB300; this chain takes ~6 dependent FMAs.
FC_DEV double fc_rsqrt(double x) {
    if (!(x >= 2.3e-308) || !(x <= 1.7e308)) return 1.0 / sqrt(x);   // subnormal, 0, Inf, NaN
    const long long bits = __double_as_longlong(x);
    const int e2 = ((int)((bits >> 52) & 0x7FF) - 1023) >> 1;           // floor(ex / 2)
    const double m = __longlong_as_double(bits - ((long long)(2 * e2) << 52));   // [1, 4)
    double y = (double)rsqrtf((float)m);
    const double hm = 0.5 * m;
    y = y * fma(-hm, y * y, 1.5);
    y = y * fma(-hm, y * y, 1.5);
    return __longlong_as_double(__double_as_longlong(y) - ((long long)e2 << 52));
}

// Sum over the block; every thread gets the result.  `red` needs blockDim/32 doubles.
FC_DEV double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0) t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}

}  // namespace fc
