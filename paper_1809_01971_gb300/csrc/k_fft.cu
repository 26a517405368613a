// Full-format eigenbasis solve by fast sine transforms (Section 3.2, eqn:DiagFLaplace3D /
// eqn:DiagFLaplace2D):  u = (F x .. x F) diag(1/g(rho)) (F x .. x F) b  on the n^d grid,
// F the orthonormal DST-I, F[j,k] = sqrt(2/N) sin(pi j k / N), N = n + 1, rho_i = sum_l lambda_{i_l}.
//
// DST-I through a complex FFT of length N (N a power of two).  For one line x_1..x_{N-1}, the odd
// extension z of length 2N (z_0 = z_N = 0, z_j = x_j, z_{2N-j} = -x_j) has the DFT
// Z_k = -2i sum_j x_j sin(pi j k / N), so DST_k = -Im(Z_k) / 2.  The 2N real values are packed as
// w_j = z_{2j} + i z_{2j+1} (j < N); with W = FFT_N(w),
//     Z_k = (W_k + conj W_{N-k}) / 2  -  (i/2) e^{-i pi k / N} (W_k - conj W_{N-k}),
// the split of one complex FFT into the transforms of the even and odd samples.  The FFT is an
// iterative radix-2 decimation in time on shared memory (bit-reversed load), twiddles
// e^{-2 pi i m / N} = tw[2m] from the table tw[k] = e^{-i pi k / N}, k < N, built on the host.
//
// One CTA transforms LPB lines of one axis (64 KB of complex arrays, 128 KB in the scaling pass):
// the values are loaded straight into the packed bit-reversed arrays and the DST values are
// stored straight from the transformed ones.  Lines of axis 0 are contiguous; the LPB lines of
// axes 1 and 2 are neighbours in the contiguous index i_1, so every element position of the
// LPB lines is one contiguous run in HBM.  A solve is 2d - 1 passes over the array: forward
// transforms of axes 0 .. d-2, then on the last axis the forward transform, the division by
// g(rho) and the inverse transform (F = F^-1) in shared memory, then the inverse transforms of
// axes d-2 .. 0.  Each pass reads and writes the array once: (2d - 1) * 2 * 8 n^d bytes.
#include "fc_common.cuh"
#include "fc_kernels.h"

namespace fc {

namespace {

constexpr int kFftThreads = 256;

struct LineMap {   // element j of line L of the given axis in an n^d column-major array
    int d, axis, n;
    FC_DEV long long base(long long L) const {
        const long long nn = (long long)n * n;
        if (axis == 0) return L * n;
        if (axis == 1) return (d == 2) ? L : (L % n) + (L / n) * nn;
        return (L % n) + (L / n) * (long long)n;             // axis 2 (d = 3)
    }
    FC_DEV long long stride() const {
        return axis == 0 ? 1 : (axis == 1 ? (long long)n : (long long)n * n);
    }
};

FC_DEV unsigned bitrev(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

// Scatter value v = x_m (1 <= m <= N-1) of a line into its packed, bit-reversed complex array:
// x_m is z_m and -x_m is z_{2N-m} of the odd extension, and z_q is component q & 1 of
// w_{q >> 1}.  The two entries z_0 = z_N = 0 (real parts of w_0 and w_{N/2}) are set apart.
FC_DEV void scatter_x(double* sd, int m, double v, int N, int logN) {
    sd[2 * bitrev((unsigned)(m >> 1), logN) + (m & 1)] = v;
    const int q = 2 * N - m;
    sd[2 * bitrev((unsigned)(q >> 1), logN) + (q & 1)] = -v;
}

// Radix-2 decimation-in-time FFT of every line's bit-reversed array s_l (length N, lines
// l < lpb at stride N); the tpl threads of line l run its butterflies, two per iteration with
// both loads ahead of the arithmetic.  Ends with a CTA barrier.
FC_DEV void fft_lines(double2* sbase, int N, int logN, const double2* tw, int l, int t, int tpl) {
    double2* s = sbase + (size_t)l * N;
    const int nb = N / 2;
    for (int st = 1; st <= logN; ++st) {
        const int half = 1 << (st - 1);
        const int sh = logN - st + 1;               // twiddle of position pos: tw[pos << sh]
        for (int b = t; b < nb; b += 2 * tpl) {
            const int b2 = b + tpl;
            const int pos1 = b & (half - 1), i1 = ((b >> (st - 1)) << st) + pos1, j1 = i1 + half;
            const double2 w1 = tw[pos1 << sh];
            const double2 u1 = s[i1], v1 = s[j1];
            double2 w2 = make_double2(0.0, 0.0), u2 = w2, v2 = w2;
            int i2 = 0, j2 = 0;
            const bool two = b2 < nb;
            if (two) {
                const int pos2 = b2 & (half - 1);
                i2 = ((b2 >> (st - 1)) << st) + pos2;
                j2 = i2 + half;
                w2 = tw[pos2 << sh];
                u2 = s[i2];
                v2 = s[j2];
            }
            const double a1 = v1.x * w1.x - v1.y * w1.y, c1 = v1.x * w1.y + v1.y * w1.x;
            s[i1] = make_double2(u1.x + a1, u1.y + c1);
            s[j1] = make_double2(u1.x - a1, u1.y - c1);
            if (two) {
                const double a2 = v2.x * w2.x - v2.y * w2.y, c2 = v2.x * w2.y + v2.y * w2.x;
                s[i2] = make_double2(u2.x + a2, u2.y + c2);
                s[j2] = make_double2(u2.x - a2, u2.y - c2);
            }
        }
        __syncthreads();
    }
}

// Orthonormal DST-I value k (1 <= k <= N-1) of a line from its transformed array s:
// -Im(Z_k) / 2 * sqrt(2/N) with Z_k = E_k - (i/2) e^{-i pi k/N} D_k,
// E_k = (W_k + conj W_{N-k}) / 2, D_k = W_k - conj W_{N-k}.
FC_DEV double dst_value(const double2* s, int k, int N, const double2* tw, double scale) {
    const double2 a = s[k], c = s[N - k];
    const double ey = 0.5 * (a.y - c.y);
    const double dx = a.x - c.x, dy = a.y + c.y;
    const double2 e = tw[k];
    const double px = e.x * dx - e.y * dy;
    return scale * (ey - 0.5 * px);
}

template <bool SCALE>
__global__ void __launch_bounds__(kFftThreads)
dst_pass_kernel(const double* in, double* out, int d, int axis, int n, int logN, long long nlines,
                int lpb, const double2* tw, const double* lam, int lstride, double ga, double sn,
                double gb, double sp, double gc)
{
    extern __shared__ double2 fft_smem[];
    const int N = n + 1;
    double2* s1 = fft_smem;                                   // lpb x N complex
    double2* s2 = fft_smem + (size_t)lpb * N;                 // second transform (SCALE)
    const LineMap map{d, axis, n};
    const long long L0 = (long long)blockIdx.x * lpb;
    const int nl = (int)min((long long)lpb, nlines - L0);
    const long long stride = map.stride();
    const double scale = -0.5 * sqrt(2.0 / (double)N);
    // zero the arrays of lines beyond nl and the two fixed zeros of every line
    for (int e = threadIdx.x; e < lpb; e += blockDim.x) {
        double* sd = reinterpret_cast<double*>(s1 + (size_t)e * N);
        sd[0] = 0.0;                                           // z_0: real part of w_0
        sd[2 * bitrev((unsigned)(N >> 1), logN)] = 0.0;        // z_N: real part of w_{N/2}
    }
    for (int e = nl * N + threadIdx.x; e < lpb * N; e += blockDim.x)
        s1[e] = make_double2(0.0, 0.0);
    // load straight into the packed arrays: axis 0 lines are contiguous (element fastest);
    // other axes: the lpb neighbouring lines fastest (contiguous runs in HBM)
    for (int e = threadIdx.x; e < nl * n; e += blockDim.x) {
        int l, j;
        if (axis == 0) { l = e / n; j = e - l * n; }
        else { j = e / nl; l = e - j * nl; }
        scatter_x(reinterpret_cast<double*>(s1 + (size_t)l * N), j + 1,
                  in[map.base(L0 + l) + j * stride], N, logN);
    }
    __syncthreads();
    const int tpl = blockDim.x / lpb;
    const int l = threadIdx.x / tpl, t = threadIdx.x - l * tpl;
    fft_lines(s1, N, logN, tw, l, t, tpl);
    double2* sres = s1;
    if (SCALE) {
        // DST values divided by g(rho), rho = the line's fixed eigenvalues + lam of position k,
        // scattered as the input of the inverse transform (F = F^-1)
        for (int e = threadIdx.x; e < lpb; e += blockDim.x) {
            double* sd = reinterpret_cast<double*>(s2 + (size_t)e * N);
            sd[0] = 0.0;
            sd[2 * bitrev((unsigned)(N >> 1), logN)] = 0.0;
        }
        const double* lk = lam + (size_t)(d - 1) * lstride;
        for (int e = threadIdx.x; e < lpb * n; e += blockDim.x) {
            const int li = e / n, k = e - li * n + 1;
            const long long L = L0 + li;
            double v = 0.0;
            if (li < nl) {
                const double rfix = (d == 3) ? lam[L % n] + lam[lstride + L / n] : lam[L];
                const double lr = log(rfix + lk[k - 1]);
                double g = gc;
                if (sn == sp) {                      // a rho^-s + b rho^s: one exponential
                    const double x = exp(sp * lr);
                    g += ga / x + gb * x;
                } else {
                    if (ga != 0.0) g += ga * exp(-sn * lr);
                    if (gb != 0.0) g += gb * exp(sp * lr);
                }
                v = dst_value(s1 + (size_t)li * N, k, N, tw, scale) / g;
            }
            scatter_x(reinterpret_cast<double*>(s2 + (size_t)li * N), k, v, N, logN);
        }
        __syncthreads();
        fft_lines(s2, N, logN, tw, l, t, tpl);
        sres = s2;
    }
    for (int e = threadIdx.x; e < nl * n; e += blockDim.x) {
        int li, j;
        if (axis == 0) { li = e / n; j = e - li * n; }
        else { j = e / nl; li = e - j * nl; }
        out[map.base(L0 + li) + j * stride] = dst_value(sres + (size_t)li * N, j + 1, N, tw, scale);
    }
}

}  // namespace

// Lines per CTA: 64 KB of complex arrays per transform (at least 8 threads per line).
int fft_lines_per_block(int N) { return std::max(1, std::min(32, 4096 / N)); }

// Dynamic shared memory of a pass: one complex array per line, two for the scaling pass.
size_t fft_smem_bytes(int N, bool scale) {
    return (size_t)(scale ? 2 : 1) * fft_lines_per_block(N) * N * sizeof(double2);
}

cudaError_t set_fft_attributes(int N) {
    const int bytes = (int)fft_smem_bytes(N, true);
    cudaError_t e = cudaFuncSetAttribute(dst_pass_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(dst_pass_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

void launch_dst_pass(cudaStream_t st, const double* in, double* out, int d, int axis, int n,
                     const double2* tw, bool scale, const double* lam, int lstride, double ga,
                     double sn, double gb, double sp, double gc)
{
    const int N = n + 1;
    int logN = 0;
    while ((1 << logN) < N) ++logN;
    const long long nlines = (d == 3) ? (long long)n * n : (long long)n;
    const int lpb = fft_lines_per_block(N);
    const long long blocks = (nlines + lpb - 1) / lpb;
    const size_t smem = fft_smem_bytes(N, scale);
    note_launch();
    if (scale)
        dst_pass_kernel<true><<<(unsigned)blocks, kFftThreads, smem, st>>>(
            in, out, d, axis, n, logN, nlines, lpb, tw, lam, lstride, ga, sn, gb, sp, gc);
    else
        dst_pass_kernel<false><<<(unsigned)blocks, kFftThreads, smem, st>>>(
            in, out, d, axis, n, logN, nlines, lpb, tw, lam, lstride, ga, sn, gb, sp, gc);
}

}  // namespace fc
