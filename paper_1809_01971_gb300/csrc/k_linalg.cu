// Small dense FP64 linear algebra on one CTA (or warp) per problem (sizes <= kMaxC = 64):
//   * pivoted Cholesky orthonormaliser (range of a sketch, Gram-Schmidt by Cholesky),
//   * rank selection by the Frobenius tail rule and canonical-term selection.
#include "fc_common.cuh"
#include "fc_kernels.h"
#include <math.h>

namespace fc {

// ---------------------------------------------------------------------------------------
// Pivoted-Cholesky orthonormaliser.  Item b: Gram M = Y^T Y (c x c, ld ldm) of a sketch Y.
// Diagonal pivoting stops when the largest remaining diagonal is <= relTol * max diag(M);
// with rank r and pivot order piv, Y P[:, :r] = Q R11, and T[:, :r] = P[:, :r] R11^{-1}
// (T zero elsewhere) gives Q = Y T with orthonormal first r columns.  rank[b*rstride] = r.
// One warp per matrix: the factorisation is a chain of c dependent pivot steps, so warp
// shuffles (pivot arg-max) and __syncwarp replace block barriers; each lane owns rows
// (and later columns of L^-1) lane and lane + 32.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(32)
pchol_kernel(const double* __restrict__ M, int ldm, long long bsM, const int* dims, int dstride,
             int cmax, double relTol, double* __restrict__ T, int ldt, long long bsT,
             int* rank, int rstride)
{
    extern __shared__ double sm[];
    constexpr int SS = kMaxC + 1;
    double* L = sm;                    // L[i*SS + k], i in pivot-position order
    double* Mi = L + kMaxC * SS;       // copy of M
    double* Li = Mi + kMaxC * SS;      // L11^{-1}
    __shared__ double dg[kMaxC];
    __shared__ double invd[kMaxC];     // 1 / L[k][k] (one reciprocal per pivot)
    __shared__ int perm[kMaxC];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x;
    const int b = blockIdx.x;
    int c = cmax;
    if (dims) c = min(dims[b * dstride], cmax);
    if (c < 0) c = 0;
    const double* Mb = M + b * bsM;
    for (int e = lane; e < c * c; e += 32) {
        const int i = e % c, j = e / c;
        Mi[i * SS + j] = Mb[i + (long long)j * ldm];
    }
    for (int i = lane; i < kMaxC; i += 32) perm[i] = i;
    __syncwarp();
    double mx = 0.0;
    for (int i = lane; i < c; i += 32) { dg[i] = Mi[i * SS + i]; mx = fmax(mx, dg[i]); }
    const double dmax0 = warp_max(mx);
    __syncwarp();
    int rk = c;
    for (int k = 0; k < c; ++k) {
        // pivot: largest remaining diagonal among positions k..c-1 (ties: smallest position)
        double best = -1.0;
        int bp = c;
        for (int p = k + lane; p < c; p += 32) {
            const double v = dg[perm[p]];
            if (v > best || (v == best && p < bp)) { best = v; bp = p; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(full, best, o);
            const int op = __shfl_xor_sync(full, bp, o);
            if (ob > best || (ob == best && op < bp)) { best = ob; bp = op; }
        }
        if (!(best > relTol * dmax0) || !(best > 0.0)) { rk = k; break; }   // uniform
        if (bp != k) {
            // rows of L are stored by pivot position: move the computed part with the pivot
            if (lane == 0) { const int t = perm[k]; perm[k] = perm[bp]; perm[bp] = t; }
            for (int j = lane; j < k; j += 32) {
                const double x = L[k * SS + j]; L[k * SS + j] = L[bp * SS + j]; L[bp * SS + j] = x;
            }
            __syncwarp();
        }
        const double ik = fc_rsqrt(best);
        const double lkk = best * ik;
        if (lane == 0) { L[k * SS + k] = lkk; invd[k] = ik; }
        const int pk = perm[k];
        for (int i = k + 1 + lane; i < c; i += 32) {
            // four independent accumulators: a dependent FP64 FMA costs 64 cycles on GB300
            double s0 = Mi[perm[i] * SS + pk], s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int j = 0;
            for (; j + 4 <= k; j += 4) {
                s0 = fma(-L[i * SS + j], L[k * SS + j], s0);
                s1 = fma(-L[i * SS + j + 1], L[k * SS + j + 1], s1);
                s2 = fma(-L[i * SS + j + 2], L[k * SS + j + 2], s2);
                s3 = fma(-L[i * SS + j + 3], L[k * SS + j + 3], s3);
            }
            for (; j < k; ++j) s0 = fma(-L[i * SS + j], L[k * SS + j], s0);
            s0 = (s0 + s1) + (s2 + s3);
            const double l = s0 * ik;
            L[i * SS + k] = l;
            dg[perm[i]] -= l * l;
        }
        __syncwarp();
    }
    const int r = rk;
    // L11^{-1} (lower triangular): column j by lane j (and j + 32), forward substitution
    for (int j = lane; j < r; j += 32) {
        for (int i = 0; i < j; ++i) Li[i * SS + j] = 0.0;
        Li[j * SS + j] = invd[j];
        for (int i = j + 1; i < r; ++i) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int t = j;
            for (; t + 4 <= i; t += 4) {
                s0 = fma(-L[i * SS + t], Li[t * SS + j], s0);
                s1 = fma(-L[i * SS + t + 1], Li[(t + 1) * SS + j], s1);
                s2 = fma(-L[i * SS + t + 2], Li[(t + 2) * SS + j], s2);
                s3 = fma(-L[i * SS + t + 3], Li[(t + 3) * SS + j], s3);
            }
            for (; t < i; ++t) s0 = fma(-L[i * SS + t], Li[t * SS + j], s0);
            s0 = (s0 + s1) + (s2 + s3);
            Li[i * SS + j] = s0 * invd[i];
        }
    }
    __syncwarp();
    // R11^{-1} = (L11^T)^{-1} = (L11^{-1})^T ; T[perm[j], i] = Rinv[j, i] = Linv[i, j]
    double* Tb = T + b * bsT;
    for (int e = lane; e < cmax * cmax; e += 32) Tb[(e % cmax) + (long long)(e / cmax) * ldt] = 0.0;
    __syncwarp();
    for (int e = lane; e < r * r; e += 32) {
        const int j = e % r, i = e / r;
        if (j <= i) Tb[perm[j] + (long long)i * ldt] = Li[i * SS + j];
    }
    if (lane == 0) rank[b * rstride] = r;
}

size_t pchol_smem() { return sizeof(double) * 3 * kMaxC * (kMaxC + 1); }

cudaError_t set_linalg_attributes()
{
    return cudaFuncSetAttribute(pchol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pchol_smem());
}

void launch_pchol(cudaStream_t st, int batch, const double* M, int ldm, long long bsM,
                  const int* dims, int dstride, int cmax, double relTol, double* T, int ldt,
                  long long bsT, int* rank, int rstride)
{
    if (batch <= 0) return;
    const size_t sm = pchol_smem();
    note_launch(); pchol_kernel<<<batch, 32, sm, st>>>(M, ldm, bsM, dims, dstride, cmax, relTol, T, ldt, bsT,
                                         rank, rstride);
}

// ---------------------------------------------------------------------------------------
// Tucker-rank choice (stage 1).  rho[i] (i < live) is the energy of the weighted side matrix
// W_l along basis direction i (directions ordered by decreasing Ritz value), computed from
// the projection itself; missed[l] the energy outside the basis.  Projecting onto the first
// r directions loses exactly tail(r) = sum_{i >= r} rho[i] + missed, so r = the smallest
// r >= 1 with tail(r) <= thr^2, clamped to min(cap, live).
// ---------------------------------------------------------------------------------------
__global__ void select_tucker_kernel(int d, const double* rho, int ldrho, const double* missed,
                                     const double* wn2, double epsfac2, int cap, int* r_out,
                                     double* tail2_out, const int* live)
{
    int l = threadIdx.x;
    if (l >= d) return;
    const double thr2 = epsfac2 * (*wn2);
    const double* rh = rho + (long long)l * ldrho;
    const int nl = live[l];
    const int lim = max(1, min(cap, nl));
    double tail = fmax(missed[l], 0.0);
    for (int i = nl - 1; i >= lim; --i) tail += fmax(rh[i], 0.0);   // always dropped
    int r = lim;
    while (r > 1 && tail + fmax(rh[r - 1], 0.0) <= thr2) { tail += fmax(rh[r - 1], 0.0); --r; }
    r_out[l] = r;
    tail2_out[l] = tail;
}

void launch_select_tucker(cudaStream_t st, int d, const double* rho, int ldrho,
                          const double* missed, const double* wn2, double epsfac2, int cap,
                          int* r_out, double* tail2_out, const int* live)
{
    note_launch(); select_tucker_kernel<<<1, 32, 0, st>>>(d, rho, ldrho, missed, wn2, epsfac2, cap, r_out,
                                                          tail2_out, live);
}

// ---------------------------------------------------------------------------------------
// Canonical-term selection (stage 2).  Candidate terms (slice s, index i) with energy
// mu[s*ldmu + i] (descending within a slice), s < nslice (device count), i < nper (device
// count).  Sort all energies descending, drop the smallest while their total energy stays
// <= thr2frac * core_energy, keep at least one term if any is positive, at most maxq.
// Outputs: q, sigma (sqrt energy), slice and index of each kept term, est. dropped energy.
// One CTA, up to 4096 candidates (64 x 64).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
select_terms_kernel(const double* mu, int ldmu, const int* nslice, const int* nper, int smax,
                    int pmax, const double* core_e, double frac2, int maxq, int* q_out,
                    double* sigma, int* tslice, int* tidx, double* dropped)
{
    __shared__ double key[4096];
    __shared__ short val[4096];                 // candidate index (< 4096), -1 for padding
    const int ns = min(*nslice, smax), np = min(*nper, pmax);
    const int tot = ns * np;
    int P = 1;
    while (P < tot) P <<= 1;
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        if (e < tot) {
            int s = e / np, i = e - s * np;
            key[e] = fmax(mu[(long long)s * ldmu + i], 0.0);
            val[e] = (short)e;
        } else { key[e] = -1.0; val[e] = -1; }
    }
    __syncthreads();
    // bitonic sort, descending by key, ties by ascending val
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int e = threadIdx.x; e < P; e += blockDim.x) {
                int o = e ^ j;
                if (o > e) {
                    bool desc = ((e & k) == 0);
                    double ke = key[e], ko = key[o];
                    short ve = val[e], vo = val[o];
                    bool eFirst = (ke > ko) || (ke == ko && ve < vo);
                    bool swap = desc ? !eFirst : eFirst;
                    if (swap) { key[e] = ko; key[o] = ke; val[e] = vo; val[o] = ve; }
                }
            }
            __syncthreads();
        }
    }
    // Tails T[t] = sum_{t' >= t} key[t'] of the sorted energies (block-wide suffix scan: each
    // thread owns kPer consecutive entries, T[tot] = 0).  The terms kept are the shortest
    // prefix whose tail is within thr (T is non-increasing, so the first t with T[t] <= thr),
    // at least one term if any energy is positive, at most maxq, and no zero-energy term.
    constexpr int kPer = 4;                     // 4096 entries / 1024 threads
    __shared__ double wsum[32];
    __shared__ int s_first, s_pos;
    __shared__ double s_tail;
    const double thr = frac2 * (*core_e);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int e0 = tid * kPer;
    double own = 0.0;
    for (int u = 0; u < kPer; ++u)
        if (e0 + u < tot) own += key[e0 + u];
    // inclusive suffix within the warp, then the sums of the warps after this one
    double suf = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_down_sync(0xffffffffu, suf, o);
        if (lane + o < 32) suf += v;
    }
    if (lane == 0) wsum[wid] = suf;
    if (tid == 0) { s_first = tot; s_pos = tot; }
    __syncthreads();
    double after = suf - own;                   // entries of later threads in this warp
    for (int w2 = wid + 1; w2 < nw; ++w2) after += wsum[w2];
    double T[kPer];
    double run = after;
    for (int u = kPer - 1; u >= 0; --u) {
        const int e = e0 + u;
        if (e < tot) run += key[e];
        T[u] = run;                             // T[e0 + u]
    }
    for (int u = 0; u < kPer; ++u) {
        const int e = e0 + u;
        if (e >= tot) break;
        if (T[u] <= thr) atomicMin(&s_first, e);
        if (!(key[e] > 0.0)) atomicMin(&s_pos, e);
    }
    __syncthreads();
    int q = s_first;
    if (q < 1 && tot > 0 && key[0] > 0.0) q = 1;
    if (q > maxq) q = maxq;
    if (tid == 0 && q >= tot) s_tail = 0.0;
    if (q >= e0 && q < e0 + kPer && q < tot) s_tail = T[q - e0];
    q = min(q, s_pos);                          // zero-energy terms drop for free
    __syncthreads();
    if (tid == 0) {
        *q_out = q;
        *dropped = s_tail;
    }
    for (int t = threadIdx.x; t < q; t += blockDim.x) {
        int e = val[t];
        int s = e / np;
        sigma[t] = sqrt(key[t]);
        tslice[t] = s;
        tidx[t] = e - s * np;
    }
}

void launch_select_terms(cudaStream_t st, const double* mu, int ldmu, const int* nslice,
                         const int* nper, int smax, int pmax, const double* core_e, double frac2,
                         int maxq, int* q_out, double* sigma, int* tslice, int* tidx,
                         double* dropped)
{
    note_launch(); select_terms_kernel<<<1, 1024, 0, st>>>(mu, ldmu, nslice, nper, smax, pmax, core_e, frac2, maxq,
                                            q_out, sigma, tslice, tidx, dropped);
}

}  // namespace fc
