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
//
// One CTA of four warps per matrix, one block barrier per pivot step.  GB300 issues FP64 FMAs
// at about half a lane per clock per SM sub-partition and a dependent FP64 operation takes
// ~64 cycles, so the work of every step is spread over all four warps with every lane busy,
// and the steps are kept short:
//  * the remaining rows are a 64-bit mask held by every thread (no shared list); the g-th
//    remaining row is the g-th set bit;
//  * step k: every warp finds the pivot pk (largest remaining diagonal, ties: smallest
//    index); the R other remaining rows go to groups of tpr threads (the largest power of
//    two with tpr * R <= 128, dealt round robin over the warps) for
//    L[o,k] = (M[o,pk] - sum_{j<k} L[o,j] L[pk,j]) / L[pk,pk] (every tpr-th j per thread,
//    combined by shuffles; M is copied to shared memory once);
//  * in the same step, row k-1 of L11^{-1} (pivot order):
//    Li[i,j] = -(sum_{t=j}^{i-1} L[i,t] Li[t,j]) / L[i,i], outputs j and i-1-j paired so every
//    group has i + 1 terms.
// Rows of L are kept by original index (no row swaps).
// ---------------------------------------------------------------------------------------
constexpr int kPcThreads = 128;

// Index of the g-th (from 0) set bit of m (m has more than g bits set).
FC_DEV int nth_set_bit(unsigned long long m, int g) {
    unsigned w = (unsigned)m;
    int base = 0, r = g;
    const int pl = __popc(w);
    if (r >= pl) { r -= pl; w = (unsigned)(m >> 32); base = 32; }
    int p = __popc(w & 0xFFFFu);
    if (r >= p) { r -= p; w >>= 16; base += 16; }
    p = __popc(w & 0xFFu);
    if (r >= p) { r -= p; w >>= 8; base += 8; }
    p = __popc(w & 0xFu);
    if (r >= p) { r -= p; w >>= 4; base += 4; }
    p = __popc(w & 0x3u);
    if (r >= p) { r -= p; w >>= 2; base += 2; }
    if (r >= (int)(w & 1u)) base += 1;
    return base;
}

// Row i of L11^{-1} (pivot order) from rows 0..i-1 and row i of L; see the kernel's comment.
FC_DEV void pchol_inverse_row(int i, const double* Lo, double* Li, const int* piv,
                              const double* invd, int lane, int wid)
{
    constexpr int SS = kMaxC + 1;
    const unsigned full = 0xffffffffu;
    const double* Lr = Lo + piv[i] * SS;
    const int np = (i + 1) / 2;            // pairs of outputs j < i
    int tpr = 32;
    while (tpr > 1 && tpr * np > kPcThreads) tpr >>= 1;
    const int slot = lane / tpr, sub = lane - slot * tpr, g = slot * 4 + wid;
    double acc_a = 0.0, acc_b = 0.0;
    int a = -1, bb = -1;
    if (g < np) {
        a = g;
        bb = i - 1 - g;                    // == a for the middle output of an odd i
        const int na = i - a, ntot = (bb == a) ? na : i + 1;
        int u = sub;
        for (; u < na; u += tpr) acc_a = fma(Lr[a + u], Li[(a + u) * SS + a], acc_a);
        for (; u < ntot; u += tpr) {
            const int t = bb + (u - na);
            acc_b = fma(Lr[t], Li[t * SS + bb], acc_b);
        }
    }
    for (int off = tpr >> 1; off > 0; off >>= 1) {
        acc_a += __shfl_xor_sync(full, acc_a, off);
        acc_b += __shfl_xor_sync(full, acc_b, off);
    }
    if (a >= 0 && sub == 0) {
        Li[i * SS + a] = -invd[i] * acc_a;
        if (bb != a) Li[i * SS + bb] = -invd[i] * acc_b;
    }
    if (lane == 0 && wid == 0) Li[i * SS + i] = invd[i];
}

__global__ void __launch_bounds__(kPcThreads)
pchol_kernel(const double* __restrict__ M, int ldm, long long bsM, const int* dims, int dstride,
             int cmax, double relTol, double* __restrict__ T, int ldt, long long bsT,
             int* rank, int rstride)
{
    extern __shared__ double sm[];
    constexpr int SS = kMaxC + 1;
    double* Lo = sm;                   // Lo[o*SS + j]: L of original row o, pivot step j
    double* Li = Lo + kMaxC * SS;      // Li[i*SS + j]: (L11^{-1})[i, j], pivot order
    double* Ms = Li + kMaxC * SS;      // Ms[o*SS + p] = M[o, p] (an L2 read per step would sit
                                       // on the critical path)
    // remaining diagonal by original index, double-buffered: step k reads dg[k & 1] (every
    // warp's pivot search) and its updates go to dg[(k + 1) & 1], so no warp can see a value
    // of step k's updates while another still searches
    __shared__ double dg[2][kMaxC];
    __shared__ double invd[kMaxC];     // 1 / L[k, k] (one reciprocal square root per pivot)
    __shared__ int piv[kMaxC];         // original index of pivot k
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int b = blockIdx.x;
    int c = cmax;
    if (dims) c = min(dims[b * dstride], cmax);
    if (c < 0) c = 0;
    const double* Mb = M + b * bsM;
    for (int e = tid; e < c * c; e += kPcThreads) {
        const int i = e % c, j = e / c;
        Ms[i * SS + j] = Mb[i + (long long)j * ldm];
    }
    __syncthreads();
    for (int i = tid; i < c; i += kPcThreads) dg[0][i] = Ms[i * SS + i];
    __syncthreads();
    double mx = 0.0;
    for (int i = lane; i < c; i += 32) mx = fmax(mx, dg[0][i]);
    const double dmax0 = warp_max(mx);      // every warp alike
    unsigned long long rem = (c >= 64) ? ~0ull : ((1ull << c) - 1ull);   // remaining rows
    int rk = c;
    for (int k = 0; k <= c; ++k) {
        if (k > 0) pchol_inverse_row(k - 1, Lo, Li, piv, invd, lane, wid);
        if (k == c) break;
        // pivot: largest remaining diagonal (ties: smallest original index), every warp alike
        const double* dcur = dg[k & 1];
        double* dnxt = dg[(k + 1) & 1];
        double best = -1.0;
        int bo = kMaxC;
        for (int o = lane; o < c; o += 32)
            if ((rem >> o) & 1ull) {
                const double v = dcur[o];
                if (v > best || (v == best && o < bo)) { best = v; bo = o; }
            }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ob = __shfl_xor_sync(full, best, off);
            const int oo = __shfl_xor_sync(full, bo, off);
            if (ob > best || (ob == best && oo < bo)) { best = ob; bo = oo; }
        }
        if (!(best > relTol * dmax0) || !(best > 0.0)) { rk = k; break; }   // uniform
        const int pk = bo;
        rem &= ~(1ull << pk);
        // the R other remaining rows: group g = slot * 4 + warp, slot = lane / tpr
        const int R = __popcll(rem);
        int tpr = 32;
        while (tpr > 1 && tpr * R > kPcThreads) tpr >>= 1;
        const int slot = lane / tpr, sub = lane - slot * tpr, g = slot * 4 + wid;
        double s0 = 0.0, s1 = 0.0, mo = 0.0;
        int o = -1;
        if (g < R) {
            o = nth_set_bit(rem, g);
            if (sub == 0) mo = Ms[o * SS + pk];
            const double* Lr = Lo + o * SS;
            const double* Lk = Lo + pk * SS;
            int j = sub;
            for (; j + tpr < k; j += 2 * tpr) {
                s0 = fma(Lr[j], Lk[j], s0);
                s1 = fma(Lr[j + tpr], Lk[j + tpr], s1);
            }
            if (j < k) s0 = fma(Lr[j], Lk[j], s0);
        }
        const double ik = fc_rsqrt(best);
        double sdot = s0 + s1;
        for (int off = tpr >> 1; off > 0; off >>= 1) sdot += __shfl_xor_sync(full, sdot, off);
        if (o >= 0 && sub == 0) {
            const double l = (mo - sdot) * ik;
            Lo[o * SS + k] = l;
            dnxt[o] = dcur[o] - l * l;
        }
        if (tid == 0) {
            Lo[pk * SS + k] = best * ik;
            invd[k] = ik;
            piv[k] = pk;
        }
        __syncthreads();
    }
    __syncthreads();                       // the last inverse row
    const int r = rk;
    // R11^{-1} = (L11^T)^{-1} = (L11^{-1})^T ; T[piv[j], i] = Rinv[j, i] = Li[i, j]
    double* Tb = T + b * bsT;
    for (int e = tid; e < cmax * cmax; e += kPcThreads) Tb[(e % cmax) + (long long)(e / cmax) * ldt] = 0.0;
    __syncthreads();
    for (int e = tid; e < r * r; e += kPcThreads) {
        const int j = e % r, i = e / r;
        if (j <= i) Tb[piv[j] + (long long)i * ldt] = Li[i * SS + j];
    }
    if (tid == 0) rank[b * rstride] = r;
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
    note_launch(); pchol_kernel<<<batch, kPcThreads, sm, st>>>(M, ldm, bsM, dims, dstride, cmax,
                                                               relTol, T, ldt, bsT, rank, rstride);
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
