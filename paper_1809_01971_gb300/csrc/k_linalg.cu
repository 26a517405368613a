// Small dense FP64 linear algebra on one CTA per problem (sizes <= kMaxC = 64):
//   * cyclic two-sided Jacobi eigen-decomposition of symmetric matrices (the SVDs of the
//     RHOSVD truncation, Section 5, are taken through the eigen-decomposition of Grams),
//   * pivoted Cholesky orthonormaliser (range of a sketch, Gram-Schmidt by Cholesky),
//   * rank selection by the Frobenius tail rule and canonical-term selection.
#include "fc_common.cuh"
#include "fc_kernels.h"
#include <math.h>

namespace fc {

// ---------------------------------------------------------------------------------------
// Jacobi eigen-decomposition.  Item b: symmetric c x c matrix at A + b*bsA (ld lda),
// c = dims ? min(dims[b*dstride], cmax) : cmax.  Writes eigenvalues in descending order to
// ev + b*bsE (cmax entries, zero-padded) and the eigenvectors as columns of V + b*bsV
// (ld ldv, cmax x cmax, zero-padded).  Rounds follow the circle (round-robin) ordering so
// the m/2 rotations of a round are disjoint and are applied together.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
jacobi_eig_kernel(const double* __restrict__ A, int lda, long long bsA,
                  const int* __restrict__ dims, int dstride, int cmax,
                  double* __restrict__ ev, long long bsE,
                  double* __restrict__ V, int ldv, long long bsV, int maxSweeps, int prof)
{
    extern __shared__ double sm[];
    const int b = blockIdx.x;
    int c = cmax;
    if (dims) c = min(dims[b * dstride], cmax);
    if (c < 0) c = 0;
    (void)prof;
    const int m = (c + 1) & ~1;           // even number of players
    const int S = m + 1;                  // smem row stride
    double* a = sm;                       // m x S
    double* v = a + m * S;                // m x S
    double* coefS = v + m * S;            // self coefficient per index
    double* coefP = coefS + m;            // partner coefficient per index
    int* partner = (int*)(coefP + m);
    int* rotated = partner + m;           // per pair: rotation applied
    __shared__ double red[32];
    __shared__ int anyRot;

    const double* Ab = A + b * bsA;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        a[i * S + j] = (i < c && j < c) ? Ab[i + (long long)j * lda] : 0.0;
        v[i * S + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    double fro = 0.0;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        double x = a[(e % m) * S + e / m];
        fro += x * x;
    }
    fro = sqrt(block_sum(fro, red));
    const double absTol = 1e-18 * fro;
    const int half = m / 2;

    for (int sweep = 0; sweep < maxSweeps && m >= 2; ++sweep) {
        if (threadIdx.x == 0) anyRot = 0;
        __syncthreads();
        for (int rnd = 0; rnd < m - 1; ++rnd) {
            // rotation parameters, one thread per disjoint pair
            for (int i = threadIdx.x; i < half; i += blockDim.x) {
                int p, q;
                if (i == 0) { p = rnd; q = m - 1; }
                else { p = (rnd + i) % (m - 1); q = (rnd - i + (m - 1)) % (m - 1); }
                if (p > q) { int t = p; p = q; q = t; }
                double app = a[p * S + p], aqq = a[q * S + q], apq = a[p * S + q];
                double cs = 1.0, sn = 0.0;
                int rot = 0;
                double thr = fmax(2.2e-16 * sqrt(fabs(app * aqq)), absTol);
                if (fabs(apq) > thr) {
                    double th = (aqq - app) / (2.0 * apq);
                    double t;
                    if (fabs(th) > 1e150) t = 0.5 / th;
                    else t = copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
                    cs = 1.0 / sqrt(t * t + 1.0);
                    sn = t * cs;
                    rot = 1;
                }
                partner[p] = q; partner[q] = p;
                coefS[p] = cs; coefP[p] = -sn;
                coefS[q] = cs; coefP[q] = sn;
                rotated[i] = rot;
                if (rot) anyRot = 1;
            }
            __syncthreads();
            // A <- J^T A J on 2x2 blocks (pair I) x (pair J); in place, each block owned
            // by one thread.  Pair index of player x: position in the round (recomputed).
            for (int e = threadIdx.x; e < half * half; e += blockDim.x) {
                int pi = e % half, pj = e / half;
                int p1, q1, p2, q2;
                if (pi == 0) { p1 = rnd; q1 = m - 1; } else { p1 = (rnd + pi) % (m - 1); q1 = (rnd - pi + (m - 1)) % (m - 1); }
                if (pj == 0) { p2 = rnd; q2 = m - 1; } else { p2 = (rnd + pj) % (m - 1); q2 = (rnd - pj + (m - 1)) % (m - 1); }
                if (!rotated[pi] && !rotated[pj]) continue;
                int xs[2] = {p1, q1}, ys[2] = {p2, q2};
                double o[2][2];
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        int x = xs[u], y = ys[w];
                        int xp = partner[x], yp = partner[y];
                        double cx = coefS[x], sx = coefP[x], cy = coefS[y], sy = coefP[y];
                        o[u][w] = cx * (cy * a[x * S + y] + sy * a[x * S + yp]) +
                                  sx * (cy * a[xp * S + y] + sy * a[xp * S + yp]);
                    }
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int w = 0; w < 2; ++w) a[xs[u] * S + ys[w]] = o[u][w];
                if (pi == pj && rotated[pi]) {   // annihilated entry: exact zero
                    a[xs[0] * S + xs[1]] = 0.0;
                    a[xs[1] * S + xs[0]] = 0.0;
                }
            }
            // V <- V J: rows of V stored as v[row*S + col]
            for (int e = threadIdx.x; e < m * half; e += blockDim.x) {
                int r = e % m, pi = e / m;
                if (!rotated[pi]) continue;
                int p, q;
                if (pi == 0) { p = rnd; q = m - 1; } else { p = (rnd + pi) % (m - 1); q = (rnd - pi + (m - 1)) % (m - 1); }
                double vp = v[r * S + p], vq = v[r * S + q];
                v[r * S + p] = coefS[p] * vp + coefP[p] * vq;
                v[r * S + q] = coefS[q] * vq + coefP[q] * vp;
            }
            __syncthreads();
        }
        if (!anyRot) break;
        __syncthreads();
    }
    // sort descending (rank by counting; ties by index), write padded outputs
    double* evb = ev + b * bsE;
    double* Vb = V + b * bsV;
    for (int e = threadIdx.x; e < cmax * cmax; e += blockDim.x) Vb[(e % cmax) + (long long)(e / cmax) * ldv] = 0.0;
    for (int i = threadIdx.x; i < cmax; i += blockDim.x) evb[i] = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
        double di = a[i * S + i];
        int rk = 0;
        for (int j = 0; j < c; ++j) {
            double dj = a[j * S + j];
            rk += (dj > di) || (dj == di && j < i);
        }
        evb[rk] = di;
        for (int r = 0; r < c; ++r) Vb[r + (long long)rk * ldv] = v[r * S + i];
    }
}

size_t jacobi_smem(int cmax) {
    int m = (cmax + 1) & ~1;
    return sizeof(double) * (2 * (size_t)m * (m + 1) + 2 * m) + sizeof(int) * 2 * m;
}

void launch_jacobi(cudaStream_t st, int batch, const double* A, int lda, long long bsA,
                   const int* dims, int dstride, int cmax, double* ev, long long bsE,
                   double* V, int ldv, long long bsV)
{
    if (batch <= 0) return;
    size_t sm = jacobi_smem(cmax);
    note_launch(); jacobi_eig_kernel<<<batch, 256, sm, st>>>(A, lda, bsA, dims, dstride, cmax, ev, bsE, V, ldv,
                                               bsV, 30, 0);
}

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
        const double lkk = sqrt(best);
        const double ik = 1.0 / lkk;
        if (lane == 0) { L[k * SS + k] = lkk; invd[k] = ik; }
        const int pk = perm[k];
        for (int i = k + 1 + lane; i < c; i += 32) {
            double s0 = Mi[perm[i] * SS + pk];
            for (int j = 0; j < k; ++j) s0 = fma(-L[i * SS + j], L[k * SS + j], s0);
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
            double s0 = 0.0;
            for (int t = j; t < i; ++t) s0 = fma(-L[i * SS + t], Li[t * SS + j], s0);
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
    cudaError_t e = cudaFuncSetAttribute(jacobi_eig_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)jacobi_smem(kMaxC));
    if (e != cudaSuccess) return e;
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
    __shared__ int val[4096];
    const int ns = min(*nslice, smax), np = min(*nper, pmax);
    const int tot = ns * np;
    int P = 1;
    while (P < tot) P <<= 1;
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        if (e < tot) {
            int s = e / np, i = e - s * np;
            key[e] = fmax(mu[(long long)s * ldmu + i], 0.0);
            val[e] = e;
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
                    int ve = val[e], vo = val[o];
                    bool eFirst = (ke > ko) || (ke == ko && ve < vo);
                    bool swap = desc ? !eFirst : eFirst;
                    if (swap) { key[e] = ko; key[o] = ke; val[e] = vo; val[o] = ve; }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        double thr = frac2 * (*core_e);
        // suffix sums from the end: drop while cumulative tail <= thr
        int q = tot;
        double tail = 0.0;
        while (q > 0 && tail + key[q - 1] <= thr) { tail += key[q - 1]; --q; }
        if (q < 1 && tot > 0 && key[0] > 0.0) q = 1;
        while (q > maxq) { tail += key[q - 1]; --q; }
        // never keep zero-energy terms
        while (q > 0 && !(key[q - 1] > 0.0)) --q;
        *q_out = q;
        *dropped = tail;
    }
    __syncthreads();
    const int q = *q_out;
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
